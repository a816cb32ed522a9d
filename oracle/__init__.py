"""FP64 CPU oracle (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline and
reference legs may import, call, link or execute anything under ``oracle/``.  The
CUDA library never uses it and shares no code with it.
"""
