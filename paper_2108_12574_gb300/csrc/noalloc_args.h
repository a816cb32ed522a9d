// Argument checks of ie_matvec_noalloc, written without any CUDA call so that a host-only
// program can include this header and test every rejection without a GPU.  The caller gathers
// the facts that need the CUDA runtime (which device is current, where x, y and the stream
// live) and this function decides.
#ifndef IEDD_NOALLOC_ARGS_H
#define IEDD_NOALLOC_ARGS_H

#include <cmath>
#include <cstdint>

struct NoallocArgs {
    int dim, n, grid;
    double a_shift;
    const void *x, *y;
    int dev_current;  // cudaGetDevice
    int x_device;     // device that owns x's memory, -1 for host or unregistered memory
    int y_device;     // the same for y
    int stream_device;  // device of the caller's stream (cudaStreamGetDevice)
};

// Returns 0 and N = n^dim when the call may proceed; else -1 (IE_ERR_ARG) with *why set.
// grid: 0 (text) or 1 (table); max_n: the largest N the static scratch array holds.
inline int noalloc_check_args(const NoallocArgs &a, long long max_n, long long *N_out, const char **why) {
    if (a.dim != 2 && a.dim != 3) { *why = "dim must be 2 or 3"; return -1; }
    if (a.n < 2) { *why = "n must be >= 2"; return -1; }
    if (a.grid != 0 && a.grid != 1) { *why = "unknown grid convention"; return -1; }
    if (!std::isfinite(a.a_shift)) { *why = "a_shift must be finite"; return -1; }
    long long N = 1;
    for (int d = 0; d < a.dim; ++d) {
        N *= a.n;
        if (N > max_n) { *why = "N = n^dim exceeds the limit of the static scratch array"; return -1; }
    }
    if (!a.x || !a.y) { *why = "NULL vector"; return -1; }
    if (a.x_device < 0 || a.y_device < 0) {
        *why = "x and y must be device memory (host data would need staging)";
        return -1;
    }
    if (a.x_device != a.dev_current || a.y_device != a.dev_current) {
        *why = "x and y must be memory of the current device";
        return -1;
    }
    if (a.stream_device != a.dev_current) { *why = "the stream belongs to another device"; return -1; }
    const uintptr_t px = reinterpret_cast<uintptr_t>(a.x), py = reinterpret_cast<uintptr_t>(a.y);
    const uintptr_t bytes = static_cast<uintptr_t>(8 * N);
    if (px < py + bytes && py < px + bytes) { *why = "x and y overlap"; return -1; }
    *N_out = N;
    return 0;
}

#endif  // IEDD_NOALLOC_ARGS_H
