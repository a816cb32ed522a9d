"""Learned warm start for the 2D 256^2 workload: data, training and evaluation driver.

Everything numerical runs in the library's kernels: pcg_solve makes the training pairs, the
ws_* calls run the U-Net (forward, backward, Adam) and the prediction.  This module only
orchestrates them.

  python -m paper_2108_12574_gb300.warmstart train   # writes weights/ws_unet_n256.f32
  python -m paper_2108_12574_gb300.warmstart eval    # zero start vs warm start on held-out fields

Workload: 256 x 256 cell-centred grid, Schwarz preconditioner with 16 x 16 partitions extended
by 2 cells (the 512^2 solver's partition size), FP32 factors.  Training right-hand sides are
Gaussian random fields with length scale l uniform in [0.03, 0.3] (drawn from SplitMix64 with
the field's seed), seeds 1000 + k; the reference solutions are solved to a true relative
residual of 1e-10.  The eight symmetries of the square map solutions to solutions (A commutes
with them), which multiplies the training set by eight.  Held-out fields use seeds 0..255.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights", "ws_unet_n256.f32")
N_GRID, M_PART, DELTA = 256, 16, 2
ELL_LO, ELL_HI = 0.03, 0.3


def ell_of(seed: int) -> float:
    from . import inputs as I
    return ELL_LO + (ELL_HI - ELL_LO) * float(I.unit_doubles(seed ^ 0x5EED, 1)[0])


def fields(seeds, n=N_GRID):
    from . import inputs as I
    return np.stack([I.grf(2, n, ell_of(s), s) for s in seeds])


def setup(n=N_GRID, device=0):
    from . import iedd
    prob = iedd.ie_discretize(2, n, device=device)
    part = iedd.dd_partition(prob, n // 16, DELTA, iedd.DD_SCHWARZ)
    fac = iedd.dd_factor(prob, part, iedd.IE_MIXED)
    return prob, part, fac


def solve_batch(prob, fac, F, tol):
    """Solutions (torch, device) of A u = f for the rows of F (torch, device)."""
    import torch

    from . import iedd
    U = torch.zeros_like(F)
    reps = iedd.pcg_solve(prob, fac, F, U, tol=tol, precision=iedd.IE_MIXED, check=False)
    return U, reps


def symmetries(X, n):
    """The 8 images of each row of X (rows are n x n grids) under the symmetries of the square."""
    import torch
    G = X.reshape(-1, n, n)
    outs = []
    for k in range(4):
        R = torch.rot90(G, k, dims=(1, 2))
        outs.append(R)
        outs.append(torch.flip(R, dims=(2,)))
    return torch.cat([o.reshape(-1, n * n) for o in outs], dim=0)


def make_dataset(count=512, tol=1e-10, n=N_GRID, log=print):
    import torch
    prob, part, fac = setup(n)
    seeds = [1000 + k for k in range(count)]
    F = torch.from_numpy(fields(seeds, n)).cuda()
    U = torch.empty_like(F)
    t0 = time.time()
    its = []
    for b0 in range(0, count, 16):
        Ub, reps = solve_batch(prob, fac, F[b0:b0 + 16].contiguous(), tol)
        U[b0:b0 + 16] = Ub
        its += [r["iterations"] for r in reps]
    log(f"solved {count} training fields in {time.time() - t0:.1f}s, mean iterations {np.mean(its):.1f}")
    return prob, F, U


def train(model, prob, F, U, epochs=20, batch=16, lr=1e-3, seed=0, log=print):
    import torch
    n = prob.n
    Fa, Ua = symmetries(F, n), symmetries(U, n)
    g = torch.Generator(device="cpu").manual_seed(seed)
    steps = epochs * (Fa.shape[0] // batch)
    hist = []
    step = 0
    t0 = time.time()
    for ep in range(epochs):
        perm = torch.randperm(Fa.shape[0], generator=g).cuda()
        ep_loss = []
        for b0 in range(0, Fa.shape[0] - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            fb, ub = Fa[idx].contiguous(), Ua[idx].contiguous()
            cur = lr * 0.5 * (1 + np.cos(np.pi * step / steps))
            ep_loss.append(model.train_step(prob, fb, ub, float(cur)))
            step += 1
        hist.append(float(np.mean(ep_loss)))
        log(f"epoch {ep + 1}/{epochs}: loss {hist[-1]:.4e} ({time.time() - t0:.1f}s)")
    return hist


def evaluate(model, prob, fac, seeds, tol=1e-8):
    """Per field: iterations and GPU time (s) to tol from zero and from the network's u0
    (ws_predict + pcg_solve with the fallback start), and the relative residual of u0."""
    import torch

    from . import iedd
    F = torch.from_numpy(fields(seeds, prob.n)).cuda()
    rows = []
    for k in range(F.shape[0]):
        f = F[k].contiguous()
        u = torch.zeros_like(f)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r0 = iedd.pcg_solve(prob, fac, f, u, tol=tol, precision=iedd.IE_MIXED)[0]
        torch.cuda.synchronize()
        t_zero = time.perf_counter() - t0
        u0 = torch.zeros_like(f)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        model.predict(prob, f, u0)
        r1 = iedd.pcg_solve(prob, fac, f, u0, tol=tol, precision=iedd.IE_MIXED, use_x0=2)[0]
        torch.cuda.synchronize()
        t_warm = time.perf_counter() - t0
        # relative residual of the prediction alone
        up = torch.zeros_like(f)
        model.predict(prob, f, up)
        au = torch.zeros_like(f)
        iedd.ie_matvec(prob, up, au, iedd.IE_ACCURATE)
        rel0 = float(torch.linalg.norm(f - au) / torch.linalg.norm(f))
        rows.append({"seed": int(seeds[k]), "it_zero": r0["iterations"], "it_warm": r1["iterations"],
                     "t_zero": t_zero, "t_warm": t_warm, "relres_u0": rel0, "x0_used": r1["x0_used"],
                     "true_zero": r0["true_relres"], "true_warm": r1["true_relres"]})
    return rows


def summarize(rows):
    a = lambda k: float(np.mean([r[k] for r in rows]))
    return {"fields": len(rows), "iterations_zero": a("it_zero"), "iterations_warm": a("it_warm"),
            "time_zero_s": a("t_zero"), "time_warm_s": a("t_warm"), "speedup": a("t_zero") / a("t_warm"),
            "median_relres_u0": float(np.median([r["relres_u0"] for r in rows])),
            "fallbacks": int(sum(1 - r["x0_used"] for r in rows)),
            "max_true_relres_warm": float(max(r["true_warm"] for r in rows))}


def load_model(path=WEIGHTS, device=0):
    from . import iedd
    model = iedd.ws_create(device, 0)
    theta = np.fromfile(path, dtype=np.float32)
    model.set_params(theta)
    return model


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train", "eval"])
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=20)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--eval-fields", type=int, default=256)
    ap.add_argument("--out", default=WEIGHTS)
    a = ap.parse_args(argv)
    import torch
    torch.cuda.init()
    from . import build, iedd
    build.build()
    if a.cmd == "train":
        prob, F, U = make_dataset(a.count)
        model = iedd.ws_create(0, 12345)
        hist = train(model, prob, F, U, epochs=a.epochs, lr=a.lr)
        os.makedirs(os.path.dirname(a.out), exist_ok=True)
        model.get_params().astype(np.float32).tofile(a.out)
        json.dump({"loss_history": hist, "count": a.count, "epochs": a.epochs, "lr": a.lr, "n": N_GRID},
                  open(a.out + ".json", "w"), indent=1)
        print(f"wrote {a.out}")
    prob, part, fac = setup()
    model = load_model(a.out)
    rows = evaluate(model, prob, fac, list(range(a.eval_fields)))
    print(json.dumps(summarize(rows)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
