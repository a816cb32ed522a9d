"""Recursive skeletonization (RS) of the CBD subproblems -- plain FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this module.  It shares no code with
the CUDA library in ``paper_2108_12574_gb300/`` and never imports it.

What it follows: Sec. 4.3 ("Recursive skeletonization (RS) as subdomain solver", Eqs.
e:oi, e:block, e:id, e:id_err, e:al, e:alu, e:b, e:schur) applied to every subdomain
A_c = R_c A R_c^T of the colouring-based decomposition (Eq. e:second, D = 2^d), and the
additive preconditioner of Eq. e:ad built from those approximate factors.

For one colour subdomain the factorization runs level by level:
  * level 1: the regions are the extended boxes of that colour (Eq. e:oi);
  * at every level, for every region p (its DOFs: all of its points at level 1, the
    skeletons its children kept above), the interpolative decomposition of A_qp, q = the
    DOFs of the other regions of the subdomain (Eq. e:id), computed through the proxy
    trick; then compress-then-eliminate (Eqs. e:al, e:alu, e:b), which leaves the
    skeleton block B_ss and does not touch A_qq, A_qs (Eq. e:schur);
  * the regions are merged 2^d at a time (spatially close ones) and the process repeats
    until one region remains; its Schur complement is factored by dense Cholesky.
The application of A_c^{-1} is R diag(I, S^{-1}) R^T with R the product of the
operators L_p U_r (Eq. e:alu), recursively.

Readings where the paper is silent (each also listed in the design notes):
  * The regions of one colour are disjoint only when 2 delta <= w; that is required.
  * Proxy surface: a circle (2D) or sphere (3D) centred on the region's bounding box (in
    grid points), radius rho times the box's longest side (rho = 1.5, the value the
    paper's footnote gives), with P points uniform in angle (2D) or on a Fibonacci lattice
    (3D).  The DOFs of other regions strictly inside it enter the ID as explicit rows of
    A (near field); the proxy rows are h^d K(x_proxy - y).  Inside/outside is decided in
    lattice units (exact for rho = 1.5).
  * 2D adds one row of constants to the proxy rows: the log kernel's far field has a
    monopole term that point values on one circle do not control.
  * The ID is column-pivoted Gram-Schmidt (the pivoted QR the paper cites for the ID).
    The squared column norms are recomputed after every step.  The pivot is the
    lowest-index column whose squared norm nu_j is at least top - w, top the largest,
    w = min(top / 2, max(tau top, tau_abs nu0)) (nu0: the largest squared norm before the
    first step; tau = 1e-10, tau_abs = 1e-13), so that the exact ties of the symmetric
    grid break the same way under any rounding order (rounding moves nu_j by far less
    than w).  It stops when the largest remaining norm is at most eps * sqrt(nu0)
    (Eq. e:id_err's relative accuracy).
  * DOF order: ascending global index inside a level-1 region; a merged region lists its
    children's skeletons in child order (row-major colour-grid coordinate), each child's
    in pivot order; redundant DOFs keep their relative order.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
import scipy.linalg

from oracle import ie_oracle as O

TAU = 1e-10
TAU_ABS = 1e-13


# ---------------------------------------------------------------------------
# Regions of the colour subdomains (Eqs. e:oi, e:second)
# ---------------------------------------------------------------------------

def colour_regions(dim: int, n: int, m: int, delta: int):
    """For every colour (k_1 mod 2, ..., k_d mod 2) in row-major order, the list of its
    level-1 regions: dicts with ``points`` (ascending global indices), ``lo``/``hi``
    (the clipped extended box, grid indices, hi exclusive) and ``K`` (the colour-grid
    coordinate k // 2).  Regions are listed row-major by K."""
    if m < 1 or n % m != 0:
        raise ValueError("n must be a multiple of m")
    w = n // m
    if delta < 0 or 2 * delta > w:
        raise ValueError("RS needs 0 <= 2 delta <= w (disjoint regions in a colour)")
    out = []
    for colour in itertools.product(range(2), repeat=dim):
        regs = []
        for K in itertools.product(*[range((m - c + 1) // 2) for c in colour]):
            k = [2 * KK + c for KK, c in zip(K, colour)]
            lo = [max(kk * w - delta, 0) for kk in k]
            hi = [min((kk + 1) * w + delta, n) for kk in k]
            mesh = np.meshgrid(*[np.arange(a, b) for a, b in zip(lo, hi)], indexing="ij")
            idx = np.zeros(mesh[0].shape, dtype=np.int64)
            for a in mesh:
                idx = idx * n + a
            regs.append(dict(points=idx.reshape(-1), lo=np.array(lo), hi=np.array(hi), K=np.array(K)))
        out.append(regs)
    return out


def proxy_directions(dim: int, nproxy: int) -> np.ndarray:
    """Unit vectors of the proxy surface: 2D angles 2 pi j / P; 3D the Fibonacci lattice
    z_j = 1 - (2 j + 1) / P, azimuth j * pi (3 - sqrt 5)."""
    j = np.arange(nproxy, dtype=np.float64)
    if dim == 2:
        t = 2.0 * math.pi * j / nproxy
        return np.stack([np.cos(t), np.sin(t)], axis=1)
    z = 1.0 - (2.0 * j + 1.0) / nproxy
    rho = np.sqrt(np.maximum(1.0 - z * z, 0.0))
    phi = j * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([rho * np.cos(phi), rho * np.sin(phi), z], axis=1)


# ---------------------------------------------------------------------------
# Interpolative decomposition (Eqs. e:id, e:id_err) by column-pivoted Gram-Schmidt
# ---------------------------------------------------------------------------

def interp_decomp(Y: np.ndarray, eps: float, tau: float = TAU):
    """Split the columns of Y into skeletons s (pivot order) and redundant r (ascending)
    with Y[:, r] ~ Y[:, s] T, T = R11^{-1} R12 from the pivoted Gram-Schmidt factors."""
    Y = np.array(Y, dtype=np.float64, copy=True)
    rows, ncol = Y.shape
    nu = np.einsum("ij,ij->j", Y, Y)
    nu0 = float(nu.max()) if ncol else 0.0
    steps = min(rows, ncol)
    coef = np.zeros((steps, ncol))
    chosen = np.zeros(ncol, dtype=bool)
    skel = []
    if nu0 > 0.0:
        for step in range(steps):
            cand = np.flatnonzero(~chosen)
            top = nu[cand].max()
            if top <= eps * eps * nu0:
                break
            window = min(0.5 * top, max(tau * top, TAU_ABS * nu0))
            j = int(cand[nu[cand] >= top - window][0])
            norm = math.sqrt(nu[j])
            q = Y[:, j] / norm
            coef[step, j] = norm
            chosen[j] = True
            skel.append(j)
            rest = np.flatnonzero(~chosen)
            if rest.size == 0:
                break
            r = q @ Y[:, rest]
            Y[:, rest] -= np.outer(q, r)
            coef[step, rest] = r
            nu[rest] = np.einsum("ij,ij->j", Y[:, rest], Y[:, rest])
    skel = np.array(skel, dtype=np.int64)
    red = np.flatnonzero(~chosen)
    k = skel.size
    if k and red.size:
        T = scipy.linalg.solve_triangular(coef[:k][:, skel], coef[:k][:, red], lower=False)
    else:
        T = np.zeros((k, red.size))
    return skel, red, T


# ---------------------------------------------------------------------------
# Compress-then-eliminate (Eqs. e:al, e:alu, e:b)
# ---------------------------------------------------------------------------

def eliminate(D: np.ndarray, skel, red, T: np.ndarray):
    """With L_p (block (s, r) = -T) and U_r of Eq. e:alu on the region's block D:
    B_rr = D_rr - D_rs T - T^T D_sr + T^T D_ss T,  B_sr = D_sr - D_ss T,
    B_rr = L L^T (Cholesky),  X = B_rr^{-1} B_rs,  B_ss = D_ss - B_sr X  (Eq. e:b)."""
    Dss = D[np.ix_(skel, skel)]
    Dsr = D[np.ix_(skel, red)]
    Drr = D[np.ix_(red, red)]
    Brr = Drr - Dsr.T @ T - T.T @ Dsr + T.T @ Dss @ T
    Bsr = Dsr - Dss @ T
    L = O.cholesky(Brr)
    Linv = scipy.linalg.solve_triangular(L, np.eye(L.shape[0]), lower=True)
    Binv = Linv.T @ Linv
    X = Binv @ Bsr.T
    Bss = Dss - Bsr @ X
    return dict(L=L, Binv=Binv, Bsr=Bsr, X=X, Bss=Bss)


# ---------------------------------------------------------------------------
# The factorization of one colour subdomain and of the whole preconditioner
# ---------------------------------------------------------------------------

_GRIDS = {}


def _grid(dim, n, convention):
    """(points, lattice indices) of the grid, kept per (dim, n, convention)."""
    key = (dim, n, convention)
    if key not in _GRIDS:
        _GRIDS.clear()
        _GRIDS[key] = (O.points(dim, n, convention), O.lattice(dim, n))
    return _GRIDS[key]


def _entries(P, weight, diag, rows, cols):
    """A[rows, cols] (global indices); the diagonal value where a row equals a column."""
    d = P[rows][:, None, :] - P[cols][None, :, :]
    r = np.sqrt((d * d).sum(axis=2))
    same = rows[:, None] == cols[None, :]
    r = np.where(same, 1.0, r)
    return np.where(same, diag, weight * O.kernel(P.shape[1], r))


def id_matrix(dim, n, lo, hi, own, others, nproxy, rho=1.5, convention=O.GRID_TEXT):
    """The matrix whose columns the ID of a region splits (Eq. e:id through the proxy trick).

    own: the region's DOFs (global points, columns); others: the DOFs of the other regions of
    the subdomain at this level.  Rows: h^d K(x_proxy - y) for the P proxy points on the
    circle / sphere of radius rho W around the box [lo, hi) (W its longest side, lattice
    units), in 2D a row of h^d, then A[near, own] for the DOFs of ``others`` strictly inside
    the proxy surface.  Returns (Y, near)."""
    spacing, offset, weight, _ = O.grid_geometry(dim, n, convention)
    diag = O.diagonal(dim, n, 0.0)
    P, lat = _grid(dim, n, convention)
    lo, hi = np.asarray(lo), np.asarray(hi)
    W = int((hi - lo).max())
    twice_ctr = lo + hi - 1                                   # 2 x centre, lattice units
    others = np.asarray(others, dtype=np.int64)
    d2 = ((2 * lat[others] - twice_ctr) ** 2).sum(axis=1)       # (2 |x - centre|)^2
    near = others[d2 < (2.0 * rho * W) ** 2]
    centre = offset + spacing * 0.5 * twice_ctr
    prox = centre + rho * W * spacing * proxy_directions(dim, nproxy)
    xp = P[np.asarray(own)]
    dp = prox[:, None, :] - xp[None, :, :]
    rows = [weight * O.kernel(dim, np.sqrt((dp * dp).sum(axis=2)))]
    if dim == 2:
        rows.append(np.full((1, xp.shape[0]), weight))
    if near.size:
        rows.append(_entries(P, weight, diag, near, np.asarray(own)))
    return np.vstack(rows), near


def level1_id(dim, n, m, delta, colour, index, eps, nproxy, rho=1.5, convention=O.GRID_TEXT, tau=TAU):
    """The level-1 ID of one region alone (region ``index`` of colour ``colour``, as listed by
    colour_regions): (its points with the skeletons first in pivot order, then the redundant
    ones; rank).  Level 1's IDs do not depend on one another."""
    regs = colour_regions(dim, n, m, delta)[colour]
    r = regs[index]
    others = np.concatenate([o["points"] for i, o in enumerate(regs) if i != index])
    Y, _ = id_matrix(dim, n, r["lo"], r["hi"], r["points"], others, nproxy, rho, convention)
    skel, red, _ = interp_decomp(Y, eps, tau)
    return np.concatenate([r["points"][skel], r["points"][red]]), int(skel.size)


def factor_colour(dim, n, regions, eps, nproxy, rho=1.5, convention=O.GRID_TEXT, a_shift=0.0,
                  tau=TAU):
    """RS factorization of A_c for the colour whose level-1 regions are ``regions``.

    Returns dict(points = the colour's points in local order (global indices), levels =
    per compression level the list of region records (dofs: local positions, skel, red,
    T, Binv, Bsr, X), top = dict(dofs, L) of the last Schur complement)."""
    _, _, weight, _ = O.grid_geometry(dim, n, convention)
    diag = O.diagonal(dim, n, a_shift)
    P, _ = _grid(dim, n, convention)
    pts = np.concatenate([r["points"] for r in regions])
    cur = []
    off = 0
    for r in regions:
        npt = r["points"].size
        dofs = np.arange(off, off + npt)
        off += npt
        cur.append(dict(dofs=dofs, lo=r["lo"], hi=r["hi"], K=r["K"],
                        D=_entries(P, weight, diag, r["points"], r["points"])))
    levels = []
    while len(cur) > 1:
        active = np.concatenate([c["dofs"] for c in cur])
        owner = np.concatenate([np.full(c["dofs"].size, b) for b, c in enumerate(cur)])
        recs = []
        for b, c in enumerate(cur):
            Y, near = id_matrix(dim, n, c["lo"], c["hi"], pts[c["dofs"]], pts[active[owner != b]], nproxy,
                                rho, convention)
            skel, red, T = interp_decomp(Y, eps, tau)
            if red.size:
                e = eliminate(c["D"], skel, red, T)
            else:
                e = dict(L=np.zeros((0, 0)), Binv=np.zeros((0, 0)), Bsr=np.zeros((skel.size, 0)),
                         X=np.zeros((0, skel.size)), Bss=c["D"][np.ix_(skel, skel)])
            recs.append(dict(dofs=c["dofs"], skel=skel, red=red, T=T, nnear=int(near.size),
                             Binv=e["Binv"], Bsr=e["Bsr"], X=e["X"], Bss=e["Bss"]))
        levels.append(recs)
        # merge 2^d neighbouring regions by their colour-grid coordinate K >> 1
        groups = {}
        for b, c in enumerate(cur):
            groups.setdefault(tuple(int(v) for v in (c["K"] >> 1)), []).append(b)
        nxt = []
        for key in sorted(groups):
            kids = groups[key]
            dofs = [cur[b]["dofs"][recs[b]["skel"]] for b in kids]
            allp = pts[np.concatenate(dofs)]
            D = _entries(P, weight, diag, allp, allp)
            o = 0
            for b, dd in zip(kids, dofs):
                D[o:o + dd.size, o:o + dd.size] = recs[b]["Bss"]
                o += dd.size
            nxt.append(dict(dofs=np.concatenate(dofs),
                            lo=np.min([cur[b]["lo"] for b in kids], axis=0),
                            hi=np.max([cur[b]["hi"] for b in kids], axis=0),
                            K=np.array(key), D=D))
        cur = nxt
    top = cur[0]
    return dict(points=pts, levels=levels, top=dict(dofs=top["dofs"], L=O.cholesky(top["D"]), D=top["D"]))


def factor(dim, n, m, delta, eps, nproxy, rho=1.5, convention=O.GRID_TEXT, a_shift=0.0, tau=TAU):
    """The RS factors of all 2^d colour subdomains."""
    return [factor_colour(dim, n, regs, eps, nproxy, rho, convention, a_shift, tau)
            for regs in colour_regions(dim, n, m, delta)]


def apply_colour(fc, y: np.ndarray) -> np.ndarray:
    """A_c^{-1} y ~ R diag(I, S^{-1}) R^T y for y in the colour's local order.

    Down (R^T): per region u_r = y_r - T^T y_s (L_p^T), v_r = B_rr^{-1} u_r, y_s -= B_sr v_r
    (U_r^T, keeping v_r in place of y_r).  Top: S^{-1} by the Cholesky factor.  Up (R):
    a_r = v_r - X a_s (U_r), then y_s = a_s - T a_r (L_p)."""
    y = np.array(y, dtype=np.float64, copy=True)
    for recs in fc["levels"]:
        for rec in recs:
            s = rec["dofs"][rec["skel"]]
            r = rec["dofs"][rec["red"]]
            if r.size == 0:
                continue
            u = y[r] - rec["T"].T @ y[s]
            v = rec["Binv"] @ u
            y[s] = y[s] - rec["Bsr"] @ v
            y[r] = v
    t = fc["top"]["dofs"]
    L = fc["top"]["L"]
    y[t] = scipy.linalg.solve_triangular(L.T, scipy.linalg.solve_triangular(L, y[t], lower=True), lower=False)
    for recs in reversed(fc["levels"]):
        for rec in recs:
            s = rec["dofs"][rec["skel"]]
            r = rec["dofs"][rec["red"]]
            if r.size == 0:
                continue
            a_r = y[r] - rec["X"] @ y[s]
            y[r] = a_r
            y[s] = y[s] - rec["T"] @ a_r
    return y


def apply(factors, r: np.ndarray) -> np.ndarray:
    """z = sum_c R_c^T F_c^{-1} R_c r (Eq. e:ad with the RS factors F_c ~ A_c).
    r: (N,) or (N, k); a plain sum over the overlaps."""
    r = np.asarray(r, dtype=np.float64)
    z = np.zeros_like(r)
    for fc in factors:
        p = fc["points"]
        if r.ndim == 1:
            z[p] += apply_colour(fc, r[p])
        else:
            for k in range(r.shape[1]):
                z[p, k] += apply_colour(fc, r[p, k])
    return z


def top_dofs(factors):
    """S of Sec. 5's tables: the DOFs at the last level of each colour subdomain."""
    return [int(fc["top"]["dofs"].size) for fc in factors]


def ranks(factors):
    """Per colour and level, the list of skeleton counts |s| of the regions."""
    return [[[int(rec["skel"].size) for rec in recs] for recs in fc["levels"]] for fc in factors]


def regions_at(fc, level: int):
    """The regions of one colour's factor at ``level`` (1-based; len(levels) + 1 is the last
    level): a list of (global points with the skeletons first, in pivot order, then the
    redundant DOFs in order; rank).  The last level lists its DOFs with rank = their count."""
    pts = fc["points"]
    if level == len(fc["levels"]) + 1:
        t = fc["top"]["dofs"]
        return [(pts[t], int(t.size))]
    out = []
    for rec in fc["levels"][level - 1]:
        d = rec["dofs"]
        out.append((np.concatenate([pts[d[rec["skel"]]], pts[d[rec["red"]]]]), int(rec["skel"].size)))
    return out
