"""Planted mistakes in the RS oracle (on the CPU) must be caught by its pins.

Each case patches one plausible slip into oracle/rs_oracle.py -- a dropped term or a wrong sign
in compress-then-eliminate (Eqs. e:al, e:alu, e:b), a skipped operator in the application, the
Schur update left out of the merged block (Eq. e:schur), the near field left out of the proxy
ID (Eq. e:id) in 2D and 3D or at the merged levels only, a 3D proxy sphere flattened onto its
equator or cut to a polar cap -- and checks that the named pin of test_oracle_rs.py now fails.
"""
import numpy as np
import pytest

from oracle import ie_oracle as O
from oracle import rs_oracle as RS

CASE = (2, 32, 4, 1)     # 2 x 2 regions per colour: one compression level, then the top
EPS = 1e-6


def _factor_error_pin():
    """test_factor_error_is_proportional_to_eps at one eps: max ||F_c^{-1} A_c - I||_2 <= 100 eps."""
    dim, n, m, delta = CASE
    try:
        F = RS.factor(dim, n, m, delta, EPS, 64)
    except O.NotSPD:
        return False
    for fc in F:
        pts = fc["points"]
        Ac = O.dense_matrix(dim, n, index=pts)
        Finv = RS.apply_colour(fc, np.eye(pts.size))
        if not np.linalg.norm(Finv @ Ac - np.eye(pts.size), 2) <= 100 * EPS:
            return False
    return True


def _id_bound_pin():
    """test_proxy_id_meets_the_bound_on_the_full_block at one eps."""
    dim, n, m, delta = 2, 64, 8, 1
    F = RS.factor(dim, n, m, delta, EPS, 64)
    P = O.points(dim, n)
    _, _, wgt, _ = O.grid_geometry(dim, n)
    for fc in F:
        for rec in fc["levels"][0]:
            p = fc["points"][rec["dofs"]]
            q = np.setdiff1d(fc["points"], p)
            d = P[q][:, None, :] - P[p][None, :, :]
            A = wgt * O.kernel(dim, np.sqrt((d * d).sum(axis=2)))
            Aqr, Aqs = A[:, rec["red"]], A[:, rec["skel"]]
            if not np.linalg.norm(Aqr - Aqs @ rec["T"]) <= EPS * np.linalg.norm(Aqr):
                return False
    return True


def test_unmutated_oracle_passes_both_pins():
    assert _factor_error_pin()
    assert _id_bound_pin()


def _patched_eliminate(variant):
    orig = RS.eliminate

    def bad(D, skel, red, T):
        Dss = D[np.ix_(skel, skel)]
        Dsr = D[np.ix_(skel, red)]
        Drr = D[np.ix_(red, red)]
        if variant == "drop_TtDssT":
            Brr = Drr - Dsr.T @ T - T.T @ Dsr
        else:
            Brr = Drr - Dsr.T @ T - T.T @ Dsr + T.T @ Dss @ T
        Bsr = Dsr + Dss @ T if variant == "sign_Bsr" else Dsr - Dss @ T
        if variant == "no_schur_update":
            e = orig(D, skel, red, T)
            e["Bss"] = Dss
            return e
        L = O.cholesky(Brr)
        Linv = np.linalg.inv(L)
        Binv = Linv.T @ Linv
        X = Binv @ Bsr.T
        return dict(L=L, Binv=Binv, Bsr=Bsr, X=X, Bss=Dss - Bsr @ X)
    return bad


@pytest.mark.parametrize("variant", ["drop_TtDssT", "sign_Bsr", "no_schur_update"])
def test_elimination_slips_are_caught(monkeypatch, variant):
    monkeypatch.setattr(RS, "eliminate", _patched_eliminate(variant))
    assert not _factor_error_pin()


@pytest.mark.parametrize("variant", ["skip_Lp_transpose", "skip_Lp", "skip_X"])
def test_application_slips_are_caught(monkeypatch, variant):
    import scipy.linalg

    def bad_apply(fc, y):
        y = np.array(y, dtype=np.float64, copy=True)
        for recs in fc["levels"]:
            for rec in recs:
                s = rec["dofs"][rec["skel"]]
                r = rec["dofs"][rec["red"]]
                if r.size == 0:
                    continue
                u = y[r] if variant == "skip_Lp_transpose" else y[r] - rec["T"].T @ y[s]
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
                a_r = y[r] if variant == "skip_X" else y[r] - rec["X"] @ y[s]
                y[r] = a_r
                if variant != "skip_Lp":
                    y[s] = y[s] - rec["T"] @ a_r
        return y
    monkeypatch.setattr(RS, "apply_colour", bad_apply)
    assert not _factor_error_pin()


def test_proxy_id_without_the_near_field_is_caught(monkeypatch):
    orig = RS.id_matrix

    def no_near(dim, n, lo, hi, own, others, nproxy, rho=1.5, convention=O.GRID_TEXT):
        return orig(dim, n, lo, hi, own, np.zeros(0, dtype=np.int64), nproxy, rho, convention)
    monkeypatch.setattr(RS, "id_matrix", no_near)
    assert not _id_bound_pin()


def _id_bound_pin_3d():
    """test_proxy_id_meets_the_bound_on_the_full_block_3d over every region of one colour."""
    dim, n, m, delta, eps = 3, 16, 4, 1, 1e-3
    regs = RS.colour_regions(dim, n, m, delta)[0]
    P = O.points(dim, n)
    _, _, wgt, _ = O.grid_geometry(dim, n)
    allp = np.concatenate([r["points"] for r in regs])
    for r in regs:
        p = r["points"]
        q = np.setdiff1d(allp, p)
        d = P[q][:, None, :] - P[p][None, :, :]
        A = wgt * O.kernel(dim, np.sqrt((d * d).sum(axis=2)))
        Y, _ = RS.id_matrix(dim, n, r["lo"], r["hi"], p, q, 128)
        skel, red, T = RS.interp_decomp(Y, eps)
        if not np.linalg.norm(A[:, red] - A[:, skel] @ T) <= eps * np.linalg.norm(A[:, red]):
            return False
    return True


def test_unmutated_oracle_passes_the_3d_pin():
    assert _id_bound_pin_3d()


@pytest.mark.parametrize("variant", ["flattened", "polar_cap", "no_near"])
def test_3d_proxy_slips_are_caught(monkeypatch, variant):
    orig_dirs, orig_id = RS.proxy_directions, RS.id_matrix
    if variant == "flattened":    # the sphere's points squashed onto its equator
        monkeypatch.setattr(RS, "proxy_directions",
                            lambda dim, P: orig_dirs(dim, P) * np.array([1.0, 1.0, 0.0]) if dim == 3 else orig_dirs(dim, P))
    elif variant == "polar_cap":  # only the first eighth of the Fibonacci lattice
        monkeypatch.setattr(RS, "proxy_directions",
                            lambda dim, P: orig_dirs(dim, P)[: P // 8] if dim == 3 else orig_dirs(dim, P))
    else:
        def no_near(dim, n, lo, hi, own, others, nproxy, rho=1.5, convention=O.GRID_TEXT):
            return orig_id(dim, n, lo, hi, own, np.zeros(0, dtype=np.int64), nproxy, rho, convention)
        monkeypatch.setattr(RS, "id_matrix", no_near)
    assert not _id_bound_pin_3d()


def test_near_field_dropped_at_the_merged_levels_is_caught(monkeypatch):
    """Level 1 keeps its near field, so the level-1 pin cannot see the slip; the merged-level pin
    (test_proxy_id_meets_the_bound_at_the_merged_levels) does."""
    from test_oracle_rs import upper_level_id_ratios
    orig = RS.id_matrix
    box = 64 // 8 + 2   # the extended box side of the 64^2 grid with 8^2 boxes, one layer of overlap

    def near_at_level1_only(dim, n, lo, hi, own, others, nproxy, rho=1.5, convention=O.GRID_TEXT):
        if int((np.asarray(hi) - np.asarray(lo)).max()) > box:
            others = np.zeros(0, dtype=np.int64)
        return orig(dim, n, lo, hi, own, others, nproxy, rho, convention)
    monkeypatch.setattr(RS, "id_matrix", near_at_level1_only)
    assert _id_bound_pin()
    worst = upper_level_id_ratios(2, 64, 8, 1, EPS, 64)
    assert max(worst.values()) > 1.0, worst
