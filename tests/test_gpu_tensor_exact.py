"""The exact tensor-core 2D matvec (IE_TENSOR_EXACT, Ozaki-scheme digit slices) against the FP64
CPU oracle, through the C ABI (needs a GB300).

Tolerance: |y - y_ref|_inf <= 1e-13 * ||A||_inf ||x||_inf, ten times below the FP64-class bound of
the other exact matvecs.  The kernel's own error is ~1e-16 of sum |A_ij x_j|: the six digits of
each factor carry 52 bits, the dropped digit pairs weigh <= 2^-54, the leading levels are summed
exactly and the tail is rounded to 2^-(14 + F) sigma_t sigma_x per 128-term window.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ie_oracle as O  # noqa: E402
from paper_2108_12574_gb300 import iedd  # noqa: E402
from paper_2108_12574_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available()
    torch.cuda.init()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.detach().cpu().numpy()


def _scale(n, x, conv=O.GRID_TEXT):
    # ||A||_inf ||x||_inf from the oracle's row sums (factor 2 for the negative far entries)
    rows = O.matvec_direct(2, n, np.ones(n * n), rows=np.array([0, (n * n) // 2]), convention=conv)
    return 2.0 * float(np.max(np.abs(rows))) * float(np.max(np.abs(x)))


def _mv(prob, X):
    X = np.array(np.atleast_2d(X), dtype=np.float64, order="C")  # (nrhs, N) with row stride N
    Xd = dev(X)
    Y = torch.zeros_like(Xd)
    iedd.ie_matvec(prob, Xd, Y, iedd.IE_TENSOR_EXACT)
    return host(Y)


@pytest.mark.parametrize("n,conv,nrhs", [(128, O.GRID_TEXT, 1), (256, O.GRID_TEXT, 2), (128, O.GRID_TABLE, 1),
                                         (384, O.GRID_TEXT, 1)])
def test_tensor_exact_matvec_parity(n, conv, nrhs):
    # several tiles, column blocks and d1 splits; two columns share the launch sequence
    N = n * n
    X = I.uniform_rhs_batch(N, list(range(21, 21 + nrhs))).T.copy()
    prob = iedd.ie_discretize(2, n, grid=conv)
    Y = _mv(prob, X)
    for k in range(nrhs):
        rows = None if n <= 256 else np.unique(np.random.default_rng(k).integers(0, N, 97))
        ref = O.matvec_direct(2, n, X[k], rows=rows, convention=conv)
        got = Y[k] if rows is None else Y[k][rows]
        err = np.max(np.abs(got - ref))
        assert err <= 1e-13 * _scale(n, X[k], conv), (k, err)


def test_tensor_exact_matvec_full_size_sampled_rows():
    # the 512^2 workload's launch configuration; a smooth field (the PCG right-hand side's kind)
    n = 512
    N = n * n
    x = I.grf(2, n, 0.1, 2)
    rows = np.unique(np.concatenate([[0, n - 1, N - 1, N // 2 + n // 2], np.random.default_rng(3).integers(0, N, 29)]))
    ref = O.matvec_direct(2, n, x, rows=rows)
    prob = iedd.ie_discretize(2, n)
    y = _mv(prob, x)[0]
    assert np.max(np.abs(y[rows] - ref)) <= 1e-13 * _scale(n, x)


def test_tensor_exact_unit_vectors_give_columns_of_a():
    # x = e_j: y is column j of A (52-bit digits; the tail is rounded to 2^-(14 + F) sigma_t sigma_x)
    n = 128
    N = n * n
    prob = iedd.ie_discretize(2, n)
    for j in (0, n - 1, N // 2 + 3, N - 1):
        x = np.zeros(N)
        x[j] = 1.0
        y = _mv(prob, x)[0]
        col = O.matvec_direct(2, n, x)
        assert np.max(np.abs(y - col)) <= 1e-13 * np.max(np.abs(col)), j


def test_tensor_exact_zero_and_power_of_two_scaling():
    # x = 0 gives 0 exactly; scaling x by 2^k scales y by 2^k bit for bit (power-of-two digit
    # scales); two calls agree bit for bit
    n = 128
    N = n * n
    prob = iedd.ie_discretize(2, n)
    assert np.all(_mv(prob, np.zeros(N)) == 0.0)
    x = I.uniform_rhs(N, 5)
    y = _mv(prob, x)[0]
    assert np.array_equal(_mv(prob, x)[0], y)
    for k in (-40, 7):
        assert np.array_equal(_mv(prob, np.ldexp(x, k))[0], np.ldexp(y, k))


def test_tensor_exact_wide_dynamic_range():
    # entries spread over 12 decades: the bound is relative to ||x||_inf, as for the other kernels
    n = 128
    N = n * n
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, N) * 10.0 ** rng.uniform(-12, 0, N)
    prob = iedd.ie_discretize(2, n)
    y = _mv(prob, x)[0]
    assert np.max(np.abs(y - O.matvec_direct(2, n, x))) <= 1e-13 * _scale(n, x)


def test_tensor_exact_rejects_unsupported_grids():
    for dim, n in ((2, 96), (3, 128)):
        prob = iedd.ie_discretize(dim, n if dim == 2 else 16)
        x = torch.zeros(prob.N, dtype=torch.float64, device="cuda")
        y = torch.zeros_like(x)
        with pytest.raises(iedd.IEError):
            iedd.ie_matvec(prob, x, y, iedd.IE_TENSOR_EXACT)


def test_pcg_tensor_exact_inner_fp64_parity():
    # FP64 factors with the exact tensor-core inner matvec: the oracle's iterations (+-1), and the
    # oracle's iterate after the same number of iterations to 1e-10 -- compared at iteration counts
    # where the iterate is well conditioned.  Near the stopping count of this problem single
    # iterations are hypersensitive (two FP64 oracles, FFT and direct-sum matvec, differ there by
    # up to ~1e-10 at iteration 23 and agree to ~1e-13 two iterations later), so each compared count
    # is first checked on the oracle itself: its two matvecs must agree to 1e-11 there.
    n, m, delta = 128, 8, 1
    N = n * n
    f = I.uniform_rhs(N, 0)
    prob = iedd.ie_discretize(2, n)
    part = iedd.dd_partition(prob, m, delta, iedd.DD_SCHWARZ)
    fac = iedd.dd_factor(prob, part, iedd.IE_FP64)
    u = torch.zeros(N, dtype=torch.float64, device="cuda")
    rep = iedd.pcg_solve(prob, fac, dev(f), u, tol=1e-8, precision=iedd.IE_FP64, inner=iedd.IE_TENSOR_EXACT)[0]
    Pf = O.Problem(2, n, m, delta, O.SCHWARZ, matvec="fft")
    _, it_ref, _ = Pf.solve(f, 1e-8)
    assert abs(rep["iterations"] - it_ref) <= 1, (rep, it_ref)
    assert O.true_relative_residual(2, n, f, host(u)) <= 1e-8 * 1.05
    Pd = O.Problem(2, n, m, delta, O.SCHWARZ, matvec="direct")
    compared = []
    for k in (rep["iterations"], rep["iterations"] + 2, rep["iterations"] + 4):
        u_f, _, _ = Pf.solve(f, 0.0, max_it=k)
        u_d, _, _ = Pd.solve(f, 0.0, max_it=k)
        if np.linalg.norm(u_f - u_d) > 1e-11 * np.linalg.norm(u_d):
            continue  # an ill-conditioned iterate: FP64 implementations differ here
        uk = torch.zeros(N, dtype=torch.float64, device="cuda")
        iedd.pcg_solve(prob, fac, dev(f), uk, tol=0.0, max_it=k, precision=iedd.IE_FP64,
                       inner=iedd.IE_TENSOR_EXACT, check=False)
        err = np.linalg.norm(host(uk) - u_d) / np.linalg.norm(u_d)
        assert err <= 1e-10, (k, err)
        compared.append(k)
    assert len(compared) >= 2, compared


def test_pcg_tensor_exact_inner_mixed_512():
    # the 512^2 workload with the exact tensor-core inner matvec (forced) and FP32 inverses: the
    # checks of the mixed parity tests (true residual, the oracle's solution, the count within the
    # oracle ensemble's counts at 1e-8 and at the stable tolerance)
    import pcg_golden as G
    c = G.case("ie2d_n512_m32_d2_grf")
    n, m, delta = c["n"], c["m"], c["delta"]
    f = G.rhs(c)[:, 0]
    prob = iedd.ie_discretize(2, n)
    part = iedd.dd_partition(prob, m, delta, iedd.DD_SCHWARZ)
    fac = iedd.dd_factor(prob, part, iedd.IE_MIXED)
    its = {}
    for tol in (1e-8, c["tol"]):
        u = torch.zeros(n * n, dtype=torch.float64, device="cuda")
        rep = iedd.pcg_solve(prob, fac, dev(f), u, tol=tol, precision=iedd.IE_MIXED, inner=iedd.IE_TENSOR_EXACT)[0]
        assert rep["status"] == 0 and rep["true_relres"] <= tol
        assert O.true_relative_residual(2, n, f, host(u)) <= tol * 1.01
        its[tol] = rep["iterations"]
        if tol == 1e-8:
            u8 = host(u)
    lo, hi = G.band_at_1e8(c)
    assert lo <= its[1e-8] <= hi, (its, (lo, hi))
    G.check_mixed_counts(c, [its[c["tol"]]])
    u_ref, it_ref, _ = O.Problem(2, n, m, delta, O.SCHWARZ, matvec="fft").solve(f, 1e-8)
    assert np.linalg.norm(u8 - u_ref) / np.linalg.norm(u_ref) <= 1e-6
