"""Host logic of the learned warm start (no GPU): the symmetry augmentation of its training set
and the length-scale draw of its fields.

The training set multiplies each solved pair (f, u) by the eight symmetries of the square.  That
is only valid because A commutes with them on the cell-centred grid: the oracle's dense A checks it.
"""
import numpy as np
import scipy.linalg
import torch

from oracle import ie_oracle as O
from paper_2108_12574_gb300 import inputs as I
from paper_2108_12574_gb300 import warmstart as WS


def test_symmetry_images_of_a_solution_are_solutions():
    n = 8
    A = O.dense_matrix(2, n)
    f = I.uniform_rhs(n * n, 5)
    u = scipy.linalg.solve(A, f, assume_a="pos")
    F = WS.symmetries(torch.from_numpy(f[None]), n).numpy()
    U = WS.symmetries(torch.from_numpy(u[None]), n).numpy()
    assert F.shape == (8, n * n) and U.shape == (8, n * n)
    # eight different images of a generic field
    assert len({F[k].tobytes() for k in range(8)}) == 8
    for k in range(8):
        assert np.linalg.norm(A @ U[k] - F[k]) <= 1e-12 * np.linalg.norm(F[k])


def test_symmetries_keep_batches_grouped_by_image():
    n = 4
    X = torch.arange(2 * n * n, dtype=torch.float64).reshape(2, n * n)
    S = WS.symmetries(X, n)
    assert S.shape == (16, n * n)
    assert torch.equal(S[0], X[0]) and torch.equal(S[1], X[1])  # the identity comes first
    # every image is a permutation of its source row
    for k in range(16):
        assert torch.equal(torch.sort(S[k]).values, torch.sort(X[k % 2]).values)


def test_length_scales_cover_the_stated_range():
    ells = np.array([WS.ell_of(s) for s in range(1000, 1512)])
    assert np.all(ells >= WS.ELL_LO) and np.all(ells < WS.ELL_HI)
    assert ells.min() < 0.05 and ells.max() > 0.28  # spread over [0.03, 0.3]
    assert WS.ell_of(1000) == WS.ell_of(1000)  # seeded
