"""Warm-start U-Net on the GPU against the FP64 oracle network (needs a GB300).

Tolerances: the GPU stores weights and activations in bfloat16 (8-bit mantissa, unit
round-off 2^-9 = 2e-3) and accumulates in FP32; the oracle rounds the same tensors to bfloat16
and computes in FP64.  The remaining differences come from FP32 sums and from the occasional
value that rounds to the neighbouring bfloat16 on one side only, so outputs agree to ~1e-2 and
parameter gradients (which also flow through ReLU masks set by those rounded values) to ~5e-2
in relative 2-norm.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ie_oracle as O  # noqa: E402
from oracle import unet_oracle as U  # noqa: E402
from paper_2108_12574_gb300 import iedd  # noqa: E402
from paper_2108_12574_gb300 import inputs as I  # noqa: E402
from paper_2108_12574_gb300 import warmstart as WS  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    torch.cuda.init()


def _he_params(seed):
    rng = np.random.default_rng(seed)
    return np.concatenate([np.concatenate([rng.standard_normal(co * k * k * ci) * np.sqrt(2.0 / (k * k * ci)),
                                           rng.standard_normal(co) * 0.1]) for ci, co, k in U.SPEC]).astype(np.float32)


def test_param_count_matches_oracle():
    m = iedd.ws_create(0, 1)
    assert m.nparams == U.num_params()


@pytest.mark.parametrize("B,n", [(1, 16), (2, 32), (3, 64)])
def test_forward_parity(B, n):
    # the forward 3x3 convolutions run on the tensor cores, 128 pixels per CTA: at 16^2 and 32^2 the
    # coarse levels' tiles span several images and end past the last pixel
    theta = _he_params(5)
    m = iedd.ws_create(0, 1)
    m.set_params(theta)
    x = np.random.default_rng(6).standard_normal((B, n, n, 2)).astype(np.float32)
    out_gpu = m.forward_raw(x)
    out_ref, _ = U.forward(theta.astype(np.float64), x.astype(np.float64), bf16=True)
    err = np.linalg.norm(out_gpu - out_ref) / np.linalg.norm(out_ref)
    assert err <= 1e-2, err


def test_backward_parity():
    B, n = 2, 32
    theta = _he_params(7)
    m = iedd.ws_create(0, 1)
    m.set_params(theta)
    rng = np.random.default_rng(8)
    x = rng.standard_normal((B, n, n, 2)).astype(np.float32)
    dout = rng.standard_normal((B, n, n)).astype(np.float32)
    g_gpu = m.backward_raw(x, dout).astype(np.float64)
    g_ref = U.backward(theta.astype(np.float64), x.astype(np.float64), dout.astype(np.float64), bf16=True)
    assert np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref) <= 5e-2
    # layer by layer (weights and biases of each layer), to catch a wrong layer hidden by big ones
    offs = np.cumsum([0] + [co * k * k * ci + co for ci, co, k in U.SPEC])
    for l in range(len(U.SPEC)):
        a, b = g_gpu[offs[l]:offs[l + 1]], g_ref[offs[l]:offs[l + 1]]
        assert np.linalg.norm(a - b) <= 1e-1 * np.linalg.norm(b) + 1e-6, l


def test_training_reduces_loss():
    n = 32
    prob = iedd.ie_discretize(2, n)
    part = iedd.dd_partition(prob, 2, 2, iedd.DD_SCHWARZ)
    fac = iedd.dd_factor(prob, part, iedd.IE_MIXED)
    F = torch.from_numpy(np.stack([I.grf(2, n, 0.2, s) for s in range(8)])).cuda()
    Usol = torch.zeros_like(F)
    iedd.pcg_solve(prob, fac, F, Usol, tol=1e-10)
    m = iedd.ws_create(0, 3)
    losses = [m.train_step(prob, F, Usol, 1e-3) for _ in range(60)]
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])


def test_warm_start_fallback_keeps_tolerance():
    n = 32
    prob = iedd.ie_discretize(2, n)
    part = iedd.dd_partition(prob, 2, 2, iedd.DD_SCHWARZ)
    fac = iedd.dd_factor(prob, part, iedd.IE_MIXED)
    f = torch.from_numpy(I.grf(2, n, 0.1, 1)).cuda()
    # a bad initial iterate (huge) must fall back to zero and still meet the tolerance
    u0 = torch.full_like(f, 1e6)
    rep = iedd.pcg_solve(prob, fac, f, u0, tol=1e-8, use_x0=2)[0]
    assert rep["x0_used"] == 0 and rep["status"] == 0 and rep["true_relres"] <= 1e-8
    # a good one (the solution itself) is used and needs no iteration
    u1 = u0.clone().zero_()
    iedd.pcg_solve(prob, fac, f, u1, tol=1e-11, precision=iedd.IE_FP64)
    rep = iedd.pcg_solve(prob, fac, f, u1, tol=1e-8, use_x0=2)[0]
    assert rep["x0_used"] == 1 and rep["iterations"] == 0
    assert O.true_relative_residual(2, n, f.cpu().numpy(), u1.cpu().numpy()) <= 1e-8


def test_predict_matches_forward_on_features():
    n = 32
    prob = iedd.ie_discretize(2, n)
    theta = _he_params(9)
    m = iedd.ws_create(0, 1)
    m.set_params(theta)
    fh = I.grf(2, n, 0.15, 4)
    feat, rl = U.features(fh, n)
    out_ref, _ = U.forward(theta.astype(np.float64), feat, bf16=True)
    u0_ref = out_ref.reshape(-1) * rl / (1.0 / n) ** 2
    u0 = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    m.predict(prob, torch.from_numpy(fh).cuda(), u0)
    err = np.linalg.norm(u0.cpu().numpy() - u0_ref) / np.linalg.norm(u0_ref)
    assert err <= 2e-2, err


@pytest.mark.skipif(not os.path.exists(WS.WEIGHTS), reason="trained weights not present")
def test_trained_warm_start_saves_iterations():
    # what the trained network gains over the method without it, on held-out fields
    prob, part, fac = WS.setup()
    model = WS.load_model()
    rows = WS.evaluate(model, prob, fac, list(range(8)))
    s = WS.summarize(rows)
    assert s["max_true_relres_warm"] <= 1e-8
    assert s["iterations_warm"] < s["iterations_zero"], s
