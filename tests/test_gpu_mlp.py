"""GPU tests of the surrogate network kernels against the FP64 oracle.

Tolerances: the GPU runs FP32 with fused multiply-adds and fast exp; the
oracle runs FP64 on the same FP32-rounded parameters and inputs.  Forward
outputs agree to 1e-4 relative (three 128-wide FP32 dot products), the
gradient to 1e-3 relative in norm and per coordinate above 1e-4 of its
largest entry, and one Adam step exactly up to FP32 rounding (1e-5)."""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1601_00918_gb300 import build
    build.build()
    from paper_1601_00918_gb300 import lbm as mod
    mod.library()
    return mod


def data(n, seed):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(n, 5)).astype(np.float32)
    y = (np.sin(x[:, 0]) + 0.5 * x[:, 1] * x[:, 2] - 0.3 * x[:, 3] + 0.1 * rng.normal(size=n)).astype(np.float32)
    return x, y


def test_forward_matches_oracle(lbm):
    th = mlp.init_params(3).astype(np.float32)
    x, _ = data(300, 1)
    net = lbm.Surrogate(params=th)
    try:
        out = net.forward(x)
        np.testing.assert_array_equal(net.params(), th)
    finally:
        net.close()
    ref, _, _ = mlp.forward(th.astype(np.float64), x.astype(np.float64))
    np.testing.assert_allclose(out, ref, rtol=1e-4, atol=1e-5)


@pytest.mark.parametrize("B", [1, 17, 256])
def test_gradient_matches_oracle(lbm, B):
    th = mlp.init_params(5).astype(np.float32)
    th[-1] = 0.4          # a non-zero log-variance bias
    x, y = data(B, 2)
    net = lbm.Surrogate(params=th)
    try:
        L, g = net.loss_grad(x, y)
    finally:
        net.close()
    L_ref, g_ref = mlp.grad(th.astype(np.float64), x.astype(np.float64), y.astype(np.float64))
    assert L == pytest.approx(L_ref, rel=1e-4)
    assert np.linalg.norm(g - g_ref) <= 1e-3 * np.linalg.norm(g_ref)
    big = np.abs(g_ref) > 1e-4 * np.abs(g_ref).max()
    np.testing.assert_allclose(g[big], g_ref[big], rtol=1e-3, atol=1e-4 * np.abs(g_ref).max())


def test_adam_step_matches_formula(lbm):
    th = mlp.init_params(7).astype(np.float32)
    x, y = data(64, 3)
    net = lbm.Surrogate(params=th)
    try:
        _, g = net.loss_grad(x, y)
        net.adam(1e-3)
        th1 = net.params()
    finally:
        net.close()
    ref, _, _ = mlp.adam_step(th.astype(np.float64), g.astype(np.float64), np.zeros(th.size), np.zeros(th.size), 1,
                              lr=1e-3)
    np.testing.assert_allclose(th1, ref, rtol=0, atol=1e-5 * 1e-3 + 1e-7)


def test_training_fits_a_smooth_target(lbm):
    """Minibatch Adam on the GPU lowers the NLL well below the untrained
    value and the predicted mean follows a smooth synthetic target."""
    x, y = data(4096, 4)
    xt, yt = data(512, 5)
    net = lbm.Surrogate(seed=11)
    try:
        L0 = mlp.loss(net.params().astype(np.float64), xt.astype(np.float64), yt.astype(np.float64))
        net.train(x, y, epochs=60, batch=256, lr=2e-3, seed=0)
        th = net.params()
        pred = net.forward(xt)
    finally:
        net.close()
    L1 = mlp.loss(th.astype(np.float64), xt.astype(np.float64), yt.astype(np.float64))
    assert L1 < L0 - 1.0
    rmse = float(np.sqrt(np.mean((pred[:, 0] - yt) ** 2)))
    assert rmse < 0.25, rmse
