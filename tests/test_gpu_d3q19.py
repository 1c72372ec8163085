"""GPU parity of the D3Q19 step (lbm3d_*, the paper's own lattice) with the
D3Q19 oracle (oracle/d3q19.py), on the paper's 3-D geometry: a periodic
sinusoidal tube of circular cross sections holding an oil slug.

Tolerances: FP64 on both sides evaluates the same formulas in a different
order, 1e-12 absolute on populations <= 1/3 after 50 steps; FP32 storage
and arithmetic, one step from the same state: each population goes through
~80 FP32 operations on O(1) values, 1e-5 absolute; after 200 FP32 steps the
densities within 1e-4 relative and the mass within 1e-6.
"""
import numpy as np
import pytest

from oracle import d3q19
from paper_1601_00918_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
G = -1.79


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


def tube_case(collision="bgk"):
    mask = wl.sinusoidal_tube(48, 18, 6.0, 2.5, 24.0)
    rho = wl.tube_slug(48, 18, 14.0, 34.0)
    kw = dict(tau=(1.0, 0.9), G=G, rho_wall=(0.1, 0.4), g=(1e-5, 2e-6, 0.0), periodic=(True, False, False),
              collision=collision)
    return mask, rho, kw


@pytest.mark.parametrize("collision", ["bgk", "regularized"])
@pytest.mark.parametrize("steps", [1, 50])
def test_fp64_tube_matches_oracle(lbm, collision, steps):
    mask, rho, kw = tube_case(collision)
    sim = lbm.Simulation3(mask, rho, precision="fp64", **kw)
    try:
        sim.step(steps)
        f_gpu = sim.save()
        obs = sim.observables()
        rho_g, u_g = sim.fields()
    finally:
        sim.close()
    P = d3q19.Problem3(mask, **kw)
    f_ref, hist = P.run(P.init(rho), steps, history=True)
    np.testing.assert_allclose(f_gpu, f_ref, rtol=0, atol=1e-12)
    rho_r, u_r = P.fields(f_ref)
    np.testing.assert_allclose(rho_g, rho_r, rtol=0, atol=1e-12)
    np.testing.assert_allclose(u_g, u_r, rtol=0, atol=1e-13)
    assert obs["step"] == steps and obs["nan_flag"] == 0
    np.testing.assert_allclose(obs["mass"], hist[-1, :2], rtol=1e-12)
    np.testing.assert_allclose(obs["oil_mom_x"], hist[-1, 2], rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(obs["max_u"], hist[-1, 3], rtol=1e-9, atol=1e-15)


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 4, 5), (5, 1, 9), (2, 7, 33), (4, 3, 130)])
def test_fp64_odd_periodic_boxes(lbm, shape):
    """Fully periodic boxes of odd and degenerate sizes (one node, widths
    not a multiple of the 128-thread block, a ragged last block) with a
    random mixture and a force along all three axes."""
    nz, ny, nx = shape
    rng = np.random.default_rng(nx * 7 + ny * 3 + nz)
    rho = 0.5 + 0.4 * rng.random((2, nz, ny, nx))
    mask = np.zeros(shape, np.uint8)
    kw = dict(tau=(0.9, 1.3), G=G, g=(1e-5, -2e-5, 3e-5), periodic=(True, True, True))
    sim = lbm.Simulation3(mask, rho, precision="fp64", **kw)
    try:
        sim.step(7)
        f_gpu = sim.save()
    finally:
        sim.close()
    P = d3q19.Problem3(mask, **kw)
    np.testing.assert_allclose(f_gpu, P.run(P.init(rho), 7), rtol=0, atol=1e-12)


def test_fp32_tube_one_step_and_200_steps(lbm):
    mask, rho, kw = tube_case("regularized")
    P = d3q19.Problem3(mask, **kw)
    f0 = P.run(P.init(rho), 20).astype(np.float32).astype(np.float64)
    sim = lbm.Simulation3(mask, rho, precision="fp32", **kw)
    try:
        sim.load(f0)
        sim.step(1)
        f1 = sim.save()
        sim.load(P.init(rho))
        sim.step(200)
        obs = sim.observables()
        rho_g, _ = sim.fields()
    finally:
        sim.close()
    np.testing.assert_allclose(f1, P.step(f0)[0], rtol=0, atol=1e-5)
    f_ref, hist = P.run(P.init(rho), 200, history=True)
    rho_r, _ = P.fields(f_ref)
    fluid = mask == 0
    assert np.max(np.abs(rho_g - rho_r)[:, fluid]) / np.max(rho_r[:, fluid]) < 1e-4
    np.testing.assert_allclose(obs["mass"], hist[-1, :2], rtol=1e-6)


def test_create_rejects_open_boundaries_and_bad_densities(lbm):
    mask, rho, kw = tube_case()
    with pytest.raises(lbm.LbmError) as err:
        lbm.Simulation3(np.zeros_like(mask), rho, **kw)        # not periodic in y, z but fluid there
    assert err.value.code == lbm.LBM_EINVAL
    bad = rho.copy()
    z, y, x = np.argwhere(mask == 0)[0]
    bad[0, z, y, x] = np.nan
    with pytest.raises(lbm.LbmError):
        lbm.Simulation3(mask, bad, **kw)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_index_widths_give_the_same_bits(lbm, precision, monkeypatch):
    """The 32-bit-offset kernels (any grid whose population planes stay
    below 2^32 elements) and the 64-bit ones (larger grids, forced here by
    GB300LBM_INDEX64=1) run the same arithmetic: 30 steps of the tube, BGK
    and regularised, give identical populations and fields."""
    for collision in ("bgk", "regularized"):
        mask, rho, kw = tube_case(collision)
        out = []
        for force64 in ("0", "1"):
            monkeypatch.setenv("GB300LBM_INDEX64", force64)
            sim = lbm.Simulation3(mask, rho, precision=precision, **kw)
            try:
                sim.step(30)
                rho_g, u_g = sim.fields()
                out.append((sim.save(), rho_g, u_g))
            finally:
                sim.close()
        for a, b in zip(out[0], out[1]):
            np.testing.assert_array_equal(a, b)
