"""The allocation-free step (lbm_step_noalloc) through the C ABI.

This entry point serves callers that cannot allocate device memory (code
running inside a CUDA graph capture, real-time loops, plug-ins whose device
memory belongs to a host framework): they pass device inputs and outputs and
the step's scratch is a fixed device array inside the library.  Here two
calls in a row are checked against the handle-based step (lbm_create /
lbm_step with the same FP32 kernel) and against the FP64 oracle, within the
one-step FP32 tolerance of the parity tests (5e-6 absolute on populations);
a call without observables (obs = NULL), a grid taller than 65 535 rows and
the parameter checks are covered too.  The file is named so that pytest
collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1601_00918_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_step_matches_handle_step_on_two_calls():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1601_00918_gb300 import build, lbm
    build.build()
    lib = lbm.library()

    nx, ny = 300, 40
    mask = wl.sinusoidal_channel(nx, ny, 12.0, 5.0, 100.0)
    rho = wl.slug(nx, ny, 90.0, 210.0)
    kw = dict(tau=(1.0, 0.9), G=-1.79, rho_wall=(0.3, 0.1), g=(2e-5, 0.0), periodic=(True, False))

    # reference: the handle-based path, same FP32 step kernel
    sim = lbm.Simulation(mask, rho, precision="fp32", variant="simple", **kw)
    try:
        sim.step(7)
        f0 = sim.save()
        sim.load(f0)
        sim.step(1)
        f1 = sim.save()
        o1 = sim.observables()
        sim.step(1)
        f2 = sim.save()
        o2 = sim.observables()
    finally:
        sim.close()

    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    d_mask = torch.from_numpy(mask).to(dev)
    a = torch.from_numpy(f0.astype(np.float32)).to(dev).contiguous()
    b = torch.zeros_like(a)
    d_obs = torch.zeros(ctypes.sizeof(lbm.Obs), dtype=torch.uint8, device=dev)
    p = lbm.make_params(nx, ny, precision="fp32", stream=stream.cuda_stream, **kw)

    def call(src, dst):
        rc = lib.lbm_step_noalloc(d_mask.data_ptr(), src.data_ptr(), dst.data_ptr(), d_obs.data_ptr(),
                                  ctypes.byref(p))
        assert rc == lbm.LBM_OK, lbm.lbm_last_error(None)
        torch.cuda.synchronize()
        return lbm.Obs.from_buffer_copy(d_obs.cpu().numpy().tobytes()).as_dict()

    ob1 = call(a, b)
    np.testing.assert_allclose(b.cpu().numpy().astype(np.float64), f1, rtol=0, atol=5e-6)
    P = oracle.Problem(mask, **kw)
    f1_ref, _ = P.step(f0.astype(np.float32).astype(np.float64))
    fluid = mask == 0
    np.testing.assert_allclose(b.cpu().numpy().astype(np.float64)[:, :, fluid], f1_ref[:, :, fluid], rtol=0,
                               atol=5e-6)
    np.testing.assert_allclose(ob1["mass"], o1["mass"], rtol=1e-6)
    assert ob1["step"] == 1 and ob1["nan_flag"] == 0 and ob1["timeout_flag"] == 0

    ob2 = call(b, a)      # second call: the scratch keeps the first call's contents
    np.testing.assert_allclose(a.cpu().numpy().astype(np.float64), f2, rtol=0, atol=5e-6)
    np.testing.assert_allclose(ob2["mass"], o2["mass"], rtol=1e-6)
    assert ob2["step"] == 1

    # without observables: the same populations
    c = torch.zeros_like(a)
    assert lib.lbm_step_noalloc(d_mask.data_ptr(), b.data_ptr(), c.data_ptr(), None, ctypes.byref(p)) == lbm.LBM_OK
    torch.cuda.synchronize()
    assert torch.equal(c, a)

    # sizes beyond the scratch limit are rejected before any work
    big = lbm.make_params(4096, 1024, precision="fp32", stream=stream.cuda_stream, **kw)
    assert lib.lbm_step_noalloc(d_mask.data_ptr(), a.data_ptr(), b.data_ptr(), None,
                                ctypes.byref(big)) == lbm.LBM_EINVAL
    assert "2097152" in lbm.lbm_last_error(None)
    # non-finite parameters are rejected as lbm_create rejects them
    for field, value in (("G", float("nan")), ("tau", (float("inf"), 1.0)), ("rho_wall", (0.3, float("nan")))):
        bad = lbm.make_params(nx, ny, precision="fp32", stream=stream.cuda_stream, **{**kw, field: value})
        assert lib.lbm_step_noalloc(d_mask.data_ptr(), a.data_ptr(), b.data_ptr(), None,
                                    ctypes.byref(bad)) == lbm.LBM_EINVAL


def test_noalloc_step_on_a_grid_taller_than_65535_rows():
    """A 4 x 70 000 periodic mixture (280 000 nodes, within the limit):
    the set-up and the step visit rows beyond the 65 535 a grid dimension can
    hold, and the result matches the FP64 oracle's step."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1601_00918_gb300 import build, lbm
    build.build()
    lib = lbm.library()
    nx, ny = 4, 70000
    mask = wl.periodic_box(nx, ny)
    kw = dict(tau=(0.9, 1.2), G=-1.79, rho_wall=(0.0, 0.0), g=(1e-5, 2e-6), periodic=(True, True))
    P = oracle.Problem(mask, **kw)
    f0 = P.run(P.init(wl.random_perturbed(nx, ny, seed=5, amp=0.2)), 2).astype(np.float32).astype(np.float64)
    f1_ref, obs_ref = P.step(f0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    d_mask = torch.from_numpy(mask).to(dev)
    a = torch.from_numpy(f0.astype(np.float32)).to(dev).contiguous()
    b = torch.zeros_like(a)
    d_obs = torch.zeros(ctypes.sizeof(lbm.Obs), dtype=torch.uint8, device=dev)
    p = lbm.make_params(nx, ny, precision="fp32", stream=stream.cuda_stream, **kw)
    rc = lib.lbm_step_noalloc(d_mask.data_ptr(), a.data_ptr(), b.data_ptr(), d_obs.data_ptr(), ctypes.byref(p))
    assert rc == lbm.LBM_OK, lbm.lbm_last_error(None)
    torch.cuda.synchronize()
    np.testing.assert_allclose(b.cpu().numpy().astype(np.float64), f1_ref, rtol=0, atol=5e-6)
    ob = lbm.Obs.from_buffer_copy(d_obs.cpu().numpy().tobytes()).as_dict()
    np.testing.assert_allclose(ob["mass"], obs_ref[:2], rtol=1e-6)
