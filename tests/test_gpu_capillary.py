"""GPU checks of the wetting calibration (Section 3.3) and of the critical
body force of a slug (Section 3.4) against the FP64 oracle.

tests/golden/capillary_channel_64.json (written by
tests/golden/make_capillary_golden.py, which calls only the oracle) holds
the oracle's contact angle theta(r) of slugs between flat plates and, for a
scaled-down sinusoidal channel (lambda = 64, h0 = 12, A = 6, 256 x 38, slug
1.5 lambda), the wall potentials of five contact angles and the planar 2-D
critical body force of the oracle's static slug.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_1601_00918_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "capillary_channel_64.json")


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


@pytest.fixture(scope="module")
def gold():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_calibration_matches_oracle(lbm, gold):
    """The library's calibration (GPU FP32 runs, its own interface crossings
    and algebraic circle fit) reproduces the oracle's theta(r) (FP64 runs,
    tanh fits and geometric circle fit) to 1 degree."""
    from paper_1601_00918_gb300 import wetting
    cal = gold["calibration"]
    table = wetting.calibrate(lbm, r_values=cal["r"], H=cal["H"], nx=cal["nx"], steps=gold["steps"])
    np.testing.assert_allclose(table.theta, cal["theta"], atol=1.0)
    k = cal["r"].index(0.0)
    assert table.theta[k] == pytest.approx(90.0, abs=0.2)


def test_critical_force_against_the_2d_balance(lbm, gold):
    """All five channels bisected together on the GPU (2 % bracket, moving
    <=> the oil centre travels more than lambda / 2 in 80 000 steps): for the
    water-wet (40, 60 degrees) and strongly oil-wet (140 degrees) slugs the
    critical force is within 10 % of the oracle's planar 2-D balance
    (measured 1.08, 1.05, 1.01); near neutral wetting (90, 120 degrees) the
    model moves the slug at 0.82-0.85 of it, bounded here at [0.7, 1.1]."""
    ch = gold["channel"]
    insts, g_ref = [], []
    for run in gold["runs"]:
        spec = wl.ChannelSpec(lam=ch["lam"], amp_ratio=ch["amp_ratio"],
                              slug_len_over_lambda=ch["slug_len_over_lambda"], theta_deg=run["theta"],
                              visc_ratio=1.0)
        w = wl.channel_instance(spec)
        insts.append(dict(mask=w.mask, rho_init=w.rho, tau=tuple(gold["tau"]), G=gold["G"],
                          rho_wall=tuple(run["rho_wall"]), g=(0.0, 0.0), periodic=w.periodic,
                          disp_threshold=0.5 * spec.lam))
        g_ref.append(run["g_crit"])
    g_ref = np.array(g_ref)
    b = lbm.Batch(insts, precision="fp32")
    try:
        res = b.critical_pressure(0.5 * g_ref, 2.0 * g_ref, rel_bracket=0.02, t_eq=gold["steps"], t_obs=80000,
                                  max_probes=30, check_bracket=True, check=False)
    finally:
        b.close()
    for run, r, g in zip(gold["runs"], res, g_ref):
        assert r["status"] == 0, (run["theta"], r)
        ratio = math.sqrt(r["g_lo"] * r["g_hi"]) / g
        if run["theta"] in (40.0, 60.0, 140.0):
            assert abs(ratio - 1.0) <= 0.10, (run["theta"], ratio)
        else:
            assert 0.7 <= ratio <= 1.1, (run["theta"], ratio)
