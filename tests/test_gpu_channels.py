"""GPU tests of the channel-level calls of the C ABI: the paper's question
(Section 3.4) posed from channel descriptions, with every set-up step inside
the library (geometry, Section 3.3 wetting calibration, Section 3.1 surface
tension, planar starting bracket or surrogate bracket, batched bisection,
Bond numbers)."""
import json
import math
import os

import numpy as np
import pytest

from paper_1601_00918_gb300 import sweep, wetting
from paper_1601_00918_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
T_EQ, T_OBS = 800, 1600


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
def table(lbm):
    return wetting.calibrate(lbm)


def test_channel_call_matches_the_host_built_sweep_bit_for_bit(lbm, table):
    """lbm_critical_pressure_channels from a spec array gives the brackets,
    probe counts and statuses of the sweep built on the host from the same
    descriptions (sweep.instance_of + analytic brackets +
    lbm_critical_pressure_batch), bit for bit, and the starting brackets are
    0.5 and 2 times the planar balance of each slug."""
    specs = sweep.small_specs(12, seed=4)
    kw = dict(t_eq=T_EQ, t_obs=T_OBS, rel_bracket=0.02, max_probes=24)
    lo, hi = sweep.analytic_brackets(specs)
    host, _ = sweep.run_sweep(lbm, specs, lo, hi, table=table, **kw)
    lib, _ = sweep.run_channels(lbm, specs, table=table, sigma=wetting.SIGMA, rho=wetting.RHO_BULK, **kw)
    for k, (h, c) in enumerate(zip(host, lib)):
        assert (c["g_lo"], c["g_hi"], c["probes"], c["status"]) == (h["g_lo"], h["g_hi"], h["probes"],
                                                                    h["status"]), k
        assert (c["g_start_lo"], c["g_start_hi"]) == (lo[k], hi[k])
        assert c["rho_wall"] == table.potentials_for(specs[k].theta_deg)
        assert c["tau"] == sweep.relaxation_times(specs[k].visc_ratio)
        D = specs[k].h0 - specs[k].amp
        assert c["bo_lo"] == pytest.approx(wetting.RHO_BULK * c["g_lo"] * specs[k].nx * D / wetting.SIGMA,
                                           rel=1e-14)
    assert sum(r["status"] == 0 for r in lib) >= 9


def test_surface_tension_matches_the_oracle_laplace_fit(lbm):
    """lbm_surface_tension (four droplets, radius from the mid-density
    crossings, pressure from the equation of state, least squares) lands
    within 1 % of the oracle's Laplace fit over five droplets with tanh-fitted
    radii (tests/golden/laplace_droplets_128.json); the bulk total density
    (middle of a flat interface's phase) within 0.2 % of the oracle's
    flat-interface coexistence value 1.0116 + 0.0303."""
    with open(os.path.join(GOLDEN, "laplace_droplets_128.json")) as fh:
        gold = json.load(fh)
    sigma, rho_bulk = lbm.lbm_surface_tension(steps=gold["steps"])
    assert sigma == pytest.approx(gold["sigma"], rel=1e-2)
    assert rho_bulk == pytest.approx(1.0116 + 0.0303, rel=2e-3)


def test_default_calibration_and_bond_numbers(lbm, table):
    """Without a table or a surface tension the library calibrates and
    measures on its own (cached per device): the wall potentials equal
    those of an explicit calibration, and Bo = rho g L D / sigma with the
    measured sigma and rho."""
    specs = sweep.small_specs(4, seed=9)
    res, _ = sweep.run_channels(lbm, specs, t_eq=T_EQ, t_obs=T_OBS)
    sigma, rho_bulk = lbm.lbm_surface_tension()
    for s, r in zip(specs, res):
        np.testing.assert_allclose(r["rho_wall"], table.potentials_for(s.theta_deg), rtol=0, atol=1e-9)
        assert r["sigma"] == sigma and r["rho_bulk"] == rho_bulk
        D = s.h0 - s.amp
        assert r["bo_hi"] == pytest.approx(rho_bulk * r["g_hi"] * s.nx * D / sigma, rel=1e-14)


def test_channel_call_with_the_surrogate(lbm, table):
    """use_surrogate: the starting bracket is the network's exp(mu -+ 2
    sigma) of the normalised features (the host helper computes the same
    bracket from the same network), and the bisection from it ends where the
    planar-bracket bisection ends (the brackets overlap or touch)."""
    specs = sweep.small_specs(8, seed=6)
    train = sweep.small_specs(64, seed=7)
    res_t, _ = sweep.run_channels(lbm, train, table=table, sigma=wetting.SIGMA, rho=wetting.RHO_BULK,
                                  t_eq=T_EQ, t_obs=T_OBS)
    ok = [k for k, r in enumerate(res_t) if r["status"] == 0]
    x = np.stack([sweep.features(train[k]) for k in ok])
    y = np.array([0.5 * math.log(res_t[k]["g_lo"] * res_t[k]["g_hi"]) for k in ok])
    scale = (x.mean(axis=0), x.std(axis=0) + 1e-12)
    net = lbm.Surrogate(seed=0)
    try:
        net.train((x - scale[0]) / scale[1], y, epochs=200, batch=32, lr=2e-3, seed=0)
        lo, hi = sweep.surrogate_brackets(net, specs, (scale[0].astype(np.float32), scale[1].astype(np.float32)))
        res_s, _ = sweep.run_channels(lbm, specs, table=table, sigma=wetting.SIGMA, rho=wetting.RHO_BULK,
                                      surrogate=net, scale_x=scale, t_eq=T_EQ, t_obs=T_OBS)
    finally:
        net.close()
    res_p, _ = sweep.run_channels(lbm, specs, table=table, sigma=wetting.SIGMA, rho=wetting.RHO_BULK,
                                  t_eq=T_EQ, t_obs=T_OBS)
    for k, (s, p) in enumerate(zip(res_s, res_p)):
        assert s["g_start_lo"] == pytest.approx(lo[k], rel=1e-6) and s["g_start_hi"] == pytest.approx(hi[k], rel=1e-6)
        if s["status"] == 0 and p["status"] == 0:
            assert s["g_lo"] <= p["g_hi"] * 1.0001 and p["g_lo"] <= s["g_hi"] * 1.0001, (k, s, p)


def test_channel_call_rejects_bad_specs(lbm):
    bad = wl.ChannelSpec(lam=4, amp_ratio=0.5, slug_len_over_lambda=1.0, theta_deg=60.0, visc_ratio=1.0)
    with pytest.raises(lbm.LbmError) as err:
        lbm.lbm_critical_pressure_channels([bad], t_eq=10, t_obs=10)
    assert err.value.code == lbm.LBM_EINVAL


def test_two_slugs_need_twice_the_force_of_one(lbm, table):
    """Multiple slugs (the paper's closing outlook): two identical slugs in
    a four-period channel against one, at the resolution where the protocol
    converges (lambda = 128, 80 000 steps at g = 0, 320 000 per probe).  The
    planar balance over the period says the force doubles (each slug holds
    the same capillary jump); the bisected forces are each within 15 % of
    their planar balance and their ratio within 10 % of 2."""
    specs = [wl.ChannelSpec(lam=128, amp_ratio=0.5, slug_len_over_lambda=1.5, theta_deg=60.0, visc_ratio=1.0,
                            n_slugs=k) for k in (1, 2)]
    res, _ = sweep.run_channels(lbm, specs, table=table, sigma=wetting.SIGMA, rho=wetting.RHO_BULK,
                                t_eq=80000, t_obs=320000, max_probes=30)
    g = []
    for r in res:
        assert r["status"] == 0, r
        gc = math.sqrt(r["g_lo"] * r["g_hi"])
        assert gc == pytest.approx(r["g_analytic"], rel=0.15), r
        g.append(gc)
    assert g[1] / g[0] == pytest.approx(2.0, rel=0.10), g


def test_equilibrated_slug_area(lbm, table):
    """The slug volume of Section 3.4, measured as the paper does: a slug of
    the lambda = 128 channel (A/h0 = 0.5, 1.5 lambda long, 60 degrees) after
    80 000 steps at g = 0 keeps the oil-rich area of its initial fill to 3 %
    (the menisci round off; oil dissolves at the coexistence density); the
    paper's bulk + 90 % count is smaller (the 1/2 - 9/10 band along each
    meniscus) but within 10 %; and the planar balance of the measured area
    is within 10 % of the balance of the initial fill's area (measured: 5.5 %
    higher; the balance is steep in the area at this slug length)."""
    spec = wl.ChannelSpec(lam=128, amp_ratio=0.5, slug_len_over_lambda=1.5, theta_deg=60.0, visc_ratio=1.0)
    inst = sweep.instance_of(spec, table)
    sim = lbm.Simulation(inst["mask"], inst["rho_init"], tau=inst["tau"], G=inst["G"], rho_wall=inst["rho_wall"],
                         periodic=inst["periodic"], precision="fp32", collision=inst["collision"])
    try:
        a_init = lbm.lbm_slug_area(inst["rho_init"], inst["mask"])
        sim.step(80000)
        rho, _, _ = sim.fields()
    finally:
        sim.close()
    a_half, a_paper = lbm.lbm_slug_area(rho, inst["mask"])
    area0, x_rest = wetting.initial_fill(spec)
    assert a_init[0] == pytest.approx(area0, rel=0.02)
    assert a_half == pytest.approx(area0, rel=0.03), (a_half, area0)
    assert 0.9 * a_half < a_paper < a_half
    bal0 = wetting.critical_balance(60.0, area0, spec.h0, spec.amp, float(spec.lam), x_rest)
    bal = wetting.critical_balance(60.0, a_half, spec.h0, spec.amp, float(spec.lam), x_rest)
    assert bal == pytest.approx(bal0, rel=0.10), (bal, bal0, a_half, area0)
