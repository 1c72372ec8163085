"""Host-side set-up of the critical-force sweeps (paper_1601_00918_gb300/sweep.py,
no GPU): relaxation times from the viscosity ratio, wall potentials from the
contact angle, the batch instance of a channel description, the surrogate's
features and brackets, and the analytic starting bracket."""
import math

import numpy as np
import pytest

from oracle import capillary as cap
from paper_1601_00918_gb300 import sweep
from paper_1601_00918_gb300 import workloads as wl


@pytest.mark.parametrize("r", [0.5, 1.0, 2.5, 10.0])
def test_relaxation_times_give_the_viscosity_ratio(r):
    tau_o, tau_w = sweep.relaxation_times(r)
    assert tau_w == 1.0
    assert (tau_o - 0.5) / (tau_w - 0.5) == pytest.approx(r, rel=1e-12)


def test_relaxation_time_floor():
    assert sweep.relaxation_times(0.2)[0] == sweep.TAU_MIN


@pytest.mark.parametrize("theta", [20.0, 60.0, 89.0, 120.0, 160.0])
def test_wall_potentials_follow_the_wettability(theta):
    ro, rw = sweep.wall_potentials(theta)
    assert min(ro, rw) == 0.0 and max(ro, rw) <= sweep.RHO_S_MAX
    if theta < 90.0:
        assert rw > 0.0                       # water-wet: the wall attracts water
    else:
        assert ro > 0.0
    # the swap symmetry of the angle: theta <-> 180 - theta swaps the species
    assert sweep.wall_potentials(180.0 - theta) == pytest.approx((rw, ro))
    assert sweep.wall_potentials(90.0) == pytest.approx((0.0, 0.0), abs=1e-16)


def test_instance_of_a_channel_description():
    spec = wl.ChannelSpec(lam=64, amp_ratio=0.4, slug_len_over_lambda=1.5, theta_deg=50.0, visc_ratio=2.0)
    d = sweep.instance_of(spec)
    ny, nx = d["mask"].shape
    assert (nx, ny) == (spec.nx, spec.ny) == (256, 2 * math.ceil(spec.h0 + spec.amp) + 2)
    assert d["periodic"] == (True, False)
    assert d["mask"][0].all() and d["mask"][-1].all()
    assert d["disp_threshold"] == 32.0 and d["collision"] == sweep.COLLISION
    assert d["tau"] == sweep.relaxation_times(2.0) and d["rho_wall"] == sweep.wall_potentials(50.0)
    fluid = d["mask"] == 0
    assert np.all(d["rho_init"][:, fluid] > 0.0)
    # the slug (oil-rich) is centred on the neck at x = 2 lambda
    oil = d["rho_init"][0, ny // 2] > d["rho_init"][1, ny // 2]
    xs = np.nonzero(oil)[0]
    assert 0.5 * (xs.min() + xs.max()) == pytest.approx(2 * spec.lam, abs=1.0)


def test_features_are_order_one_and_exact():
    spec = wl.ChannelSpec(lam=128, amp_ratio=0.3, slug_len_over_lambda=1.2, theta_deg=120.0, visc_ratio=0.5)
    f = sweep.features(spec)
    assert f.shape == (5,)
    neck = 2.0 * (spec.h0 - spec.amp)
    assert f == pytest.approx([0.3, 1.2, math.cos(math.radians(120.0)), math.log(0.5), 1.0 / neck])


class _FixedNet:
    """Stands in for the surrogate: returns fixed (mu, log variance)."""

    def __init__(self, mu, s):
        self.mu, self.s = mu, s

    def forward(self, x):
        out = np.empty((len(x), 2), dtype=np.float32)
        out[:, 0], out[:, 1] = self.mu, self.s
        return out


def test_surrogate_brackets_are_two_sigma_and_at_least_the_floor():
    specs = wl.sweep_specs(3, seed=4)
    scale = (np.zeros(5), np.ones(5))
    lo, hi = sweep.surrogate_brackets(_FixedNet(math.log(2e-5), 2.0 * math.log(0.1)), specs, scale)
    assert lo == pytest.approx(2e-5 * math.exp(-0.2), rel=1e-6)
    assert hi == pytest.approx(2e-5 * math.exp(0.2), rel=1e-6)
    lo, hi = sweep.surrogate_brackets(_FixedNet(math.log(2e-5), -40.0), specs, scale, floor=1.05)
    assert hi / lo == pytest.approx(1.05, rel=1e-6)


def test_analytic_bracket_is_the_planar_balance_of_the_initial_slug():
    """The starting bracket's centre is the oracle's planar 2-D critical force
    of the initial fill: oil area = the channel area between the slug ends
    (no meniscus segments in the sharp initial fill), rest position at the
    rear end, scaled by sigma / (rho L)."""
    from paper_1601_00918_gb300 import wetting
    spec = wl.ChannelSpec(lam=64, amp_ratio=0.5, slug_len_over_lambda=1.5, theta_deg=60.0, visc_ratio=1.0)
    lam, half = 64.0, 0.75 * 64.0
    area = cap.channel_area(2 * lam - half, 2 * lam + half, spec.h0, spec.amp, lam)
    bal = cap.critical_force(math.radians(60.0), area, spec.h0, spec.amp, lam, 2 * lam - half)[0]
    ref = wetting.SIGMA * bal / (wetting.RHO_BULK * spec.nx)
    assert wetting.analytic_g_crit(spec, 60.0) == pytest.approx(ref, rel=3e-3)
    lo, hi = sweep.analytic_brackets([spec])
    assert lo[0] == pytest.approx(0.5 * wetting.analytic_g_crit(spec, 60.0))
    assert hi[0] == pytest.approx(2.0 * wetting.analytic_g_crit(spec, 60.0))
    # a straight channel needs no force
    flat = wl.ChannelSpec(lam=64, amp_ratio=1e-9, slug_len_over_lambda=1.5, theta_deg=60.0, visc_ratio=1.0)
    assert abs(wetting.analytic_g_crit(flat, 60.0)) < 1e-9 * ref
