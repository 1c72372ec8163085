"""Host-side parts of the wetting and channel calls of the library
(lbm_contact_angle, lbm_wall_potentials, lbm_planar_critical_balance,
lbm_channel_geometry; no GPU) through paper_1601_00918_gb300/wetting.py,
against the oracle's capillary tools and the shared input module: the
contact-angle measurement on synthetic interfaces, the inversion of the
calibration table, the planar 2-D critical balance and the channel
geometry."""
import math

import numpy as np
import pytest

from oracle import capillary as cap
from paper_1601_00918_gb300 import wetting


def synthetic_slug_end(theta_deg, H=32, nx=160):
    """Oil fraction of an ideal right slug end meeting flat walls at theta
    through water (circle from Eq. contact_angle), tanh width 2."""
    y0 = H / 2.0
    th = math.radians(theta_deg)
    acute = min(th, math.pi - th)
    R = y0 / math.cos(acute)
    x_axis, y_a = 80.0, (1 + H) / 2.0
    ys, xs = np.mgrid[0:H + 2, 0:nx].astype(np.float64)
    if abs(theta_deg - 90.0) < 1e-9:
        d = xs - x_axis
    elif th < 0.5 * math.pi:
        d = np.hypot(xs - (x_axis - R), ys - y_a) - R
    else:
        xc = x_axis + R
        d = np.where(xs > xc, R, R - np.hypot(xs - xc, ys - y_a))
    frac = np.minimum(0.5 * (1.0 - np.tanh(d / 2.0)), 0.5 * (1.0 + np.tanh((xs - 20.0) / 2.0)))
    rho_o = 0.03 + 0.97 * frac
    return rho_o, 1.03 - rho_o


@pytest.mark.parametrize("theta_deg", [30.0, 55.0, 90.0, 125.0, 150.0])
def test_contact_angle_of_synthetic_interfaces(theta_deg):
    ro, rw = synthetic_slug_end(theta_deg)
    assert wetting.contact_angle(ro, rw, 1, 32, "right") == pytest.approx(theta_deg, abs=0.5)


def test_potentials_for_inverts_the_table():
    tab = wetting.WettingTable(np.array([-0.4, 0.0, 0.4]), np.array([135.0, 90.0, 45.0]), 32, 1000)
    assert tab.potentials_for(90.0) == (0.0, 0.0)
    assert tab.potentials_for(67.5) == pytest.approx((0.0, 0.2))
    assert tab.potentials_for(112.5) == pytest.approx((0.2, 0.0))
    assert tab.potentials_for(10.0) == pytest.approx((0.0, 0.4))        # clipped to the table


@pytest.mark.parametrize("r,theta,theta_deg", [
    ([-0.4, 0.0, 0.4], [135.0, 90.0, 45.0], float("nan")),
    ([-0.4, float("nan"), 0.4], [135.0, 90.0, 45.0], 60.0),
    ([-float("inf"), 0.0, 0.4], [135.0, 90.0, 45.0], 60.0),
    ([-0.4, 0.0, 0.4], [135.0, 90.0, -float("inf")], 60.0),
    ([-0.4, 0.4, 0.0], [135.0, 90.0, 45.0], 60.0),
    ([-0.4, 0.0, 0.4], [45.0, 90.0, 135.0], 60.0),
    ([0.0], [90.0], 60.0),
])
def test_wall_potentials_reject_bad_tables(r, theta, theta_deg):
    """The table inversion refuses a contact angle or a table entry that is
    not finite, and a table that is not ascending in r and descending in
    theta (LBM_EINVAL), instead of returning interpolated garbage."""
    from paper_1601_00918_gb300 import lbm
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_wall_potentials(np.array(r), np.array(theta), theta_deg)
    assert e.value.code == lbm.LBM_EINVAL


@pytest.mark.parametrize("theta_deg,area,x_rest", [(40.0, 2612.0, 77.4), (60.0, 2528.0, 80.0),
                                                   (90.0, 2600.0, 79.7), (120.0, 2576.0, 81.3),
                                                   (140.0, 2560.0, 82.4)])
def test_critical_balance_matches_the_oracle(theta_deg, area, x_rest):
    ref = cap.critical_force(math.radians(theta_deg), area, 12.0, 6.0, 64.0, x_rest)[0]
    assert wetting.critical_balance(theta_deg, area, 12.0, 6.0, 64.0, x_rest) == pytest.approx(ref, rel=2e-3)


@pytest.mark.parametrize("lam,ratio,slug,periods", [(32, 0.2, 1.0, 4), (64, 0.5, 1.5, 4), (128, 0.6, 2.0, 4),
                                                    (48, 0.37, 1.3, 3), (40, 0.0, 0.8, 2)])
def test_channel_geometry_is_the_input_module_channel(lam, ratio, slug, periods):
    """lbm_channel_geometry builds the same channel and slug as the shared
    input module (workloads.channel_instance): the mask exactly, the
    densities to the rounding of tanh."""
    from paper_1601_00918_gb300 import lbm
    from paper_1601_00918_gb300 import workloads as wl
    spec = wl.ChannelSpec(lam=lam, amp_ratio=ratio, slug_len_over_lambda=slug, theta_deg=70.0, visc_ratio=2.0,
                          n_periods=periods)
    mask, rho = lbm.lbm_channel_geometry(spec)
    w = wl.channel_instance(spec)
    np.testing.assert_array_equal(mask, w.mask)
    np.testing.assert_allclose(rho, w.rho, rtol=0, atol=1e-15)


@pytest.mark.parametrize("lam,periods,slugs,slug", [(32, 4, 2, 1.5), (64, 6, 3, 1.2), (48, 8, 4, 1.75),
                                                    (40, 4, 4, 0.5)])
def test_multi_slug_geometry_is_the_input_module_channel(lam, periods, slugs, slug):
    """Several identical slugs on equally spaced necks: the library's channel
    equals the shared input module's, mask exactly, densities to the
    rounding of tanh."""
    from paper_1601_00918_gb300 import lbm
    from paper_1601_00918_gb300 import workloads as wl
    spec = wl.ChannelSpec(lam=lam, amp_ratio=0.4, slug_len_over_lambda=slug, theta_deg=50.0, visc_ratio=1.0,
                          n_periods=periods, n_slugs=slugs)
    mask, rho = lbm.lbm_channel_geometry(spec)
    w = wl.channel_instance(spec)
    np.testing.assert_array_equal(mask, w.mask)
    np.testing.assert_allclose(rho, w.rho, rtol=0, atol=1e-15)
    # the oil is split into `slugs` runs along the centre row
    row = rho[0, spec.ny // 2] > 0.5
    assert int(np.sum(row[1:] & ~row[:-1]) + (row[0] and not row[-1])) == slugs


def test_planar_force_adds_up_over_identical_slugs():
    """Every slug holds the same capillary balance, so k identical slugs in
    a period need k times the force of one (Section 3.4 balance over the
    period, rho g L = sum of the slugs' capillary jumps): two slugs in four
    periods need exactly the force of one slug in two periods, and twice
    that of one slug in four."""
    from paper_1601_00918_gb300 import workloads as wl
    one4 = wl.ChannelSpec(lam=64, amp_ratio=0.5, slug_len_over_lambda=1.5, theta_deg=60.0, visc_ratio=1.0)
    one2 = wl.ChannelSpec(lam=64, amp_ratio=0.5, slug_len_over_lambda=1.5, theta_deg=60.0, visc_ratio=1.0,
                          n_periods=2)
    two4 = wl.ChannelSpec(lam=64, amp_ratio=0.5, slug_len_over_lambda=1.5, theta_deg=60.0, visc_ratio=1.0,
                          n_slugs=2)
    g1, g12, g2 = (wetting.analytic_g_crit(s, 60.0) for s in (one4, one2, two4))
    assert g2 == pytest.approx(g12, rel=1e-12)
    assert g2 == pytest.approx(2.0 * g1, rel=1e-12)


def _synthetic_slug(lam, h0, amp, x_r, x_f, th_r, th_f, w=2.0):
    """Densities of a slug in the planar sinusoidal channel whose menisci are
    the arcs of the Section 3.4 planar model: centred on the axis, meeting
    the wall (inclined by atan h'(x)) at the given contact positions and
    angles through water; tanh interfaces of width w."""
    k = 2 * math.pi / lam
    ny = 2 * int(math.ceil(h0 + amp)) + 2
    nx = 4 * lam
    yc = (ny - 1) / 2.0
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))

    def end(xc, th, front):
        h = h0 - amp * math.cos(k * xc)
        phi = math.atan(amp * k * math.sin(k * xc))
        al = 0.5 * math.pi + (phi if front else -phi) - math.radians(th)
        R = h / math.sin(al)
        xm = xc - R * math.cos(al) if front else xc + R * math.cos(al)
        dist = np.hypot(X - xm, Y - yc)
        beyond = (X - xm) if front else (xm - X)
        s = np.minimum(dist - abs(R), beyond) if al > 0 else np.maximum(abs(R) - dist, beyond)
        return 0.5 * (1 - np.tanh(s / w))

    frac = np.minimum(end(x_f, th_f, True), end(x_r, th_r, False))
    ro = 0.03 + 0.97 * frac
    return np.stack([ro, 1.03 - ro])


@pytest.mark.parametrize("th_r,th_f", [(40.0, 40.0), (60.0, 52.0), (75.0, 88.0), (120.0, 118.0), (140.0, 139.0)])
def test_meniscus_angles_of_synthetic_arcs(th_r, th_f):
    """lbm_meniscus_angles recovers the contact angles (to 0.5 degree) and
    contact positions (to 0.1 node) of a slug whose menisci are planar-model
    arcs meeting the inclined walls of a lambda = 128 channel."""
    from paper_1601_00918_gb300 import lbm
    rho = _synthetic_slug(128, 24.0, 12.0, 180.3, 390.7, th_r, th_f)
    m = lbm.lbm_meniscus_angles(rho, 24.0, 12.0, 128.0)
    assert m["theta_rear"] == pytest.approx(th_r, abs=0.5)
    assert m["theta_front"] == pytest.approx(th_f, abs=0.5)
    assert m["x_rear"] == pytest.approx(180.3, abs=0.1) and m["x_front"] == pytest.approx(390.7, abs=0.1)


@pytest.mark.parametrize("theta", [40.0, 90.0, 140.0])
def test_hysteresis_balance(theta):
    """Equal front and rear angles give the static balance; a receding
    (front) water angle below the advancing (rear) one raises the force
    the slug can hold (the analysis with Delta theta != 0); the reverse
    lowers it."""
    from paper_1601_00918_gb300 import lbm
    args = (2600.0, 12.0, 6.0, 64.0, 79.7)
    b0 = lbm.lbm_planar_critical_balance(theta, *args)
    assert lbm.lbm_planar_critical_balance_hysteresis(theta, theta, *args) == b0
    assert lbm.lbm_planar_critical_balance_hysteresis(theta - 4.0, theta + 4.0, *args) > b0
    assert lbm.lbm_planar_critical_balance_hysteresis(theta + 4.0, theta - 4.0, *args) < b0


def test_slug_area_rules():
    """lbm_slug_area on planar-model slugs between two necks of a lambda =
    128 channel (rear meniscus at x = 128, front at 256, 60 degrees): the
    oil-rich count equals the model's oil area (channel area between the
    contact points plus the two circular segments, oracle/capillary.py) to
    1.5 %; with sharp interfaces (width 0.05) the paper's bulk + 90 % rule
    gives the same count but for the few nodes within 0.06 of a meniscus;
    with tanh interfaces of width 2 it leaves out the band between the
    1/2 and 9/10 oil-fraction levels, 2 atanh(0.8) = 2.197 nodes thick along
    each meniscus, whose arc at a neck (wall slope zero) is 2 h (pi/2 -
    theta) / cos(theta) long (within 25 %).  A flat meniscus (90 degrees at a
    neck) crosses no column, so the two rules agree."""
    from paper_1601_00918_gb300 import lbm
    from paper_1601_00918_gb300 import workloads as wl
    lam, h0, amp, th = 128, 24.0, 12.0, 60.0
    ny = 2 * int(math.ceil(h0 + amp)) + 2
    mask = wl.sinusoidal_channel(4 * lam, ny, h0, amp, float(lam))
    sharp = _synthetic_slug(lam, h0, amp, 128.0, 256.0, th, th, w=0.05)
    smooth = _synthetic_slug(lam, h0, amp, 128.0, 256.0, th, th, w=2.0)
    a_sharp = lbm.lbm_slug_area(sharp, mask)
    a_smooth = lbm.lbm_slug_area(smooth, mask)
    model = cap.oil_area(128.0, 256.0, math.radians(th), h0, amp, float(lam))
    assert a_sharp[0] == pytest.approx(model, rel=0.015), (a_sharp, model)
    assert a_smooth[0] == pytest.approx(model, rel=0.015), (a_smooth, model)
    assert 0 <= a_sharp[0] - a_sharp[1] <= 10
    neck = h0 - amp
    arc = 2.0 * neck * (0.5 * math.pi - math.radians(th)) / math.cos(math.radians(th))
    band = 2.0 * math.atanh(0.8) * 2.0 * arc
    assert a_smooth[0] - a_smooth[1] == pytest.approx(band, rel=0.25), (a_smooth, band)
    flat = _synthetic_slug(lam, h0, amp, 128.0, 256.0, 90.0, 90.0, w=2.0)
    a_flat = lbm.lbm_slug_area(flat, mask)
    assert a_flat[0] == a_flat[1]
