"""Pins of the oracle's capillary tools (oracle/capillary.py): the contact
angle of Section 3.3 and the planar 2-D critical body force derived from the
balance of Section 3.4.

The meniscus formulas are checked against a brute-force construction of the
circle and a quadrature of its segment; the critical force against two
closed-form limits (long wavelength: the Jamin-type difference of the two
curvatures; small amplitude: the wall-slope term alone); the contact angle
against a synthetic circular interface and against the symmetries of the
oracle's LBM (equal wall potentials give 90 degrees; swapping the species'
wall potentials gives 180 degrees minus the angle).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import capillary as cap
from paper_1601_00918_gb300 import workloads as wl

G_REPULSIVE = -1.79


# ----------------------------------------------------------------------------
# one meniscus: closed forms against the circle built point by point
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("theta_deg,phi_deg,h", [(30, 0, 8.0), (55, 20, 6.0), (120, -15, 10.0),
                                                 (80, 25, 5.0), (150, 10, 12.0), (95, -30, 7.0),
                                                 (20, 28, 6.0)])
def test_front_meniscus_against_constructed_circle(theta_deg, phi_deg, h):
    """A front meniscus with its chord at x = 0, contact points (0, +-h),
    oil at x < 0 near the axis, is an arc of an axis-centred circle (c, 0)
    whose tangent at (0, h) makes the angle theta, through the water, with
    the wall ray of angle phi.  Either the arc through (c + R, 0) (bulging
    into the water, oil encloses the centre: kappa = +1/R; a major arc when
    c > 0) covers theta - phi in (-90, 90) degrees, or the arc through
    (c - R, 0) with c > 0 (bulging into the oil: kappa = -1/R) covers (90,
    180).  c is found by bisection on the angle; the oil area beyond the
    chord is the shoelace area of the arc closed by the chord."""
    th, ph = math.radians(theta_deg), math.radians(phi_deg)
    right = th - ph < 0.5 * math.pi

    def water_angle(c):
        if right:       # ray from (0, h) along the arc: direction (h, c) / R
            return ph - math.atan2(c, h)
        return ph - math.atan2(-c, -h)      # direction (-h, -c) / R

    lo, hi = (-1e6, 1e6) if right else (1e-12, 1e6)
    for _ in range(300):
        mid = 0.5 * (lo + hi)
        # on either arc the water angle decreases as the centre moves right
        if water_angle(mid) > th:
            lo = mid
        else:
            hi = mid
    c = 0.5 * (lo + hi)
    R = math.hypot(c, h)
    beta = math.atan2(h, -c)                # angle of (0, h) seen from the centre
    if right:
        t = np.linspace(-beta, beta, 400001)
        sign, kappa_ref = 1.0, 1.0 / R
    else:
        t = np.linspace(beta, 2.0 * math.pi - beta, 400001)
        sign, kappa_ref = -1.0, -1.0 / R
    xs = np.concatenate([c + R * np.cos(t), [0.0]])
    ys = np.concatenate([R * np.sin(t), [-h if right else h]])
    shoelace = 0.5 * float(np.sum(xs * np.roll(ys, -1) - np.roll(xs, -1) * ys))
    seg_ref = sign * abs(shoelace)
    kappa, seg = cap.meniscus(th, ph, h, front=True)
    assert float(kappa) == pytest.approx(kappa_ref, rel=1e-9, abs=1e-12)
    assert float(seg) == pytest.approx(seg_ref, rel=1e-6, abs=1e-6)


def test_channel_area_is_the_integral_of_twice_the_half_width():
    xs = np.linspace(3.0, 151.0, 400001)
    h = cap.half_width(xs, 12.0, 5.0, 64.0)
    quad = float(np.sum(0.5 * (h[1:] + h[:-1]) * np.diff(xs))) * 2.0
    assert cap.channel_area(3.0, 151.0, 12.0, 5.0, 64.0) == pytest.approx(quad, rel=1e-9)


# ----------------------------------------------------------------------------
# the balance of Section 3.4 in its limits
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("theta_deg", [20, 60, 90, 140])
def test_balance_vanishes_in_a_straight_channel_and_for_symmetric_slugs(theta_deg):
    th = math.radians(theta_deg)
    assert np.max(np.abs(cap.capillary_balance(np.linspace(0, 64, 9), np.linspace(96, 160, 9), th,
                                               12.0, 0.0, 64.0))) < 1e-15
    g, _, _, _ = cap.critical_force(th, cap.channel_area(0, 96, 12.0, 0.0, 64.0), 12.0, 0.0, 64.0, 40.0)
    assert g == 0.0
    # a slug symmetric about a neck (x = 128) or a bulge (x = 96) is at rest
    for centre in (128.0, 96.0):
        for half in (20.0, 37.5, 50.0):
            b = cap.capillary_balance(centre - half, centre + half, th, 12.0, 6.0, 64.0)
            assert abs(float(b)) < 1e-14


@pytest.mark.parametrize("theta_deg", [25, 50, 75])
def test_long_wavelength_limit_is_the_curvature_difference(theta_deg):
    """lambda >> h: walls are flat where the menisci sit, so the largest
    balance of a half-wavelength slug is cos(theta) [1/(h0 - A) - 1/(h0 + A)]
    (front at a neck, rear at a bulge)."""
    th = math.radians(theta_deg)
    h0, amp, lam = 10.0, 4.0, 2.0e5
    area = cap.channel_area(0.5 * lam, lam, h0, amp, lam)
    g, s0, smax, _ = cap.critical_force(th, area, h0, amp, lam, x_rest=0.25 * lam, n=2001)
    ref = math.cos(th) * (1.0 / (h0 - amp) - 1.0 / (h0 + amp))
    assert g == pytest.approx(ref, rel=2e-3)


@pytest.mark.parametrize("theta_deg", [40, 90, 130])
def test_small_amplitude_limit_is_the_wall_slope_term(theta_deg):
    """A/h0 -> 0 with a slug whose chords are two wavelengths apart: both
    menisci see the same h and phi, so the balance is 2 sin(theta) sin(phi) /
    h, whose largest value on the loading path is 4 pi A sin(theta) / (lam
    h0) to first order in A (rear moving from a neck to the steepest point).
    The oil area of that slug at A = 0 is the channel between the chords plus
    two circular segments of half-chord h0 and half-angle 90 - theta (the
    textbook segment R^2 (2a - sin 2a) / 2, R = h0 / sin a)."""
    th = math.radians(theta_deg)
    h0, lam = 12.0, 64.0
    amp = 1e-3 * h0
    a = 0.5 * math.pi - th
    seg = 0.0 if abs(a) < 1e-12 else math.copysign((h0 / math.sin(abs(a))) ** 2 * (2 * abs(a) - math.sin(2 * abs(a))) / 2, a)
    area = 2.0 * h0 * 2.0 * lam + 2.0 * seg
    g, s0, smax, _ = cap.critical_force(th, area, h0, amp, lam, x_rest=lam, n=2881)
    ref = 4.0 * math.pi * amp * math.sin(th) / (lam * h0)
    assert g == pytest.approx(ref, rel=1e-2)
    assert s0 % lam == pytest.approx(0.0, abs=0.5) or s0 % lam == pytest.approx(lam, abs=0.5)
    assert (smax - s0) == pytest.approx(0.25 * lam, abs=1.0)


def test_water_wet_slug_on_a_neck_rests_symmetrically_and_needs_a_push():
    h0, amp, lam = 12.0, 6.0, 64.0
    area = cap.channel_area(80.0, 176.0, h0, amp, lam)
    g, s0, smax, (ss, xf, bal) = cap.critical_force(math.radians(40.0), area, h0, amp, lam, x_rest=80.0)
    xf0 = float(np.interp(s0, ss, xf))
    assert 0.5 * (s0 + xf0) == pytest.approx(128.0, abs=0.2)
    assert g > 0 and smax > s0


def _constructed_balance(points, lam):
    """Periodic piecewise-linear balance through (s / lam, value) points."""
    xs = np.array([p[0] for p in points] + [1.0]) * lam
    ys = np.array([p[1] for p in points] + [points[0][1]])
    return lambda s: np.interp(np.mod(s, lam), xs, ys)


def test_loading_path_on_a_constructed_balance():
    """The loading rule of the critical force on balances built by hand
    (the geometry replaced by a known periodic curve with its rest zero at
    s = 0): a first peak of 1.0 at 0.15 lam, a dip, a second peak of 1.5 at
    0.8 lam.  Loaded from rest the slug climbs to the first peak and jumps to
    where the balance is 1.0 again.  With a deep dip (to -0.5 at 0.3 lam)
    that point lies 0.525 lam ahead: longer than lam / 2, so the slug counts
    as moving at the first peak (1.0); with a shallow dip (0.6) it lies
    0.35 lam ahead, so the slug only moves on and escapes past the second
    peak (1.5), whose next equal value is a full period ahead.  With the
    threshold raised to 0.6 lam the deep-dip slug escapes at 1.5 too."""
    lam = 100.0
    deep = _constructed_balance([(0.0, 0.0), (0.15, 1.0), (0.3, -0.5), (0.8, 1.5), (0.9, -1.0)], lam)
    shallow = _constructed_balance([(0.0, 0.0), (0.15, 1.0), (0.3, 0.6), (0.8, 1.5), (0.9, -1.0)], lam)
    glb = cap.critical_force.__globals__     # the module the function reads its helpers from
    saved = glb["front_for"], glb["capillary_balance"]
    try:
        glb["front_for"] = lambda s, *a, **k: s + 1.0
        for bal, jump, expected in ((deep, None, 1.0), (shallow, None, 1.5), (deep, 0.6 * lam, 1.5)):
            glb["capillary_balance"] = lambda s, xf, *a, bal=bal: bal(np.asarray(s))
            g, s0, smax, _ = cap.critical_force(1.0, 50.0, 10.0, 5.0, lam, x_rest=0.0, jump=jump)
            assert s0 == pytest.approx(0.0, abs=1e-9)
            assert g == pytest.approx(expected, rel=1e-9), (jump, expected)
            assert smax == pytest.approx(0.15 * lam if expected == 1.0 else 0.8 * lam, abs=1e-6)
    finally:
        glb["front_for"], glb["capillary_balance"] = saved


# ----------------------------------------------------------------------------
# Section 3.3: contact angle
# ----------------------------------------------------------------------------
def test_circle_fit_recovers_a_circle():
    t = np.linspace(-0.9, 0.7, 25)
    pts = np.stack([3.0 + 40.0 * np.cos(t), -2.0 + 40.0 * np.sin(t)], axis=1)
    xc, yc, r = cap.fit_circle(pts)
    assert (xc, yc, r) == pytest.approx((3.0, -2.0, 40.0), abs=1e-6)


@pytest.mark.parametrize("theta_deg", [35.0, 70.0, 115.0, 150.0])
def test_contact_angle_of_a_synthetic_circular_interface(theta_deg):
    """Oil fraction field of an ideal right-end meniscus (tanh across a
    circle meeting the walls at theta through water, Eq. contact_angle
    inverted): the measured angle is theta."""
    H, nx = 32, 160
    y0 = H / 2.0
    th = math.radians(theta_deg)
    # circle centred on the axis y_a; R from Eq. (contact_angle): tan(theta) = sqrt(R^2 - y0^2) / y0
    acute = min(th, math.pi - th)
    R = y0 / math.cos(acute)
    x_axis, y_a = 80.0, (1 + H) / 2.0
    ys, xs = np.mgrid[0:H + 2, 0:nx].astype(np.float64)
    if th < 0.5 * math.pi:     # centre on the oil side (left): the interface bulges into the water
        xc = x_axis - R
        d = np.hypot(xs - xc, ys - y_a) - R              # > 0 in the water
    else:
        xc = x_axis + R
        d = np.where(xs > xc, R, R - np.hypot(xs - xc, ys - y_a))     # water: inside the circle or beyond it
    frac = 0.5 * (1.0 - np.tanh(d / 2.0))
    left = 0.5 * (1.0 + np.tanh((xs - 20.0) / 2.0))
    frac = np.minimum(frac, left)
    rho_o = 0.03 + 0.97 * frac
    rho_w = 1.03 - rho_o
    got = cap.contact_angle(rho_o, rho_w, 1, H, side="right")
    assert got == pytest.approx(theta_deg, abs=0.3)


def flat_plate_slug(rho_wall, steps=4000, H=16, nx=96):
    mask = wl.straight_channel(nx, H)
    rho = wl.slug(nx, H + 2, 24, 72)
    P = oracle.Problem(mask, tau=(1.0, 1.0), G=G_REPULSIVE, rho_wall=rho_wall, periodic=(True, False))
    r, _, _ = P.fields(P.run(P.init(rho), steps))
    return (cap.contact_angle(r[0], r[1], 1, H, "right"), cap.contact_angle(r[0], r[1], 1, H, "left"))


@pytest.mark.slow
def test_oracle_contact_angle_symmetries():
    """Section 3.3 set-up (slug between flat plates, H = 16) on the oracle:
    equal wall potentials give 90 degrees; a water-attracting wall gives
    theta < 90 and the same wall for oil gives 180 - theta (the paper's
    centre-of-symmetry property, exact here by the species swap symmetry);
    both ends of the slug agree; theta moves monotonically with the
    potential."""
    neutral = flat_plate_slug((0.0, 0.0))
    ww = flat_plate_slug((0.0, 0.3))
    ow = flat_plate_slug((0.3, 0.0))
    mild = flat_plate_slug((0.0, 0.15))
    for th in (neutral, ww, ow, mild):
        assert th[0] == pytest.approx(th[1], abs=0.05)
    assert neutral[0] == pytest.approx(90.0, abs=0.1)
    assert ww[0] + ow[0] == pytest.approx(180.0, abs=0.05)
    assert ww[0] < mild[0] < neutral[0]
    assert 40.0 < ww[0] < 70.0
