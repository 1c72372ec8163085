"""Host-side parts of paper_1601_00918_gb300/wetting.py against the oracle's
capillary tools (no GPU): the contact-angle measurement on synthetic
interfaces and the planar 2-D critical balance."""
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


def test_circle_through_points():
    t = np.linspace(-1.0, 0.4, 30)
    A, B, C, D = wetting.circle_through(5.0 + 25.0 * np.cos(t), 1.5 + 25.0 * np.sin(t))
    assert (-B / (2 * A), -C / (2 * A), 1.0 / (2 * abs(A))) == pytest.approx((5.0, 1.5, 25.0), abs=1e-8)
    # collinear points: a line (A = 0)
    A, B, C, D = wetting.circle_through(np.full(9, 3.0), np.arange(9.0))
    assert abs(A) < 1e-12 and abs(C) < 1e-9


def test_potentials_for_inverts_the_table():
    tab = wetting.WettingTable(np.array([-0.4, 0.0, 0.4]), np.array([135.0, 90.0, 45.0]), 32, 1000)
    assert tab.potentials_for(90.0) == (0.0, 0.0)
    assert tab.potentials_for(67.5) == pytest.approx((0.0, 0.2))
    assert tab.potentials_for(112.5) == pytest.approx((0.2, 0.0))
    assert tab.potentials_for(10.0) == pytest.approx((0.0, 0.4))        # clipped to the table


@pytest.mark.parametrize("theta_deg,area,x_rest", [(40.0, 2612.0, 77.4), (60.0, 2528.0, 80.0),
                                                   (90.0, 2600.0, 79.7), (120.0, 2576.0, 81.3),
                                                   (140.0, 2560.0, 82.4)])
def test_critical_balance_matches_the_oracle(theta_deg, area, x_rest):
    ref = cap.critical_force(math.radians(theta_deg), area, 12.0, 6.0, 64.0, x_rest)[0]
    assert wetting.critical_balance(theta_deg, area, 12.0, 6.0, 64.0, x_rest) == pytest.approx(ref, rel=2e-3)
