"""Contact angle and the 2-D critical body force of a static slug (Sections
3.3 and 3.4 of the paper), FP64, numpy/scipy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Contact angle (Section 3.3, Eq. contact_angle): in a slug between flat
plates the interface points are located row by row with the tanh fit of
Eq. (den-fitting); a circle is fitted through them and the angle follows
from its radius R and the half channel width y0, theta = arctan(sqrt(R^2 -
y0^2) / y0).  That arctan is the acute angle between wall and interface; it
is the angle through water when the circle's centre lies on the oil side
(the interface bulges into the water) and 180 degrees minus it otherwise.

Critical force (Section 3.4).  The paper quotes the 3-D result
Bo_crit = -2 D (H_wo + H_ow) with curvatures from a cited appendix that it
does not reproduce.  This module states the planar 2-D analogue, derived
from the same balance:
  * channel half-width h(x) = h0 - A cos(2 pi x / lam), wall angle
    phi(x) = atan h'(x), contact angle theta measured through water;
  * each meniscus is a circular arc centred on the axis; the jump across the
    front (advancing) meniscus at x_f is p_o - p_w = sigma cos(theta - phi_f)
    / h_f, across the rear (receding) one at x_r it is sigma cos(theta +
    phi_r) / h_r (the rear is the mirror image of a front);
  * static balance over one period L, dp/dx = rho g in both bulks:
        rho g L = sigma [cos(theta - phi_f) / h_f - cos(theta + phi_r) / h_r];
  * x_f follows x_r by conservation of the oil area: the area between the
    two contact chords plus the circular segments beyond them (positive
    where an arc bulges into the water);
  * the rest position s0 is a zero of the capillary balance with positive
    slope; loading g quasi-statically moves the slug forward along the
    branch where the balance equals rho g L / sigma; past a local maximum
    the slug jumps ahead to the next position where the balance is as large
    again.  The slug counts as moving once such a jump is longer than
    lam / 2, or no such position exists within the period ahead (the same
    "displacement > lam / 2" reading the bisection uses); g_crit is the
    balance at that local maximum, / (rho L).
The formulas here are evaluated by direct sampling (no root finder on the
balance) so they can be read against the statements above.
"""
from __future__ import annotations

import math

import numpy as np


# ----------------------------------------------------------------------------
# channel geometry
# ----------------------------------------------------------------------------
def half_width(x, h0: float, amp: float, lam: float):
    """h(x) = h0 - A cos(2 pi x / lam)."""
    return h0 - amp * np.cos(2.0 * math.pi * np.asarray(x, dtype=np.float64) / lam)


def wall_angle(x, h0: float, amp: float, lam: float):
    """phi(x) = atan h'(x), h'(x) = (2 pi A / lam) sin(2 pi x / lam)."""
    k = 2.0 * math.pi / lam
    return np.arctan(amp * k * np.sin(k * np.asarray(x, dtype=np.float64)))


def channel_area(a: float, b: float, h0: float, amp: float, lam: float) -> float:
    """Area between the walls from x = a to x = b: the integral of 2 h(x)."""
    k = 2.0 * math.pi / lam
    return 2.0 * (h0 * (b - a) - amp / k * (math.sin(k * b) - math.sin(k * a)))


# ----------------------------------------------------------------------------
# one meniscus
# ----------------------------------------------------------------------------
def meniscus(theta: float, phi, h, front: bool):
    """(signed curvature kappa, signed segment area) of a meniscus whose
    contact points are at half-width h on walls inclined by phi (arrays
    allowed).

    kappa = (p_o - p_w) / sigma: cos(theta - phi) / h at a front, cos(theta +
    phi) / h at a rear.  The arc is centred on the axis; seen from its centre
    the contact point lies at angle alpha = pi/2 + phi - theta from the
    channel direction (front; phi -> -phi at the rear), so R = h / |sin
    alpha| and the segment between chord and arc is R^2 (|alpha| - sin|alpha|
    cos|alpha|), oil (positive) when alpha > 0."""
    phi = np.asarray(phi, dtype=np.float64)
    h = np.asarray(h, dtype=np.float64)
    alpha = 0.5 * math.pi + (phi if front else -phi) - theta
    kappa = np.sin(alpha) / h
    a = np.abs(alpha)
    flat = a < 1e-6
    sa = np.where(flat, 1.0, np.sin(a))
    seg = np.where(flat, 0.0, (h / sa) ** 2 * (a - np.sin(a) * np.cos(a)))
    return kappa, np.copysign(seg, alpha)


def oil_area(xr, xf, theta: float, h0: float, amp: float, lam: float):
    """Oil area of a slug whose rear and front contact chords sit at xr < xf
    (xf may be an array)."""
    xr = np.asarray(xr, dtype=np.float64)
    xf = np.asarray(xf, dtype=np.float64)
    _, sr = meniscus(theta, wall_angle(xr, h0, amp, lam), half_width(xr, h0, amp, lam), front=False)
    _, sf = meniscus(theta, wall_angle(xf, h0, amp, lam), half_width(xf, h0, amp, lam), front=True)
    k = 2.0 * math.pi / lam
    between = 2.0 * (h0 * (xf - xr) - amp / k * (np.sin(k * xf) - np.sin(k * xr)))
    return between + sr + sf


def capillary_balance(xr, xf, theta: float, h0: float, amp: float, lam: float):
    """kappa_front - kappa_rear = (rho g L) / sigma at a static position."""
    kr, _ = meniscus(theta, wall_angle(xr, h0, amp, lam), half_width(xr, h0, amp, lam), False)
    kf, _ = meniscus(theta, wall_angle(xf, h0, amp, lam), half_width(xf, h0, amp, lam), True)
    return kf - kr


def front_for(xr: float, area: float, theta: float, h0: float, amp: float, lam: float,
              span: float, n: int = 4001) -> float:
    """Front chord position xf > xr with oil_area(xr, xf) = area: the area
    is sampled on xr < xf < xr + span and the first crossing interpolated."""
    xs = xr + np.linspace(1e-6, span, n)
    a = oil_area(xr, xs, theta, h0, amp, lam)
    k = np.nonzero((a[:-1] - area) * (a[1:] - area) <= 0.0)[0]
    if k.size == 0:
        raise ValueError("no front position holds that oil area")
    i = int(k[0])
    t = (area - a[i]) / (a[i + 1] - a[i])
    return float(xs[i] + t * (xs[i + 1] - xs[i]))


def critical_force(theta: float, area: float, h0: float, amp: float, lam: float, x_rest: float,
                   n: int = 1441, jump: float | None = None):
    """2-D critical body force of a static slug, in units of sigma / (rho L).

    The rear chord position s is sampled from x_rest - lam / 2 over two
    wavelengths; the rest position s0 is the zero of the balance with
    positive slope nearest to x_rest (the rear contact position of the slug
    at rest).  From s0 the loading path climbs to each local maximum in turn
    and jumps to the next sample ahead whose balance is at least as large;
    the first jump longer than `jump` (default lam / 2), or one that leaves
    the period ahead of s0, ends it: g_crit sigma / (rho L) is the balance
    there.  A balance that vanishes everywhere (a straight channel) gives 0.
    Returns (balance_crit, s0, s_at_crit, samples (s, xf, balance))."""
    span = area / (2.0 * max(h0 - amp, 1e-9)) + 2.0 * lam     # any slug fits in this window
    ss = x_rest + np.linspace(-0.5 * lam, 1.5 * lam, n)
    xf = np.array([front_for(s, area, theta, h0, amp, lam, span) for s in ss])
    bal = capillary_balance(ss, xf, theta, h0, amp, lam)
    if np.max(np.abs(bal)) < 1e-12:
        return 0.0, float(x_rest), float(x_rest), (ss, xf, bal)
    up = np.nonzero((bal[:-1] <= 0.0) & (bal[1:] > 0.0))[0]
    up = up[ss[up] <= x_rest + 0.5 * lam]
    if up.size == 0:
        raise ValueError("no stable rest position within half a wavelength")
    zs = ss[up] - bal[up] * (ss[up + 1] - ss[up]) / (bal[up + 1] - bal[up])
    k = int(np.argmin(np.abs(zs - x_rest)))
    s0 = float(zs[k])
    jump = 0.5 * lam if jump is None else jump
    j = int(up[k]) + 1
    while True:
        while j + 1 < n and bal[j + 1] >= bal[j]:
            j += 1
        nxt = j + 1
        while nxt < n and bal[nxt] < bal[j]:
            nxt += 1
        if nxt >= n or ss[nxt] - ss[j] > jump or ss[nxt] >= s0 + lam:
            return float(bal[j]), s0, float(ss[j]), (ss, xf, bal)
        j = nxt


# ----------------------------------------------------------------------------
# Section 3.3: contact angle of a slug between flat plates
# ----------------------------------------------------------------------------
def interface_points(rho_o, rho_w, rows, side: str, half_window: int = 8):
    """Interface positions along x on each of `rows`, from the tanh fit of
    Eq. (den-fitting) to the oil fraction rho^o / (rho^o + rho^w).  `side` is
    "left" or "right": the left or right end of the slug (oil in the middle
    of a periodic row)."""
    from scipy.optimize import curve_fit

    def tanh_profile(x, c1, c2, c3, c4):
        return c1 * np.tanh(c2 * (x - c3)) + c4

    pts = []
    for y in rows:
        phi = rho_o[y] / (rho_o[y] + rho_w[y])
        nx = phi.shape[0]
        oil = np.nonzero(phi > 0.5)[0]
        if oil.size == 0:
            continue
        edge = float(oil.min()) - 0.5 if side == "left" else float(oil.max()) + 0.5
        lo = max(int(edge) - half_window, 0)
        hi = min(int(edge) + half_window + 1, nx)
        xs = np.arange(lo, hi, dtype=np.float64)
        sl = 1.0 if side == "left" else -1.0
        p0 = (0.5 * sl, 0.5, edge, 0.5)
        popt, _ = curve_fit(tanh_profile, xs, phi[lo:hi], p0=p0, maxfev=20000)
        pts.append((float(popt[2]), float(y)))
    return np.array(pts)


def fit_circle(points):
    """Geometric least-squares circle through (x, y) points: minimises the
    sum of squared distances to the circle (scipy least_squares, started from
    the centroid).  Returns (xc, yc, R)."""
    from scipy.optimize import least_squares
    p = np.asarray(points, dtype=np.float64)
    x0 = np.array([p[:, 0].mean() + 1.0, p[:, 1].mean(), 10.0 * (np.ptp(p[:, 1]) + 1.0)])

    def res(v):
        return np.hypot(p[:, 0] - v[0], p[:, 1] - v[1]) - v[2]

    # start the centre well off the points on the side the points bow away from
    best = None
    for sgn in (1.0, -1.0):
        guess = x0.copy()
        guess[0] = p[:, 0].mean() + sgn * guess[2]
        r = least_squares(res, guess)
        if best is None or r.cost < best.cost:
            best = r
    xc, yc, rad = best.x
    return float(xc), float(yc), abs(float(rad))


def contact_angle(rho_o, rho_w, y_lo: int, y_hi: int, side: str = "right", margin: int = 3) -> float:
    """Contact angle through water (degrees) of one end of a slug between
    flat plates whose fluid rows are y_lo..y_hi (walls half a node beyond).
    Eq. (contact_angle) with y0 = half the channel width; rows within
    `margin` of a wall are left out of the fit (the wall layer)."""
    rows = list(range(y_lo + margin, y_hi - margin + 1))
    pts = interface_points(rho_o, rho_w, rows, side)
    y_axis = 0.5 * (y_lo + y_hi)
    y0 = 0.5 * (y_hi - y_lo + 1)
    xc, _, rad = fit_circle(pts)
    x_axis = float(np.interp(y_axis, pts[:, 1], pts[:, 0]))
    if rad <= y0:
        acute = 0.0
    else:
        acute = math.degrees(math.atan(math.sqrt(rad * rad - y0 * y0) / y0))
    # the oil lies left of a right end (and right of a left end)
    centre_on_oil = (xc < x_axis) if side == "right" else (xc > x_axis)
    return acute if centre_on_oil else 180.0 - acute
