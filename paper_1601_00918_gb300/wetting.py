"""Wettability calibration and the analytic critical force of a slug
(Sections 3.3 and 3.4 of the paper), on this library's own simulations.

* Contact angle of a slug between flat plates (Section 3.3,
  Eq. contact_angle): on every row away from the walls the interface sits
  where the oil fraction rho^o / (rho^o + rho^w) crosses 1/2 (linear
  interpolation between the two nodes around the crossing); an algebraic
  least-squares circle (x^2 + y^2 + D x + E y + F = 0) is fitted through the
  points, and theta = arctan(sqrt(R^2 - y0^2) / y0) with y0 the half channel
  width is the acute angle between wall and interface: the angle through
  water when the circle's centre is on the oil side, 180 degrees minus it
  otherwise.
* Calibration table theta(r): one flat-plate slug per wall-potential value r
  (r > 0: rho_s^w = r, the wall attracts water; r < 0: rho_s^o = -r), all
  stepped together as one batch on the GPU; theta is inverted by monotone
  interpolation (the paper's procedure for choosing the wall potentials of
  its critical-pressure runs, Section 3.3).
* 2-D critical body force (the planar analogue of the Section 3.4 balance):
  front and rear menisci are axis-centred arcs, p_o - p_w = sigma cos(theta
  -+ phi) / h at the front (-) and the rear (+), phi the wall angle; at rest
  rho g L equals sigma times the difference of the two curvatures; the
  front follows the rear by conservation of the oil area (channel between
  the contact chords plus the circular segments beyond them); loaded
  quasi-statically from its rest position the slug follows the rising
  branches of the balance and jumps ahead past each local maximum; it
  counts as moving at the first jump longer than lam / 2 (or out of the
  period), the same displacement reading the bisection decides with.  Used
  to seed the bisection bracket.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import workloads as wl

G_INTERACTION = -1.79
# Surface tension of this model at G = -1.79, tau = 1 (Laplace law over five
# static droplets, Section 3.1; the GPU reproduces the oracle's fit to 0.5 %).
SIGMA = 0.0870
# Bulk total density of either phase at that G (1.0116 + 0.0303).
RHO_BULK = 1.042


# ----------------------------------------------------------------------------
# Section 3.3: contact angle from a slug between flat plates
# ----------------------------------------------------------------------------
def half_crossings(frac_row, side: str) -> float | None:
    """Position along x where an oil fraction row crosses 1/2 at the left or
    right end of the oil (the slug is the longest run above 1/2)."""
    above = frac_row > 0.5
    if not above.any() or above.all():
        return None
    idx = np.nonzero(above)[0]
    if side == "right":
        i = int(idx.max())
        a, b = frac_row[i], frac_row[(i + 1) % frac_row.size]
        return i + (a - 0.5) / (a - b)
    i = int(idx.min())
    a, b = frac_row[i - 1], frac_row[i]
    return (i - 1) + (0.5 - a) / (b - a)


def circle_through(xs, ys):
    """Algebraic circle fit with Pratt's normalisation: the circle (or line)
    A (x^2 + y^2) + B x + C y + D = 0 minimising the sum of squared residuals
    subject to B^2 + C^2 - 4 A D = 1 (a generalised eigenproblem; it stays
    well posed as the points straighten into a line, A -> 0).  Returns
    (A, B, C, D); the radius is 1 / (2 |A|) and the centre (-B, -C) / (2 A)."""
    xs = np.asarray(xs, dtype=np.float64)
    ys = np.asarray(ys, dtype=np.float64)
    # centre the data for conditioning, undo the shift at the end
    mx, my = xs.mean(), ys.mean()
    u, v = xs - mx, ys - my
    Z = np.stack([u * u + v * v, u, v, np.ones_like(u)], axis=1)
    M = Z.T @ Z
    N = np.array([[0.0, 0.0, 0.0, -2.0], [0.0, 1.0, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0], [-2.0, 0.0, 0.0, 0.0]])
    import scipy.linalg
    w, vec = scipy.linalg.eig(M, N)
    w = np.real(w)
    ok = np.isfinite(w) & (w > -1e-9 * max(1.0, np.abs(w[np.isfinite(w)]).max()))
    k = int(np.argmin(np.where(ok, w, np.inf)))
    A, B, C, D = np.real(vec[:, k])
    norm = math.sqrt(max(B * B + C * C - 4.0 * A * D, 1e-300))
    A, B, C, D = A / norm, B / norm, C / norm, D / norm
    # back to the original coordinates: substitute u = x - mx, v = y - my
    B2 = B - 2.0 * A * mx
    C2 = C - 2.0 * A * my
    D2 = D + A * (mx * mx + my * my) - B * mx - C * my
    return A, B2, C2, D2


def contact_angle(rho_o, rho_w, y_lo: int, y_hi: int, side: str = "right", margin: int = 3) -> float:
    """Contact angle through water (degrees) of one end of a slug between
    flat plates with fluid rows y_lo..y_hi; rows within `margin` of a wall
    are left out of the fit."""
    with np.errstate(invalid="ignore", divide="ignore"):    # wall rows may hold 0 / 0; only fluid rows are read
        frac = rho_o / (rho_o + rho_w)
    ys, xs = [], []
    for y in range(y_lo + margin, y_hi - margin + 1):
        x = half_crossings(frac[y], side)
        if x is not None:
            ys.append(float(y))
            xs.append(x)
    if len(xs) < 3:
        raise ValueError("too few interface points")
    A, B, C, D = circle_through(xs, ys)
    y0 = 0.5 * (y_hi - y_lo + 1)
    # cos(acute) = y0 / R with R = 1 / (2 |A|): Eq. (contact_angle) without dividing by A
    acute = math.degrees(math.acos(min(2.0 * abs(A) * y0, 1.0)))
    if abs(A) < 1e-12:
        return 90.0
    xc = -B / (2.0 * A)
    x_axis = float(np.interp(0.5 * (y_lo + y_hi), ys, xs))
    on_oil = xc < x_axis if side == "right" else xc > x_axis
    return acute if on_oil else 180.0 - acute


def potentials(r: float):
    """(rho_s^o, rho_s^w) of a signed wall-potential value r."""
    return (max(-r, 0.0), max(r, 0.0))


def flat_plate_slug(r: float, H: int = 32, nx: int = 192, tau=(1.0, 1.0)) -> dict:
    """Batch instance of the Section 3.3 set-up: plates H apart (fluid rows
    1..H), periodic in x, oil slug over the middle half."""
    mask = wl.straight_channel(nx, H)
    rho = wl.slug(nx, H + 2, nx / 4.0, 3.0 * nx / 4.0)
    return dict(mask=mask, rho_init=rho, tau=tuple(tau), G=G_INTERACTION, rho_wall=potentials(r),
                g=(0.0, 0.0), periodic=(True, False))


@dataclass
class WettingTable:
    r: np.ndarray          # signed wall potentials, ascending
    theta: np.ndarray      # contact angle through water (degrees), descending
    H: int
    steps: int

    def potentials_for(self, theta_deg: float):
        """Wall potentials whose calibrated angle is theta (clipped to the
        calibrated range)."""
        th = float(np.clip(theta_deg, self.theta.min(), self.theta.max()))
        r = float(np.interp(th, self.theta[::-1], self.r[::-1]))
        return potentials(r)


def calibrate(lbm, r_values=None, H: int = 32, nx: int = 192, steps: int = 20000, tau=(1.0, 1.0),
              precision: str = "fp32") -> WettingTable:
    """theta(r) from flat-plate slugs stepped together on the GPU."""
    if r_values is None:
        r_values = np.linspace(-0.6, 0.6, 13)
    r_values = np.sort(np.asarray(r_values, dtype=np.float64))
    insts = [flat_plate_slug(float(r), H, nx, tau) for r in r_values]
    b = lbm.Batch(insts, precision=precision)
    try:
        b.step(steps)
        b.observables(check=True)
        thetas = []
        for i in range(len(insts)):
            f = b.save(i)
            rho = f.sum(axis=1)
            a = contact_angle(rho[0], rho[1], 1, H, "right")
            c = contact_angle(rho[0], rho[1], 1, H, "left")
            thetas.append(0.5 * (a + c))
    finally:
        b.close()
    th = np.array(thetas)
    if np.any(np.diff(th) > 0.0):
        raise ValueError("calibrated contact angle is not monotone in the wall potential: %s" % th)
    return WettingTable(r_values, th, H, steps)


# ----------------------------------------------------------------------------
# Section 3.4: 2-D critical force of a slug in a sinusoidal channel
# ----------------------------------------------------------------------------
def _menisci(theta, x, h0, amp, lam, front):
    k = 2.0 * math.pi / lam
    h = h0 - amp * np.cos(k * x)
    phi = np.arctan(amp * k * np.sin(k * x))
    alpha = 0.5 * math.pi + (phi if front else -phi) - theta
    kappa = np.sin(alpha) / h
    a = np.maximum(np.abs(alpha), 1e-9)
    seg = np.sign(alpha) * (h / np.sin(a)) ** 2 * (a - np.sin(a) * np.cos(a))
    return kappa, seg


def _area(xr, xf, theta, h0, amp, lam):
    k = 2.0 * math.pi / lam
    inner = 2.0 * h0 * (xf - xr) - 2.0 * amp / k * (np.sin(k * xf) - np.sin(k * xr))
    return inner + _menisci(theta, xf, h0, amp, lam, True)[1] + _menisci(theta, xr, h0, amp, lam, False)[1]


def critical_balance(theta_deg: float, area: float, h0: float, amp: float, lam: float, x_rest: float,
                     n: int = 2001):
    """(kappa_front - kappa_rear) at which the slug starts to move, i.e.
    rho g_crit L / sigma, loaded from the rest position nearest x_rest (rear
    contact chord).  The front position of every sampled rear position
    comes from a vectorised bisection on the oil area; the loading path is
    followed over the sampled balance."""
    th = math.radians(theta_deg)
    s = x_rest + np.linspace(-0.5 * lam, 1.5 * lam, n)
    lo = s + 1e-6
    hi = s + area / (2.0 * max(h0 - amp, 1e-9)) + 2.0 * lam
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        more = _area(s, mid, th, h0, amp, lam) > area
        hi = np.where(more, mid, hi)
        lo = np.where(more, lo, mid)
    xf = 0.5 * (lo + hi)
    bal = _menisci(th, xf, h0, amp, lam, True)[0] - _menisci(th, s, h0, amp, lam, False)[0]
    if np.max(np.abs(bal)) < 1e-12:
        return 0.0
    ups = [i for i in range(n - 1) if bal[i] <= 0.0 < bal[i + 1] and s[i] <= x_rest + 0.5 * lam]
    if not ups:
        raise ValueError("no rest position within half a wavelength")
    i = min(ups, key=lambda k: abs(s[k] - x_rest))
    start = s[i]
    level_at, pos = _loading_path(s, bal, i + 1, start + lam, 0.5 * lam)
    return float(level_at)


def _loading_path(s, bal, j, end, jump):
    """Climb to the next local maximum; jump to the next sample whose balance
    is as large; stop at a jump longer than `jump` or past `end`."""
    n = s.size
    while True:
        peaks = np.nonzero(np.diff(bal[j:]) < 0.0)[0]
        j = j + int(peaks[0]) if peaks.size else n - 1
        ahead = np.nonzero(bal[j + 1:] >= bal[j])[0]
        if ahead.size == 0:
            return bal[j], s[j]
        k = j + 1 + int(ahead[0])
        if s[k] - s[j] > jump or s[k] >= end:
            return bal[j], s[j]
        j = k


def analytic_g_crit(spec: wl.ChannelSpec, theta_deg: float, sigma: float = SIGMA, rho: float = RHO_BULK):
    """g_crit of a sweep channel from the 2-D balance: the slug's oil area and
    rest position are taken from its initial fill (centred on a neck)."""
    lam = float(spec.lam)
    centre = 2.0 * lam
    half = 0.5 * spec.slug_len_over_lambda * lam
    k = 2.0 * math.pi / lam
    area = 2.0 * spec.h0 * (2.0 * half) - 2.0 * spec.amp / k * (math.sin(k * (centre + half)) -
                                                               math.sin(k * (centre - half)))
    bal = critical_balance(theta_deg, area, spec.h0, spec.amp, lam, centre - half)
    return sigma * bal / (rho * spec.nx)
