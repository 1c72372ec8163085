"""Closed forms and fits of Section 3 of the paper (FP64, numpy/scipy).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* tanh interface fit, Eq. (den-fitting): rho(x) = C1 tanh(C2 (x - C3)) + C4;
* droplet radius from the central row and column, pressure jump between the
  centre and a far point, and the Laplace law dP = sigma / R,
  Eq. (Young-Laplace_equation), fitted over several radii (Section 3.1);
* the layered two-component Hagen-Poiseuille profile (Section 3.2);
* the Bond number Bo = rho g L D / sigma, Eq. (Bo_number), and the hydrostatic
  term rho g x of Eq. (plot_value) (Section 3.4);
* the kinematic viscosity of a BGK fluid, nu = T0 (tau - 1/2) (Section 2),
  against which the shear-wave pins measure the decay rate nu k^2.
"""
from __future__ import annotations

import numpy as np

T0 = 1.0 / 3.0


# ----------------------------------------------------------------------------
# Section 3.1: interface fit and Laplace law
# ----------------------------------------------------------------------------
def tanh_profile(x, c1, c2, c3, c4):
    """Eq. (den-fitting)."""
    return c1 * np.tanh(c2 * (x - c3)) + c4


def fit_interface(xs, rho, guess_pos):
    """Least-squares fit of Eq. (den-fitting) to one interface; returns
    (C1, C2, C3, C4), C3 being the interface position."""
    from scipy.optimize import curve_fit
    xs = np.asarray(xs, dtype=np.float64)
    rho = np.asarray(rho, dtype=np.float64)
    lo, hi = float(rho.min()), float(rho.max())
    slope = 1.0 if rho[-1] > rho[0] else -1.0
    p0 = (slope * 0.5 * (hi - lo), 0.5, float(guess_pos), 0.5 * (hi + lo))
    popt, _ = curve_fit(tanh_profile, xs, rho, p0=p0, maxfev=20000)
    return tuple(float(v) for v in popt)


def droplet_radius(rho_o, cx: float, cy: float, half_window: int = 10):
    """Radius of a droplet of species o centred near (cx, cy): tanh fits of
    rho^o along the central row and the central column, one per interface,
    radius = half the distance between the two fitted positions, averaged
    over the row and the column (Section 3.1)."""
    ny, nx = rho_o.shape
    radii = []
    for line, centre in ((rho_o[int(round(cy)), :], cx), (rho_o[:, int(round(cx))], cy)):
        n = line.shape[0]
        inside = line > 0.5 * (line.max() + line.min())
        idx = np.nonzero(inside)[0]
        left_guess, right_guess = float(idx.min()) - 0.5, float(idx.max()) + 0.5
        pos = []
        for g in (left_guess, right_guess):
            lo = max(int(g) - half_window, 0)
            hi = min(int(g) + half_window + 1, n)
            xs = np.arange(lo, hi)
            pos.append(fit_interface(xs, line[lo:hi], g)[2])
        radii.append(0.5 * (pos[1] - pos[0]))
    return float(np.mean(radii))


def laplace_fit(radii, dps):
    """Least squares dP = sigma / R + c over several droplets; returns
    (sigma, c, r2) with r2 the coefficient of determination."""
    inv_r = 1.0 / np.asarray(radii, dtype=np.float64)
    dps = np.asarray(dps, dtype=np.float64)
    A = np.stack([inv_r, np.ones_like(inv_r)], axis=1)
    (sigma, c), *_ = np.linalg.lstsq(A, dps, rcond=None)
    pred = A @ np.array([sigma, c])
    ss_res = float(np.sum((dps - pred) ** 2))
    ss_tot = float(np.sum((dps - dps.mean()) ** 2))
    return float(sigma), float(c), 1.0 - ss_res / ss_tot if ss_tot > 0 else 1.0


# ----------------------------------------------------------------------------
# Section 3.2: two-component Hagen-Poiseuille between plates
# ----------------------------------------------------------------------------
def layered_poiseuille(y, a: float, b: float, f: float, mu_out: float, mu_core: float):
    """Steady velocity of a core fluid |y| < b surrounded by a wall layer
    b < |y| < a, driven by a uniform force density f, no slip at |y| = a,
    continuous velocity and shear stress at |y| = b:
        u_out(y)  = f (a^2 - y^2) / (2 mu_out)
        u_core(y) = f (b^2 - y^2) / (2 mu_core) + f (a^2 - b^2) / (2 mu_out)."""
    y = np.asarray(y, dtype=np.float64)
    out = f * (a * a - y * y) / (2.0 * mu_out)
    core = f * (b * b - y * y) / (2.0 * mu_core) + f * (a * a - b * b) / (2.0 * mu_out)
    return np.where(np.abs(y) < b, core, out)


def bgk_viscosity(tau: float) -> float:
    """Kinematic viscosity of a BGK fluid, nu = T0 (tau - 1/2) (Section 2)."""
    return T0 * (tau - 0.5)


# ----------------------------------------------------------------------------
# Section 3.4: Bond number and hydrostatic pressure
# ----------------------------------------------------------------------------
def bond_number(rho: float, g: float, length: float, d: float, sigma: float) -> float:
    """Eq. (Bo_number): Bo = rho g L D / sigma."""
    return rho * g * length * d / sigma


def hydrostatic(rho: float, g: float, x: float) -> float:
    """The rho g x term removed in Eq. (plot_value)."""
    return rho * g * x
