"""Wettability calibration, contact angle and the planar critical force of a
slug (Sections 3.3 and 3.4 of the paper): thin callers of the library.

The measurements and the closed form live in the C ABI (include/lbm.h):
* lbm_wetting_calibrate: the Section 3.3 flat-plate slugs, one per signed
  wall potential r (r > 0: rho_s^w = r; r < 0: rho_s^o = -r), stepped
  together as one batch on the GPU, and the contact angle of each
  (lbm_contact_angle: interface points where the oil fraction crosses 1/2,
  Pratt's algebraic circle fit, Eq. contact_angle);
* lbm_wall_potentials: the potentials whose calibrated angle is theta
  (linear interpolation of r in theta, clipped to the table);
* lbm_planar_critical_balance: the planar 2-D analogue of the Section 3.4
  static balance, loaded quasi-statically from the slug's rest position.
This module only marshals arguments and keeps the table.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import lbm as _lib
from . import workloads as wl

G_INTERACTION = -1.79
# Surface tension of this model at G = -1.79, tau = 1 (Laplace law over five
# static droplets, Section 3.1; the GPU reproduces the oracle's fit to 0.5 %;
# lbm_surface_tension measures it on the GPU).
SIGMA = 0.0870
# Bulk total density of either phase at that G (1.0116 + 0.0303).
RHO_BULK = 1.042
# The calibration geometry of lbm_wetting_calibrate.
CALIB_H, CALIB_NX = 32, 192


def contact_angle(rho_o, rho_w, y_lo: int, y_hi: int, side: str = "right") -> float:
    """Contact angle through water (degrees) of one end of a slug between
    flat plates with fluid rows y_lo..y_hi (lbm_contact_angle)."""
    return _lib.lbm_contact_angle(np.stack([rho_o, rho_w]), y_lo, y_hi, side == "right")


def potentials(r: float):
    """(rho_s^o, rho_s^w) of a signed wall-potential value r."""
    return (max(-r, 0.0), max(r, 0.0))


@dataclass
class WettingTable:
    r: np.ndarray          # signed wall potentials, ascending
    theta: np.ndarray      # contact angle through water (degrees), descending
    H: int
    steps: int

    def potentials_for(self, theta_deg: float):
        """Wall potentials whose calibrated angle is theta (clipped to the
        calibrated range), lbm_wall_potentials."""
        return _lib.lbm_wall_potentials(self.r, self.theta, theta_deg)


def calibrate(lbm=None, r_values=None, H: int = CALIB_H, nx: int = CALIB_NX, steps: int = 20000,
              tau=(1.0, 1.0), precision: str = "fp32") -> WettingTable:
    """theta(r) from flat-plate slugs stepped together on the GPU
    (lbm_wetting_calibrate: plates H = 32 apart, 192 columns, tau = 1)."""
    if (H, nx, tuple(tau)) != (CALIB_H, CALIB_NX, (1.0, 1.0)):
        raise ValueError("the library calibrates on plates 32 apart, 192 columns, tau = 1")
    if r_values is None:
        r_values = np.linspace(-0.6, 0.6, 13)
    r_values = np.sort(np.asarray(r_values, dtype=np.float64))
    import torch
    stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else None
    th = _lib.lbm_wetting_calibrate(r_values, steps=steps, precision=precision, stream=stream)
    if np.any(np.diff(th) > 0.0):
        raise ValueError("calibrated contact angle is not monotone in the wall potential: %s" % th)
    return WettingTable(r_values, th, H, steps)


def critical_balance(theta_deg: float, area: float, h0: float, amp: float, lam: float, x_rest: float) -> float:
    """rho g_crit L / sigma of a slug of oil area `area` resting with its rear
    contact line near x_rest (lbm_planar_critical_balance)."""
    return _lib.lbm_planar_critical_balance(theta_deg, area, h0, amp, lam, x_rest)


def initial_fill(spec: wl.ChannelSpec):
    """(oil area, rear end) of a channel's first initial slug: the channel
    area between the slug's ends, centred on the neck at x = lambda
    floor(n_periods / (2 n_slugs))."""
    lam = float(spec.lam)
    centre = lam * (spec.n_periods // (2 * spec.n_slugs))
    half = 0.5 * spec.slug_len_over_lambda * lam
    k = 2.0 * math.pi / lam
    area = 2.0 * spec.h0 * (2.0 * half) - 2.0 * spec.amp / k * (math.sin(k * (centre + half)) -
                                                               math.sin(k * (centre - half)))
    return area, centre - half


def analytic_g_crit(spec: wl.ChannelSpec, theta_deg: float, sigma: float = SIGMA, rho: float = RHO_BULK):
    """g_crit of a sweep channel from the 2-D balance: the slug's oil area and
    rest position are taken from its initial fill; n_slugs identical slugs
    each hold the same capillary balance, so rho g L = n_slugs sigma bal."""
    area, x_rest = initial_fill(spec)
    bal = critical_balance(theta_deg, area, spec.h0, spec.amp, float(spec.lam), x_rest)
    return spec.n_slugs * (sigma * bal / (rho * spec.nx))
