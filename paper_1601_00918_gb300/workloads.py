"""Seeded synthetic inputs: wall masks, initial densities and instance specs.

This module holds no part of the lattice-Boltzmann arithmetic.  It builds the
inputs that both the CUDA path and the CPU oracle consume, so that the two
start from identical arrays:

* masks (uint8 [ny, nx], 1 = solid) for the fully periodic box, the straight
  channel and the sinusoidal channel of Section 3.4 (planar 2-D version:
  a node (x, y) is fluid iff |y - y_c| <= h(x) with
  h(x) = h0 - A cos(2 pi x / lambda), x at integer node positions);
* initial densities (float64 [2, ny, nx], species o then w): a centred droplet
  with a tanh interface (Section 3.1), the layered channel of the
  two-component Hagen-Poiseuille case (Section 3.2), and an oil slug spanning
  a constriction (Section 3.4);
* the random instance specs of the batched critical-pressure sweep.

Interface profiles use rho = rho_lo + (rho_hi - rho_lo) * s with s a tanh step
of width 2, i.e. s = (1 - tanh((r - R)/2))/2 for a droplet.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

RHO_HI = 1.0     # majority density of a bulk phase
RHO_LO = 0.03    # minority density dissolved in the other phase


# ----------------------------------------------------------------------------
# masks
# ----------------------------------------------------------------------------
def periodic_box(nx: int, ny: int) -> np.ndarray:
    """All-fluid mask, periodic in both directions."""
    return np.zeros((ny, nx), dtype=np.uint8)


def straight_channel(nx: int, width: int) -> np.ndarray:
    """Channel of `width` fluid rows between one solid row at y = 0 and one at
    y = width + 1; periodic in x.  Shape [width + 2, nx]."""
    m = np.zeros((width + 2, nx), dtype=np.uint8)
    m[0, :] = 1
    m[-1, :] = 1
    return m


def sinusoidal_half_width(x, h0: float, amp: float, lam: float):
    """h(x) = h0 - A cos(2 pi x / lambda): necks (h0 - A) at x = k lambda."""
    return h0 - amp * np.cos(2.0 * np.pi * np.asarray(x, dtype=np.float64) / lam)


def sinusoidal_channel(nx: int, ny: int, h0: float, amp: float, lam: float,
                       yc: float | None = None) -> np.ndarray:
    """Planar sinusoidal channel: fluid iff |y - y_c| <= h(x).  y_c defaults to
    the centre line (ny - 1)/2.  Rows 0 and ny - 1 are forced solid so the
    channel is closed in y; periodic in x (nx should be a multiple of lam)."""
    if yc is None:
        yc = (ny - 1) / 2.0
    x = np.arange(nx)
    y = np.arange(ny)[:, None]
    h = sinusoidal_half_width(x, h0, amp, lam)[None, :]
    m = (np.abs(y - yc) > h).astype(np.uint8)
    m[0, :] = 1
    m[-1, :] = 1
    return m


def sinusoidal_tube(nx: int, n_cross: int, h0: float, amp: float, lam: float) -> np.ndarray:
    """Mask [n_cross, n_cross, nx] (z, y, x) of the paper's 3-D geometry: a
    periodic tube of circular cross sections (Section 3.4) whose radius is
    h(x) = h0 - A cos(2 pi x / lam) about the centre line (y, z) =
    ((n_cross - 1) / 2, (n_cross - 1) / 2); fluid iff (y - y_c)^2 +
    (z - z_c)^2 <= h(x)^2; the boundary planes in y and z are solid."""
    c = (n_cross - 1) / 2.0
    x = np.arange(nx)[None, None, :]
    y = np.arange(n_cross)[None, :, None]
    z = np.arange(n_cross)[:, None, None]
    h = h0 - amp * np.cos(2.0 * np.pi * x / lam)
    m = ((y - c) ** 2 + (z - c) ** 2 > h * h).astype(np.uint8)
    m[0], m[-1], m[:, 0], m[:, -1] = 1, 1, 1, 1
    return m


def tube_slug(nx: int, n_cross: int, x_rear: float, x_front: float, rho_hi: float = RHO_HI,
              rho_lo: float = RHO_LO) -> np.ndarray:
    """Densities [2, n_cross, n_cross, nx] of an oil slug filling the tube
    between x_rear and x_front (tanh ends of width 2), water elsewhere."""
    x = np.arange(nx)[None, None, :] + np.zeros((n_cross, n_cross, 1))
    s = _step(x - x_rear) - _step(x - x_front)
    ro = rho_lo + (rho_hi - rho_lo) * s
    return np.stack([ro, rho_hi + rho_lo - ro])


# ----------------------------------------------------------------------------
# initial densities
# ----------------------------------------------------------------------------
def _step(d):
    """Smooth 0 -> 1 step of width 2: (1 + tanh(d/2))/2."""
    return 0.5 * (1.0 + np.tanh(np.asarray(d, dtype=np.float64) / 2.0))


def droplet(nx: int, ny: int, radius: float, cx: float | None = None, cy: float | None = None,
            rho_hi: float = RHO_HI, rho_lo: float = RHO_LO) -> np.ndarray:
    """Droplet of species o (density rho_hi inside) centred at (cx, cy) in
    species w; rho^w = rho_hi + rho_lo - rho^o."""
    cx = nx / 2.0 if cx is None else cx
    cy = ny / 2.0 if cy is None else cy
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    s = _step(radius - r)            # 1 inside, 0 outside
    ro = rho_lo + (rho_hi - rho_lo) * s
    return np.stack([ro, rho_hi + rho_lo - ro])


def flat_interface(nx: int, ny: int, rho_hi: float = RHO_HI, rho_lo: float = RHO_LO) -> np.ndarray:
    """Species o in the band nx/4 <= x < 3nx/4, species w elsewhere (two flat
    interfaces, periodic)."""
    x = np.arange(nx)[None, :] + np.zeros((ny, 1))
    s = _step(x - nx / 4.0) - _step(x - 3.0 * nx / 4.0)
    ro = rho_lo + (rho_hi - rho_lo) * s
    return np.stack([ro, rho_hi + rho_lo - ro])


def layered_channel(nx: int, width: int, outer: int, core_species: int = 0,
                    rho_hi: float = RHO_HI, rho_lo: float = RHO_LO) -> np.ndarray:
    """Layered fill of straight_channel(nx, width): `outer` rows next to each
    wall hold the wetting species (1 - core_species), the core holds
    core_species.  Sharp initial interface."""
    ny = width + 2
    y = np.arange(ny)
    core = (y >= 1 + outer) & (y <= width - outer)
    s = np.where(core, 1.0, 0.0)[:, None] + np.zeros((1, nx))
    r_core = rho_lo + (rho_hi - rho_lo) * s
    r_other = rho_hi + rho_lo - r_core
    out = np.empty((2, ny, nx))
    out[core_species] = r_core
    out[1 - core_species] = r_other
    return out


def slug(nx: int, ny: int, x_rear: float, x_front: float, rho_hi: float = RHO_HI,
         rho_lo: float = RHO_LO) -> np.ndarray:
    """Oil slug (species o) occupying x_rear < x < x_front across the channel,
    water (species w) elsewhere; tanh interfaces of width 2."""
    x = np.arange(nx)[None, :] + np.zeros((ny, 1))
    s = _step(x - x_rear) - _step(x - x_front)
    ro = rho_lo + (rho_hi - rho_lo) * s
    return np.stack([ro, rho_hi + rho_lo - ro])


def uniform(nx: int, ny: int, rho_o: float, rho_w: float) -> np.ndarray:
    out = np.empty((2, ny, nx))
    out[0] = rho_o
    out[1] = rho_w
    return out


def random_perturbed(nx: int, ny: int, seed: int, rho_o: float = 0.6, rho_w: float = 0.4,
                     amp: float = 0.05) -> np.ndarray:
    """Uniform mixture with seeded uniform noise of relative size amp."""
    rng = np.random.default_rng(seed)
    out = uniform(nx, ny, rho_o, rho_w)
    out *= 1.0 + amp * (2.0 * rng.random((2, ny, nx)) - 1.0)
    return out


@dataclass
class BypassSpec:
    """Two channels with joined ends (the paper's outlook on bypass
    channels): in the branch section an upper branch of one sinusoidal
    wavelength (bulge - neck - bulge, mean half-width 0.1875 lam, amplitude
    amp_ratio of it) followed by a straight part `ext` long at the bulge
    width, holds the oil slug at its neck; a straight lower branch `hl` rows
    wide runs beside it, separated by an island `island` rows thick.  Two
    full-height chambers `chamber` long join both branches to a straight pipe
    `wm` rows wide and `lm` long, which closes the periodic loop (the
    chambers are wide enough that their own resistance, the flow turning
    from the pipe into the lower branch, is a few per cent of the
    branches').  With blocked = True the lower branch is solid, so all flow
    must pass the slug."""
    lam: int = 128
    amp_ratio: float = 0.5
    slug_len_over_lambda: float = 0.6
    hl: int = 12
    island: int = 4
    ext: int = 96
    chamber: int = 32
    wm: int = 12
    lm: int = 224
    blocked: bool = False

    @property
    def h0(self) -> float:
        return 0.1875 * self.lam

    @property
    def amp(self) -> float:
        return self.amp_ratio * self.h0

    @property
    def branch_len(self) -> int:
        return self.lam + self.ext

    @property
    def nx(self) -> int:
        return self.lm + 2 * self.chamber + self.branch_len

    @property
    def upper_height(self) -> int:
        return 2 * int(math.ceil(self.h0 + self.amp))

    @property
    def ny(self) -> int:
        return self.hl + self.island + self.upper_height + 2

    @property
    def x_neck(self) -> float:
        """Column of the upper branch's neck (the slug's centre)."""
        return float(self.lm + self.chamber + self.lam // 2)


def bypass_channel(spec: BypassSpec) -> Workload:
    """Mask and slug fill of a bypass geometry (BypassSpec); periodic in x,
    solid rows 0 and ny - 1.  Row ranges (fluid): lower branch 1 .. hl,
    island hl + 1 .. hl + island (solid in the branch section), upper branch
    above it; the pipe's wm rows are centred in the channel; chambers are
    fluid over the full height.  The slug spans slug_len_over_lambda * lam
    columns about the neck and only the upper branch's rows."""
    nx, ny = spec.nx, spec.ny
    mask = np.ones((ny, nx), dtype=np.uint8)
    x = np.arange(nx)
    y = np.arange(ny)[:, None]
    x_pipe_end = spec.lm
    xb0 = spec.lm + spec.chamber                      # branch section [xb0, xb1)
    xb1 = xb0 + spec.branch_len
    # pipe
    yp0 = 1 + (ny - 2 - spec.wm) // 2
    mask[yp0:yp0 + spec.wm, :x_pipe_end] = 0
    # chambers
    mask[1:ny - 1, x_pipe_end:xb0] = 0
    mask[1:ny - 1, xb1:nx] = 0
    # lower branch
    if not spec.blocked:
        mask[1:1 + spec.hl, xb0:xb1] = 0
    # upper branch: one sinusoidal wavelength from xb0 (bulge), then straight at the bulge width
    yu0 = 1 + spec.hl + spec.island                   # first row of the upper branch
    yc = yu0 + 0.5 * (spec.upper_height - 1)
    xs = x[xb0:xb1] - xb0
    h = np.where(xs < spec.lam, spec.h0 + spec.amp * np.cos(2.0 * np.pi * xs / spec.lam), spec.h0 + spec.amp)
    fluid_u = (np.abs(y - yc) <= h[None, :]) & (y >= yu0) & (y <= ny - 2)
    sub = mask[:, xb0:xb1]
    sub[fluid_u] = 0
    # slug: oil over the neck's columns, upper-branch rows only
    half = 0.5 * spec.slug_len_over_lambda * spec.lam
    xx = x[None, :] + np.zeros((ny, 1))
    s = (_step(xx - (spec.x_neck - half)) - _step(xx - (spec.x_neck + half))) * (y >= yu0)
    ro = RHO_LO + (RHO_HI - RHO_LO) * s
    rho = np.stack([ro, RHO_HI + RHO_LO - ro])
    name = f"bypass_{nx}x{ny}" + ("_blocked" if spec.blocked else "")
    return Workload(name, mask, rho, (True, False))


def bypass_resistance_ratio(spec: BypassSpec) -> float:
    """(R_lower + R_pipe) / R_lower for plane Poiseuille flow (resistance
    12 mu length / width^3 per unit depth, walls halfway between the last
    fluid and the first solid row, the chambers' resistance neglected).  With
    the body force on every node and the slug blocking the upper branch, the
    loop's flow Q satisfies rho g L = (R_lower + R_pipe) Q, and the slug holds
    the lower branch's viscous drop R_lower Q = rho g L R_lower / (R_lower +
    R_pipe): its critical force is the blocked one times this ratio."""
    r_lower = spec.branch_len / spec.hl ** 3
    r_pipe = spec.lm / spec.wm ** 3
    return (r_lower + r_pipe) / r_lower


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    mask: np.ndarray
    rho: np.ndarray
    periodic: tuple


def droplet_box(radius: float = 20.0, n: int = 128) -> Workload:
    """Static droplet in an n x n periodic box (Section 3.1 set-up)."""
    return Workload(f"droplet_{n}x{n}_R{radius:g}", periodic_box(n, n),
                    droplet(n, n, radius, cx=n / 2.0, cy=n / 2.0), (True, True))


def sinusoidal_slug(scale: int = 1) -> Workload:
    """Sinusoidal channel with an oil slug centred on a neck.

    scale = 1: 1024 x 146 nodes, h(x) = 48 - 24 cos(2 pi x / 256), y_c = 72.5,
    slug 320 nodes long centred on the neck at x = 512.
    scale = 8: 8192 x 1170 nodes, h(x) = 384 - 192 cos(2 pi x / 2048),
    y_c = 584.5, slug 2560 long centred on x = 4096."""
    nx, ny = 1024 * scale, (146 if scale == 1 else 146 * scale + 2)
    lam = 256.0 * scale
    h0, amp = 48.0 * scale, 24.0 * scale
    yc = (ny - 1) / 2.0
    mask = sinusoidal_channel(nx, ny, h0, amp, lam, yc)
    centre, half = 2.0 * lam, 160.0 * scale
    rho = slug(nx, ny, centre - half, centre + half)
    return Workload(f"sinusoidal_slug_{nx}x{ny}", mask, rho, (True, False))


# ----------------------------------------------------------------------------
# batched-sweep instance specs
# ----------------------------------------------------------------------------
@dataclass
class ChannelSpec:
    lam: int                 # wavelength in nodes
    amp_ratio: float         # A / h0
    slug_len_over_lambda: float
    theta_deg: float         # contact angle through the water phase
    visc_ratio: float        # nu^o / nu^w
    n_periods: int = 4
    n_slugs: int = 1         # identical slugs on equally spaced necks

    @property
    def h0(self) -> float:
        return 0.1875 * self.lam

    @property
    def amp(self) -> float:
        return self.amp_ratio * self.h0

    @property
    def nx(self) -> int:
        return self.lam * self.n_periods

    @property
    def ny(self) -> int:
        return 2 * int(math.ceil(self.h0 + self.amp)) + 2


def sweep_specs(n: int, seed: int, lambdas=(128, 192, 256, 384, 512)) -> list:
    """n random channel instances: lambda uniform over `lambdas`, A/h0 ~
    U[0.2, 0.6], slug length / lambda ~ U[1, 2], contact angle ~ U[20, 160]
    degrees, viscosity ratio log-uniform on [0.2, 10]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        out.append(ChannelSpec(
            lam=int(rng.choice(np.asarray(lambdas))),
            amp_ratio=float(rng.uniform(0.2, 0.6)),
            slug_len_over_lambda=float(rng.uniform(1.0, 2.0)),
            theta_deg=float(rng.uniform(20.0, 160.0)),
            visc_ratio=float(np.exp(rng.uniform(np.log(0.2), np.log(10.0))))))
    return out


def channel_instance(spec: ChannelSpec) -> Workload:
    """Mask and slug fill of one sweep instance: mean half-width h0 =
    0.1875 lambda, amplitude A = amp_ratio h0, n_periods periods, n_slugs
    identical slugs centred on the necks at x = lambda (n_periods /
    (2 n_slugs) + k n_periods / n_slugs) (one slug: x = lambda
    floor(n_periods / 2))."""
    nx, ny = spec.nx, spec.ny
    mask = sinusoidal_channel(nx, ny, spec.h0, spec.amp, float(spec.lam))
    k = spec.n_slugs
    spacing = float(spec.lam * (spec.n_periods // k))
    first = float(spec.lam * (spec.n_periods // (2 * k)))
    half = 0.5 * spec.slug_len_over_lambda * spec.lam
    x = np.arange(nx)[None, :] + np.zeros((ny, 1))
    s = np.zeros((ny, nx))
    for j in range(k):
        c = first + j * spacing
        s = s + (_step(x - (c - half)) - _step(x - (c + half)))
    ro = RHO_LO + (RHO_HI - RHO_LO) * s
    rho = np.stack([ro, RHO_HI + RHO_LO - ro])
    return Workload(f"channel_{nx}x{ny}", mask, rho, (True, False))
