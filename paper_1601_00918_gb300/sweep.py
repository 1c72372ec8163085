"""Critical-body-force sweeps over many channels (Section 3.4 of the paper).

The paper finds the body force at which a static oil slug in a sinusoidal
channel starts to move.  Here every channel of a sweep is bisected on g by
``lbm_critical_pressure_batch`` (all channels in one launch per step,
decisions in FP64 on the device), optionally with brackets seeded by the
surrogate network.

Channel description (``workloads.ChannelSpec``): wavelength lambda, amplitude
ratio A/h0, slug length / lambda, contact-angle parameter theta, viscosity
ratio nu^o / nu^w; mean half-width h0 = 0.1875 lambda, n_periods periods.

Readings (not fixed by the paper):
* wettability: with a calibration table (wetting.calibrate, the Section 3.3
  flat-plate procedure run on the GPU) the wall potentials are the ones
  whose measured contact angle is theta; without one, cos(theta) is mapped
  linearly onto them, rho_s^w = max(cos theta, 0) * RHO_S_MAX (water-wet)
  and rho_s^o = max(-cos theta, 0) * RHO_S_MAX (oil-wet);
* starting bracket of the plain bisection: 0.5 to 2 times the planar 2-D
  critical force of the slug (wetting.analytic_g_crit);
* viscosity ratio r: tau^w = 1 and tau^o = 3 r nu^w + 1/2 >= 0.75; the
  instances use the regularised collision (Eq. Regualize).  In these wetted
  channels it keeps the densities positive for tau^o >= 0.75 (plain BGK
  loses positivity below ~0.82: 23 of 64 instances of the sweep below fail
  with BGK, none with the regularised collision at r >= 0.5; with r down to
  0.2, 8 fail, all with tau^o <= 0.73), so the sweep covers r in [0.5, 10];
* "moving": the oil centre of mass travels more than lambda / 2 within one
  probe window.

The paper's own protocol, a continuous ramp of g without restarts
(ramp_critical), is here too; the bisection replaces it in the sweeps
because it needs far fewer steps per solve.

Surrogate features (all O(1)): amplitude ratio, slug length / lambda,
cos(theta), log(viscosity ratio), 1 / resolution with the resolution the
neck width 2 (h0 - A) in nodes.  Target: log g_crit, g_crit the geometric
mean of the final bracket.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import workloads as wl

G_INTERACTION = -1.79
RHO_S_MAX = 0.5
TAU_MIN = 0.75
COLLISION = "regularized"


def relaxation_times(visc_ratio: float):
    nu_w = (1.0 - 0.5) / 3.0
    tau_o = 3.0 * visc_ratio * nu_w + 0.5
    return (max(tau_o, TAU_MIN), 1.0)


def wall_potentials(theta_deg: float):
    c = math.cos(math.radians(theta_deg))
    return (max(-c, 0.0) * RHO_S_MAX, max(c, 0.0) * RHO_S_MAX)


def instance_of(spec: wl.ChannelSpec, table=None) -> dict:
    """Batch instance of a channel spec (channel and slug from the library,
    lbm_channel_geometry); `table` (wetting.WettingTable) gives calibrated
    wall potentials."""
    from . import lbm as _lib
    mask, rho = _lib.lbm_channel_geometry(spec)
    rw = table.potentials_for(spec.theta_deg) if table is not None else wall_potentials(spec.theta_deg)
    return dict(mask=mask, rho_init=rho, tau=relaxation_times(spec.visc_ratio), G=G_INTERACTION,
                rho_wall=rw, g=(0.0, 0.0), periodic=(True, False), disp_threshold=0.5 * spec.lam,
                collision=COLLISION)


def analytic_brackets(specs, lo: float = 0.5, hi: float = 2.0):
    """(lo, hi) times the planar 2-D critical force of each slug."""
    from . import wetting
    g = np.array([wetting.analytic_g_crit(s, s.theta_deg) for s in specs])
    return lo * g, hi * g


def features(spec: wl.ChannelSpec) -> np.ndarray:
    neck = 2.0 * (spec.h0 - spec.amp)
    return np.array([spec.amp_ratio, spec.slug_len_over_lambda, math.cos(math.radians(spec.theta_deg)),
                     math.log(spec.visc_ratio), 1.0 / neck], dtype=np.float64)


def small_specs(n: int, seed: int, lambdas=(32, 48, 64)) -> list:
    """Sweep instances scaled to a budget: lambda in `lambdas`, 4 periods,
    A/h0 ~ U[0.2, 0.6], slug/lambda ~ U[1, 2], theta ~ U[20, 160] deg,
    viscosity ratio log-U[0.5, 10]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        out.append(wl.ChannelSpec(
            lam=int(rng.choice(np.asarray(lambdas))),
            amp_ratio=float(rng.uniform(0.2, 0.6)),
            slug_len_over_lambda=float(rng.uniform(1.0, 2.0)),
            theta_deg=float(rng.uniform(20.0, 160.0)),
            visc_ratio=float(np.exp(rng.uniform(np.log(0.5), np.log(10.0))))))
    return out


def run_sweep(lbm, specs, g_lo, g_hi, precision="fp32", rel_bracket=0.02, t_eq=1000, t_obs=2000,
              max_probes=24, check_bracket=True, timeout_s=0.0, table=None):
    """Batched bisection of every spec; returns (results, seconds)."""
    insts = [instance_of(s, table) for s in specs]
    t0 = time.perf_counter()
    b = lbm.Batch(insts, precision=precision)
    try:
        res = b.critical_pressure(np.broadcast_to(np.asarray(g_lo, dtype=np.float64), (len(specs),)).copy(),
                                  np.broadcast_to(np.asarray(g_hi, dtype=np.float64), (len(specs),)).copy(),
                                  rel_bracket=rel_bracket, t_eq=t_eq, t_obs=t_obs, max_probes=max_probes,
                                  check_bracket=check_bracket, timeout_s=timeout_s, check=False)
    finally:
        b.close()
    return res, time.perf_counter() - t0


def run_sweep_sharded(lbm, specs, g_lo, g_hi, **kw):
    """The sweep split across ranks (one GPU each, round-robin shares, no
    collective while stepping); results gathered back in order on every rank."""
    from . import dist as D
    world, rank, _ = D.env()
    lo = np.broadcast_to(np.asarray(g_lo, dtype=np.float64), (len(specs),))
    hi = np.broadcast_to(np.asarray(g_hi, dtype=np.float64), (len(specs),))
    mine = D.shard(range(len(specs)), rank, world)
    res, dt = run_sweep(lbm, [specs[k] for k in mine], lo[mine], hi[mine], **kw) if mine else ([], 0.0)
    return D.gather(res, len(specs)), D.max_over_ranks(dt)


def ramp_critical(lbm, specs, g_start, ratio: float = 1.05, n_levels: int = 40, t_eq: int = 2000,
                  t_level: int = 8000, precision: str = "fp32", table=None):
    """The paper's own protocol (Section 3.4): after t_eq steps at g = 0, g
    is raised level by level without restarting (level k of instance i is
    g_start[i] ratio^k, t_level steps each), and a slug counts as moving at
    the first level in which its oil centre of mass travels more than
    lambda / 2.  Unlike the bisection, the slug carries its displacement
    from level to level, as in the paper's ramp.  All instances step
    together as one batch.  Returns (list of (g_static, g_moving) with the
    last static and the first moving level, None where no level moved the
    slug; seconds)."""
    insts = [instance_of(s, table) for s in specs]
    n = len(specs)
    g0 = np.broadcast_to(np.asarray(g_start, dtype=np.float64), (n,)).copy()
    thr = np.array([0.5 * s.lam for s in specs])
    t0 = time.perf_counter()
    b = lbm.Batch(insts, precision=precision)
    out = [None] * n
    try:
        b.step(t_eq)
        prev = np.array([o["oil_disp_x"] for o in b.observables(check=False)])
        for k in range(n_levels):
            g = g0 * ratio ** k
            b.set_body_force(g)
            b.step(t_level)
            disp = np.array([o["oil_disp_x"] for o in b.observables(check=False)])
            for i in range(n):
                if out[i] is None and abs(disp[i] - prev[i]) > thr[i]:
                    out[i] = (g[i] / ratio if k > 0 else 0.0, g[i])
            prev = disp
            if all(o is not None for o in out):
                break
    finally:
        b.close()
    return out, time.perf_counter() - t0


def run_channels(lbm, specs, precision="fp32", rel_bracket=0.02, t_eq=1000, t_obs=2000, max_probes=24,
                 timeout_s=0.0, table=None, surrogate=None, scale_x=None, k_sigma=2.0, sigma=None, rho=None):
    """The whole question inside the library (lbm_critical_pressure_channels):
    channel and slug, wall potentials from `table` (or the library's own
    calibration), relaxation times, starting bracket from the planar
    balance or from `surrogate` (with its feature scaling scale_x = (mean,
    std)), the batched bisection and the Bond numbers; returns (results,
    seconds)."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    kw = {}
    if surrogate is not None:
        kw = dict(surrogate=surrogate, feature_mean=scale_x[0], feature_std=scale_x[1], k_sigma=k_sigma)
    t0 = time.perf_counter()
    res = lbm.lbm_critical_pressure_channels(
        specs, precision=precision, collision=COLLISION, rel_bracket=rel_bracket, t_eq=t_eq, t_obs=t_obs,
        max_probes=max_probes, table=table, sigma=sigma or 0.0, rho_bulk=rho or 0.0, timeout_s=timeout_s,
        stream=stream, **kw)
    return res, time.perf_counter() - t0


def run_plain(lbm, specs, g_lo, g_hi, **kw):
    """The same bisection one instance at a time (the baseline)."""
    res, total = [], 0.0
    for k, s in enumerate(specs):
        lo = np.atleast_1d(g_lo)[k if np.ndim(g_lo) else 0]
        hi = np.atleast_1d(g_hi)[k if np.ndim(g_hi) else 0]
        r, dt = run_sweep(lbm, [s], lo, hi, **kw)
        res += r
        total += dt
    return res, total


def surrogate_brackets(net, specs, scale_x, k_sigma=2.0, floor=1.05):
    """exp(mu -+ k sigma) from the surrogate; the bracket is at least a
    factor `floor` wide."""
    x = np.stack([features(s) for s in specs])
    xs = ((x - scale_x[0]) / scale_x[1]).astype(np.float32)
    out = net.forward(xs).astype(np.float64)
    mu, s = out[:, 0], out[:, 1]
    half = np.maximum(k_sigma * np.exp(0.5 * s), 0.5 * math.log(floor))
    return np.exp(mu - half), np.exp(mu + half)
