"""FP32 emulation of the two-component step on a periodic box (numpy).

TEST INFRASTRUCTURE ONLY: tests/test_precision_emulation.py uses it to show where
the error of an FP32 evaluation of the step against the FP64 oracle comes
from.  It shares no code with the CUDA library or with the oracle; it is a
third, vectorised statement of the same step (Section 2 of the paper:
Eqs. basic_LBM_eq, LBM_BGK at tau = 1, feq, comp_interaction,
collision_term), written so that the precision of each stage can be chosen:

* "store":   the stored populations f* (float32 or float64);
* "density": rho^a = sum_i f_i, either summed in the working precision or
             exactly (the float32 pulls summed in float64), the exact sum
             kept for the composition ("exact") or rounded once to the
             working precision everywhere ("exact_rounded");
* "dev":     the deviation of Eq. (feq) from its rest value,
             dev_i = 3 (c.v) + 4.5 (c.v)^2 - 1.5 v^2 + 4.5 (c.v)^3
                     - 4.5 (c.v) v^2  (T0 = 1/3: every constant exact in
             binary), or the same written with divisions by a rounded T0;
* "compose": f*_i = w_i rho + w_i rho dev_i, either in the working
             precision or with w_i rho exact and the sum rounded once;
* the weights: correctly rounded, or with 1/36 one unit lower so that the
             nine float32 weights add up to exactly 1.

Only tau = 1 is emulated (f* is then the equilibrium at the force-shifted
velocity: the non-equilibrium part drops out), on fully periodic boxes: the
static droplet that the FP32 contract is stated on.
"""
from __future__ import annotations

import numpy as np

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
W = np.array([4 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 9, 1 / 36, 1 / 36, 1 / 36, 1 / 36])


def initial_state(rho_init, dtype):
    """f*_i = w_i rho_init (the rest equilibrium), [2, 9, ny, nx]."""
    return (W[None, :, None, None] * np.asarray(rho_init, dtype=np.float64)[:, None]).astype(dtype)


def _shift(a, dx, dy):
    """a(x + dx, y + dy) on a periodic box (a is [..., ny, nx])."""
    return np.roll(a, (-dy, -dx), axis=(-2, -1))


def weights(work, kind="nearest"):
    """The nine weights in precision `work`: each correctly rounded
    ("nearest"), or with 1/36 one unit in the last place lower
    ("sum_to_one": in float32 the nine then add up to exactly 1)."""
    w = W.astype(work)
    if kind == "sum_to_one":
        w[5:] = np.nextafter(w[5:], work(0))
    return w


OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])


def collide(fl, G, g=(0.0, 0.0), work=np.float32, density="work", dev="exact_constants",
            compose="work", weight_kind="nearest", tau=(1.0, 1.0), rho_wall=(0.0, 0.0), mask=None,
            regularized=False, rest="equilibrium"):
    """The collision from the pulled populations fl [2, 9, ny, nx] (already in
    precision `work`), mask [ny, nx] (1 = solid, whose densities the wall
    potentials rho_wall replace in the force) or None for a fully fluid box.
    Returns (f* [2, 9, ny, nx] in the working precision, or in float64 the
    exact sums to be rounded once by the caller when compose is
    "single_rounding"; rho [2, ny, nx] in the working precision).  With compose "single_rounding" the non-equilibrium part is
    also taken against the exact w_i rho (so it carries no mass); rest
    "by_mass" sets the rest population to what the other eight leave of
    rho (f*_0 = rho - sum_{i>0} f*_i, the same value in exact arithmetic)."""
    m = work
    w = weights(m, weight_kind)
    # densities
    if density in ("exact", "exact_rounded"):
        rho64 = fl.astype(np.float64).sum(axis=1)
        rho = rho64.astype(m)
        if density == "exact_rounded":          # the low part dropped
            rho64 = rho.astype(np.float64)
    else:
        rho = fl[:, 0].copy()
        for i in range(1, 9):
            rho = rho + fl[:, i]
        rho64 = rho.astype(np.float64)
    # momenta (opposite directions paired) and the mixture velocity
    jx = (fl[:, 1] - fl[:, 3]) + ((fl[:, 5] - fl[:, 7]) + (fl[:, 8] - fl[:, 6]))
    jy = (fl[:, 2] - fl[:, 4]) + ((fl[:, 5] - fl[:, 7]) + (fl[:, 6] - fl[:, 8]))
    rt = rho[0] + rho[1]
    ux = (jx[0] + jx[1]) / rt
    uy = (jy[0] + jy[1]) / rt
    # mixture relaxation: nu_mix = (rho^o nu^o + rho^w nu^w) / rho, tau_mix = 3 nu_mix + 1/2
    relax = tuple(tau) != (1.0, 1.0)
    if relax:
        nu = [m((t - 0.5) / 3.0) for t in tau]
        tau_mix = m(3) * ((rho[0] * nu[0] + rho[1] * nu[1]) / rt) + m(0.5)
        keep = m(1) - m(1) / tau_mix                  # 1 - 1 / tau_mix
    cx = CX.astype(m)[:, None, None]
    cy = CY.astype(m)[:, None, None]

    def deviation(vx, vy):
        vv = vx * vx + vy * vy
        cu = cx * vx + cy * vy
        if dev == "exact_constants":
            return cu * (m(3) + cu * (m(4.5) + m(4.5) * cu)) - m(1.5) * vv * (m(1) + m(3) * cu)
        t0 = m(1.0 / 3.0)
        return (cu / t0 + cu * cu / (m(2) * t0 * t0) - vv / (m(2) * t0)
                + cu * cu * cu / (m(6) * t0 * t0 * t0) - cu * vv / (m(2) * t0 * t0))

    out = np.empty(fl.shape, dtype=np.float64 if compose == "single_rounding" else m)
    for a in range(2):
        # Eq. (comp_interaction) / rho^a: G sum_i w_i c_i rho^b(x + c_i), a
        # solid neighbour carrying the wall potential
        rb = rho[1 - a] if mask is None else np.where(mask != 0, m(rho_wall[1 - a]), rho[1 - a])
        d1 = _shift(rb, 1, 1) - _shift(rb, -1, -1)
        sx = w[1] * (_shift(rb, 1, 0) - _shift(rb, -1, 0)) + w[5] * (d1 + (_shift(rb, 1, -1) - _shift(rb, -1, 1)))
        sy = w[2] * (_shift(rb, 0, 1) - _shift(rb, 0, -1)) + w[5] * (d1 + (_shift(rb, -1, 1) - _shift(rb, 1, -1)))
        wr = w[:, None, None] * rho[a]
        exact = compose == "single_rounding"
        if exact:
            wex = W[:, None, None] * rho64[a]             # w_i rho, exact
            wl = (wex - wr.astype(np.float64)).astype(m)
        else:
            wl = m(0)
        # Eq. (collision_term): the equilibrium at the force-shifted velocity
        ds = deviation(ux + (m(G) * sx + m(g[0])), uy + (m(G) * sy + m(g[1])))
        t = wr * ds
        if relax:
            # Eq. (LBM_BGK): (1 - 1/tau_mix) f', f' = f - f^eq(rho^a, u_mix)
            fneq = ((fl[a] - wr) - wl) - wr * deviation(ux, uy)
            if regularized:
                # Eq. (Regualize): w_i Q_i : Pi / (2 T0^2), Q_i = c_i c_i - T0 I
                pxx = (cx * cx * fneq).sum(axis=0, dtype=m)
                pyy = (cy * cy * fneq).sum(axis=0, dtype=m)
                pxy = (cx * cy * fneq).sum(axis=0, dtype=m)
                third = m(1.0 / 3.0)
                fneq = w[:, None, None] * m(4.5) * ((cx * cx - third) * pxx + (cy * cy - third) * pyy
                                                   + m(2) * (cx * cy) * pxy)
            t = t + keep * fneq
        if exact:
            # (w_i rho)(1 + D_i) + (1 - 1/tau) f'_i with w_i rho exact: its low
            # part scales with the deviation too, then one rounding
            out[a] = wex + (t + wl * ds).astype(np.float64)
        else:
            out[a] = wr + t
        if rest == "by_mass":
            if exact:
                out[a, 0] = wex[0] - t[1:].sum(axis=0, dtype=m).astype(np.float64)
            else:
                out[a, 0] = rho[a] - out[a, 1:].astype(m).sum(axis=0, dtype=m)
    return out, rho


def pull(f, mask=None):
    """Streaming: f_i(x) = f*_i(x - c_i), or f*_opp(i)(x) when x - c_i is
    solid (halfway bounce-back); indices wrap."""
    out = np.empty_like(f)
    for i in range(9):
        moved = np.roll(f[:, i], (CY[i], CX[i]), axis=(-2, -1))
        if mask is None:
            out[:, i] = moved
        else:
            src_solid = np.roll(mask, (CY[i], CX[i]), axis=(0, 1)) != 0
            out[:, i] = np.where(src_solid, f[:, OPP[i]], moved)
    return out


def step(f, G, work=np.float32, mask=None, **kw):
    """One step in working precision `work` (keywords as in collide); `f`
    keeps its dtype (the storage); solid nodes hold zeros."""
    with np.errstate(invalid="ignore", divide="ignore"):     # solid nodes: 0 / 0, zeroed below
        out, _ = collide(pull(f, mask).astype(work), G, work=work, mask=mask, **kw)
    out = out.astype(f.dtype)
    if mask is not None:
        out[:, :, mask != 0] = 0
    return out


def run(rho_init, steps, G, store=np.float32, mask=None, **kw):
    """`steps` steps from the rest equilibrium of rho_init (zero at solid
    nodes of mask); returns f*."""
    f = initial_state(rho_init, store)
    if mask is not None:
        f[:, :, mask != 0] = 0
    for _ in range(steps):
        f = step(f, G, mask=mask, **kw)
    return f


# ----------------------------------------------------------------------------
# 16-bit storage of the populations, shifted by a reference equilibrium
# ----------------------------------------------------------------------------
def to16(x, fmt):
    """Round float32 values to FP16 or BF16 (nearest, ties to even); the
    result is float32 holding values of the 16-bit format."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    drop = 13 if fmt == "fp16" else 16          # mantissa bits beyond the format's
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + (((u >> drop) & 1) + (1 << (drop - 1)) - 1)) & (0xFFFFFFFF ^ ((1 << drop) - 1))
    out = u.astype(np.uint32).view(np.float32)
    if fmt == "fp16":
        # below 2^-14 FP16 is subnormal: a fixed spacing of 2^-24
        tiny = np.abs(x) < 2.0 ** -14
        out = np.where(tiny, np.round(x.astype(np.float64) * 2.0 ** 24) * 2.0 ** -24, out).astype(np.float32)
    return out


def _shifted_w(rh, shift):
    """w_i times the reference density of each stored population of a node:
    rh [2, ny, nx] is the node's own ("node") or, for direction i, that of
    the node x + c_i that will pull it ("destination")."""
    if shift == "node":
        return np.stack([W[i] * rh for i in range(9)], axis=1)
    return np.stack([W[i] * _shift(rh, CX[i], CY[i]) for i in range(9)], axis=1)


def _first_order_ref(rh, ux, uy):
    """w_i rhohat (1 + 3 c_i . uhat), [2, 9, ny, nx] float32."""
    return np.stack([W[i] * rh * (1.0 + 3.0 * (CX[i] * ux + CY[i] * uy)) for i in range(9)],
                    axis=1).astype(np.float32)


def _solid_zero(mask, *arrays):
    """Zero solid nodes (the last two axes) of each array in place."""
    if mask is not None:
        solid = mask != 0
        for a in arrays:
            a[..., solid] = 0


def _run16_first_order(rho_init, steps, G, fmt, work=np.float32, mask=None, **kw):
    """16-bit storage shifted by the storing node's first-order equilibrium,
    s_i = f*_i - w_i rhohat (1 + 3 c_i . uhat^a), with rhohat and the
    species' post-collision velocity uhat^a = j*^a / rho^a kept in 16 bits
    too (six extra planes)."""
    m = work
    f = W[None, :, None, None] * np.asarray(rho_init, dtype=np.float64)[:, None]
    rh = to16(rho_init, fmt)
    ux = np.zeros_like(rh)
    uy = np.zeros_like(rh)
    _solid_zero(mask, f, rh)
    s = to16(f - _first_order_ref(rh, ux, uy), fmt)
    for _ in range(steps):
        full = s.astype(m) + _first_order_ref(rh, ux, uy).astype(m)     # decoded at the storing node
        with np.errstate(invalid="ignore", divide="ignore"):
            out, rho = collide(pull(full, mask).astype(m), G, work=m, mask=mask, **kw)
            out = out.astype(m)
            jx = (out[:, 1] - out[:, 3]) + ((out[:, 5] - out[:, 7]) + (out[:, 8] - out[:, 6]))
            jy = (out[:, 2] - out[:, 4]) + ((out[:, 5] - out[:, 7]) + (out[:, 6] - out[:, 8]))
            ux, uy = jx / rho, jy / rho
        _solid_zero(mask, out, rho, ux, uy)
        rh, ux, uy = to16(rho, fmt), to16(ux, fmt), to16(uy, fmt)
        s = to16(out - _first_order_ref(rh, ux, uy), fmt)
    return s.astype(np.float64) + _first_order_ref(rh, ux, uy)


def run16(rho_init, steps, G, fmt="fp16", shift="node", work=np.float32, mask=None, **kw):
    """`steps` steps with the populations stored in 16 bits as
    s_i = f*_i - w_i rhohat, rhohat the 16-bit density of the storing node
    ("node"), of the node that pulls the population next ("destination",
    which knows it as its own previous density), or each species' initial
    mean ("constant"); rhohat is stored too; "first_order" also removes the
    storing node's first-order velocity term (see _run16_first_order).
    Each stored part is decoded with the reference it was stored with (the
    pulling node adds the same one), then pulled; mask as in run.
    Returns f* decoded (float64)."""
    if shift == "first_order":
        return _run16_first_order(rho_init, steps, G, fmt, work, mask=mask, **kw)
    rho_init = np.asarray(rho_init, dtype=np.float64)
    f = W[None, :, None, None] * rho_init[:, None]
    kind = "node" if shift == "constant" else shift
    if shift == "constant":
        fluid = np.ones(rho_init.shape[1:], bool) if mask is None else mask == 0
        rh = np.broadcast_to(rho_init[:, fluid].mean(axis=1)[:, None, None], rho_init.shape).astype(np.float32)
    else:
        rh = to16(rho_init, fmt)
        _solid_zero(mask, rh)
    _solid_zero(mask, f)
    s = to16(f - _shifted_w(rh, kind), fmt)
    m = work
    for _ in range(steps):
        full = s.astype(m) + _shifted_w(rh, kind).astype(m)
        with np.errstate(invalid="ignore", divide="ignore"):
            out, rho = collide(pull(full, mask).astype(m), G, work=m, mask=mask, **kw)
        out = out.astype(m)
        _solid_zero(mask, out, rho)
        if shift != "constant":
            rh = to16(rho, fmt)
        s = to16(out - _shifted_w(rh, kind).astype(m), fmt)
    return s.astype(np.float64) + _shifted_w(rh, kind)


# ----------------------------------------------------------------------------
# the cases of tests/test_precision_emulation.py, runnable in a worker process
# ----------------------------------------------------------------------------
def case_inputs(case):
    """(mask or None, rho_init, keywords) of a named case: the static droplet
    (128 x 128 periodic, R = 20, tau = 1) or the sinusoidal channel of the GPU
    parity tests (300 x 40, tau = (1, 0.9), wall potentials (0.3, 0.1), body
    force 2e-5; "channel_bgk" or "channel_reg" for the collision)."""
    from paper_1601_00918_gb300 import workloads as wl
    if case == "droplet":
        return None, wl.droplet(128, 128, 20.0, 64.0, 64.0), {}
    nx, ny = 300, 40
    mask = wl.sinusoidal_channel(nx, ny, 12.0, 5.0, 100.0)
    kw = dict(tau=(1.0, 0.9), rho_wall=(0.3, 0.1), g=(2e-5, 0.0), regularized=case == "channel_reg")
    return mask, wl.slug(nx, ny, 0.3 * nx, 0.7 * nx), kw


def run_case(job):
    """job = (case, steps, G, options): the state f* after `steps` steps, 16-bit
    storage when the options name a format ("fmt")."""
    case, steps, G, opts = job
    mask, rho, kw = case_inputs(case)
    opts = dict(opts)
    if "fmt" in opts:
        return run16(rho, steps, G, mask=mask, **kw, **opts)
    return run(rho, steps, G, mask=mask, **kw, **opts)
