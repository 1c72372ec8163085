"""FP32 emulation of the two-component step on a periodic box (numpy).

TEST INFRASTRUCTURE ONLY: tests/test_fp32_emulation.py uses it to show where
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


def step(f, G, g=(0.0, 0.0), work=np.float32, density="work", dev="exact_constants", compose="work",
         weight_kind="nearest"):
    """One step at tau = 1 in working precision `work`; `f` keeps its dtype
    (the storage).  density: "work" | "exact" | "exact_rounded"; dev: "exact_constants" |
    "rounded_t0"; compose: "work" | "single_rounding"; weight_kind: as in
    weights()."""
    store = f.dtype
    m = work
    w = weights(m, weight_kind)
    # pull (streaming): f_i(x) = f*_i(x - c_i)
    fl = np.stack([np.roll(f[:, i], (CY[i], CX[i]), axis=(-2, -1)) for i in range(9)], axis=1).astype(m)
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
    out = np.empty(f.shape, dtype=store)
    for a in range(2):
        # Eq. (comp_interaction) / rho^a: G sum_i w_i c_i rho^b(x + c_i)
        rb = rho[1 - a]
        d1 = _shift(rb, 1, 1) - _shift(rb, -1, -1)
        sx = w[1] * (_shift(rb, 1, 0) - _shift(rb, -1, 0)) + w[5] * (d1 + (_shift(rb, 1, -1) - _shift(rb, -1, 1)))
        sy = w[2] * (_shift(rb, 0, 1) - _shift(rb, 0, -1)) + w[5] * (d1 + (_shift(rb, -1, 1) - _shift(rb, 1, -1)))
        # Eq. (collision_term): the equilibrium at the force-shifted velocity
        vx = ux + (m(G) * sx + m(g[0]))
        vy = uy + (m(G) * sy + m(g[1]))
        vv = vx * vx + vy * vy
        t0 = m(1.0 / 3.0)
        for i in range(9):
            cu = m(CX[i]) * vx + m(CY[i]) * vy
            if dev == "exact_constants":
                d = cu * (m(3) + cu * (m(4.5) + m(4.5) * cu)) - m(1.5) * vv * (m(1) + m(3) * cu)
            else:
                d = (cu / t0 + cu * cu / (m(2) * t0 * t0) - vv / (m(2) * t0)
                     + cu * cu * cu / (m(6) * t0 * t0 * t0) - cu * vv / (m(2) * t0 * t0))
            if compose == "single_rounding":
                out[a, i] = (W[i] * rho64[a] + (w[i] * rho[a] * d).astype(np.float64)).astype(store)
            else:
                wr = w[i] * rho[a]
                out[a, i] = (wr + wr * d).astype(store)
    return out


def run(rho_init, steps, G, store=np.float32, **kw):
    """`steps` steps from the rest equilibrium of rho_init; returns f*."""
    f = initial_state(rho_init, store)
    for _ in range(steps):
        f = step(f, G, **kw)
    return f
