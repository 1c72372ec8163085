"""Write tests/golden/capillary_channel_64.json with the FP64 oracle.

1. Wetting calibration (Section 3.3): slug between flat plates H = 32 apart
   (192 columns, periodic, oil over the middle half), tau = 1, G = -1.79,
   wall potential r (r > 0: rho_s^w = r; r < 0: rho_s^o = -r), 20 000 oracle
   steps; contact angle through water from the tanh interface points and the
   circle fit of Eq. (contact_angle), mean of the two slug ends.
2. Critical body force (Section 3.4, planar 2-D balance of
   oracle/capillary.py) of a slug in the scaled-down sinusoidal channel
   lambda = 64, h0 = 12, A = 6, four periods (256 x 38), slug 1.5 lambda
   centred on a neck, for contact angles 40, 60, 90, 120 and 140 degrees:
   wall potentials from the calibration (monotone interpolation), 20 000
   oracle steps at g = 0, then the oil area (nodes with oil fraction > 1/2)
   and the rear interface on the centre row of the static slug; the bulk
   density is the mean total density where the oil fraction is > 0.9.

Calls only oracle/ and the input module; the runs are independent and use a
process pool (spawn).

    python tests/golden/make_capillary_golden.py
"""
import json
import math
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

G = -1.79
STEPS = 20000
H, NX_PLATE = 32, 192
R_VALUES = (-0.45, -0.3, -0.15, 0.0, 0.15, 0.3, 0.45)
THETAS = (40.0, 60.0, 90.0, 120.0, 140.0)
LAM, AMP_RATIO, SLUG = 64, 0.5, 1.5


def potentials(r):
    return (max(-r, 0.0), max(r, 0.0))


def plate_angle(r):
    import oracle
    from oracle import capillary as cap
    from paper_1601_00918_gb300 import workloads as wl
    mask = wl.straight_channel(NX_PLATE, H)
    rho = wl.slug(NX_PLATE, H + 2, NX_PLATE / 4.0, 3.0 * NX_PLATE / 4.0)
    P = oracle.Problem(mask, tau=(1.0, 1.0), G=G, rho_wall=potentials(r), periodic=(True, False))
    d, _, _ = P.fields(P.run(P.init(rho), STEPS))
    return 0.5 * (cap.contact_angle(d[0], d[1], 1, H, "right") + cap.contact_angle(d[0], d[1], 1, H, "left"))


def channel_state(args):
    theta, rw = args
    import oracle
    from paper_1601_00918_gb300 import workloads as wl
    spec = wl.ChannelSpec(lam=LAM, amp_ratio=AMP_RATIO, slug_len_over_lambda=SLUG, theta_deg=theta, visc_ratio=1.0)
    w = wl.channel_instance(spec)
    P = oracle.Problem(w.mask, tau=(1.0, 1.0), G=G, rho_wall=rw, periodic=w.periodic)
    d, _, _ = P.fields(P.run(P.init(w.rho), STEPS))
    fluid = w.mask == 0
    tot = d[0] + d[1]
    frac = np.where(fluid, d[0] / np.where(fluid, tot, 1.0), 0.0)
    area = float(np.sum(frac > 0.5))
    row = frac[spec.ny // 2]
    oil = np.nonzero(row > 0.5)[0]
    i = int(oil.min())
    x_rear = (i - 1) + (0.5 - row[i - 1]) / (row[i] - row[i - 1])
    rho_bulk = float(tot[fluid & (frac > 0.9)].mean())
    return dict(area=area, x_rear=float(x_rear), rho_bulk=rho_bulk, h0=spec.h0, amp=spec.amp, nx=spec.nx,
                ny=spec.ny)


def main():
    from oracle import capillary as cap
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count() or 1)) as pool:
        thetas_r = pool.map(plate_angle, R_VALUES)
        r_arr, th_arr = np.array(R_VALUES), np.array(thetas_r)
        assert np.all(np.diff(th_arr) < 0), th_arr
        jobs = []
        for th in THETAS:
            r = float(np.interp(th, th_arr[::-1], r_arr[::-1]))
            jobs.append((th, potentials(r)))
        states = pool.map(channel_state, jobs)
    with open(os.path.join(HERE, "laplace_droplets_128.json")) as fh:
        sigma = json.load(fh)["sigma"]
    runs = []
    for (th, rw), st in zip(jobs, states):
        bal, s0, s_crit, _ = cap.critical_force(math.radians(th), st["area"], st["h0"], st["amp"], float(LAM),
                                                st["x_rear"])
        g = sigma * bal / (st["rho_bulk"] * st["nx"])
        runs.append(dict(theta=th, rho_wall=list(rw), balance=bal, s0=s0, s_crit=s_crit, g_crit=g, **st))
    out = {"_source": "FP64 oracle (oracle/lbm_oracle.c, oracle/capillary.py) via "
                      "tests/golden/make_capillary_golden.py; Section 3.3 (Eq. contact_angle) calibration, "
                      "Section 3.4 balance in its planar 2-D form; sigma from laplace_droplets_128.json",
           "G": G, "tau": [1.0, 1.0], "steps": STEPS,
           "calibration": {"H": H, "nx": NX_PLATE, "r": list(R_VALUES), "theta": [float(t) for t in thetas_r]},
           "channel": {"lam": LAM, "amp_ratio": AMP_RATIO, "slug_len_over_lambda": SLUG, "sigma": sigma},
           "runs": runs}
    with open(os.path.join(HERE, "capillary_channel_64.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
