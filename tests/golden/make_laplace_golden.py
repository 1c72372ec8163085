"""Write tests/golden/laplace_droplets_128.json with the FP64 oracle.

Static droplets of Section 3.1 on the 128 x 128 periodic box (radii 12, 16,
20, 24, 28; densities 1.0 / 0.03, tanh interface of width 2; tau = 1;
G = -1.79), 6000 oracle steps each (after 1000 steps the pressure waves of
the initial state have not died out: the fit has R^2 = 0.76); radius from tanh fits of the central row
and column (Eq. den-fitting), pressure jump between the centre and the
corner, surface tension from the least-squares line dP = sigma / R + c
(Eq. Young-Laplace_equation).  Calls only oracle/ and the input module.

    python tests/golden/make_laplace_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import analytic  # noqa: E402
from paper_1601_00918_gb300 import workloads as wl  # noqa: E402

N, STEPS, G = 128, 6000, -1.79
RADII = (12.0, 16.0, 20.0, 24.0, 28.0)


def main():
    radii, dps = [], []
    for R0 in RADII:
        P = oracle.Problem(wl.periodic_box(N, N), tau=(1.0, 1.0), G=G)
        f = P.run(P.init(wl.droplet(N, N, R0, N / 2.0, N / 2.0)), STEPS)
        rho, _, pr = P.fields(f)
        radii.append(analytic.droplet_radius(rho[0], N / 2.0, N / 2.0))
        dps.append(float(pr[N // 2, N // 2] - pr[0, 0]))
    sigma, c, r2 = analytic.laplace_fit(radii, dps)
    out = {"_source": "FP64 oracle (oracle/lbm_oracle.c) via tests/golden/make_laplace_golden.py; "
                      "Section 3.1 procedure (Eq. den-fitting, Eq. Young-Laplace_equation)",
           "n": N, "steps": STEPS, "G": G, "tau": [1.0, 1.0], "initial_radii": list(RADII),
           "radii": radii, "dp": dps, "sigma": sigma, "intercept": c, "r2": r2}
    with open(os.path.join(HERE, "laplace_droplets_128.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
