"""Write tests/golden/critical_channel_64.json: the FP64 oracle's own
bisection of the critical body force (Section 3.4) on the scaled-down
sinusoidal channel of capillary_channel_64.json.

For each of the five contact angles of that file (wall potentials from its
Section 3.3 calibration; lambda = 64, h0 = 12, A = 6, four periods,
256 x 38, slug 1.5 lambda centred on a neck, tau = 1, G = -1.79):
  1. run the oracle T_EQ steps at g = 0 (the static slug);
  2. bisect g with oracle/bisect.py from the starting bracket
     [0.5, 2] x the planar 2-D critical force stored in
     capillary_channel_64.json, relative bracket 2 %, bracket checks on;
     each probe restarts from the step-1 state, runs T_OBS oracle steps at
     that g and calls the slug moving when the oil centre of mass moved
     more than lambda / 2 (the sum over the window of the oil momentum over
     the oil mass, as the library's observables integrate it).
Every value stored is computed by the oracle (oracle/lbm_oracle.c,
oracle/bisect.py) from the inputs above; nothing comes from the CUDA path.
The five channels run in parallel (spawned processes); at about 4 ms per
oracle step the whole file takes about an hour per T_OBS on five cores.

    python tests/golden/make_critical_golden.py [T_OBS ...]   (default 80000)
"""
import json
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

REL = 0.02
MAX_PROBES = 30
OUT = os.path.join(HERE, "critical_channel_64.json")


def bisect_channel(args):
    run, gold, t_obs = args
    import oracle
    from oracle.bisect import bisect_critical
    from paper_1601_00918_gb300 import workloads as wl
    ch = gold["channel"]
    spec = wl.ChannelSpec(lam=ch["lam"], amp_ratio=ch["amp_ratio"],
                          slug_len_over_lambda=ch["slug_len_over_lambda"], theta_deg=run["theta"],
                          visc_ratio=1.0)
    w = wl.channel_instance(spec)
    kw = dict(tau=tuple(gold["tau"]), G=gold["G"], rho_wall=tuple(run["rho_wall"]), periodic=w.periodic)
    P0 = oracle.Problem(w.mask, g=(0.0, 0.0), **kw)
    t0 = time.time()
    f_eq = P0.run(P0.init(w.rho), gold["steps"])
    probes = []

    def moving(g):
        P = oracle.Problem(w.mask, g=(g, 0.0), **kw)
        _, hist = P.run(f_eq, t_obs, history=True)
        if hist[:, 4].any():
            probes.append(dict(g=g, disp=None))
            return None
        disp = float(np.sum(hist[:, 2] / hist[:, 0]))
        probes.append(dict(g=g, disp=disp))
        return abs(disp) > 0.5 * spec.lam

    g_ref = run["g_crit"]
    res = bisect_critical(moving, 0.5 * g_ref, 2.0 * g_ref, rel=REL, max_probes=MAX_PROBES,
                          check_bracket=True)
    return dict(theta=run["theta"], t_obs=t_obs, g_start=[0.5 * g_ref, 2.0 * g_ref], probe_log=probes,
                seconds=time.time() - t0, **res)


def main(t_obs_list):
    with open(os.path.join(HERE, "capillary_channel_64.json")) as fh:
        gold = json.load(fh)
    jobs = [(run, gold, t) for t in t_obs_list for run in gold["runs"]]
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(len(jobs), os.cpu_count() or 1)) as pool:
        results = pool.map(bisect_channel, jobs)
    old = {}
    if os.path.exists(OUT):
        with open(OUT) as fh:
            old = {(r["theta"], r["t_obs"]): r for r in json.load(fh)["runs"]}
    for r in results:
        old[(r["theta"], r["t_obs"])] = r
    out = {"_source": "FP64 oracle bisection (oracle/lbm_oracle.c, oracle/bisect.py) via "
                      "tests/golden/make_critical_golden.py; channel, wall potentials and starting "
                      "brackets from capillary_channel_64.json (Section 3.3 calibration, Section 3.4 "
                      "planar balance)",
           "rel_bracket": REL, "t_eq": gold["steps"], "max_probes": MAX_PROBES, "check_bracket": True,
           "disp_threshold": "lambda / 2",
           "runs": sorted(old.values(), key=lambda r: (r["t_obs"], r["theta"]))}
    with open(OUT, "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps([{k: r[k] for k in ("theta", "t_obs", "g_lo", "g_hi", "probes", "status")}
                      for r in out["runs"]], indent=1))


if __name__ == "__main__":
    main([int(a) for a in sys.argv[1:]] or [80000])
