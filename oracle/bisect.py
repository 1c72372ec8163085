"""Bisection of the critical body force, host statement (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 3.4 of the paper looks for the body force g at which a static slug
starts to move (it ramps g and watches the oil centre of mass).  The
protocol restated here bisects instead:
  1. (optional) check the bracket: probe g_hi; while the slug stays static,
     g_lo := g_hi, g_hi := 2 g_hi.  Then probe g_lo; while it moves,
     g_hi := g_lo, g_lo := g_lo / 2;
  2. bisect at the geometric midpoint sqrt(g_lo g_hi): moving -> g_hi := g,
     static -> g_lo := g;
  3. stop once g_hi - g_lo <= rel * g_hi (status 0) or after max_probes
     probes (status 1).
`moving(g)` answers one probe (a fresh run from the state equilibrated at
g = 0); it may return None for an unstable run (status 2).
"""
from __future__ import annotations

import math


def bisect_critical(moving, g_lo: float, g_hi: float, rel: float = 0.02, max_probes: int = 24,
                    check_bracket: bool = True):
    state = "hi" if check_bracket else "bisect"
    probes = 0
    while True:
        g = g_hi if state == "hi" else (g_lo if state == "lo" else math.sqrt(g_lo * g_hi))
        m = moving(g)
        probes += 1
        if m is None:
            return {"g_lo": g_lo, "g_hi": g_hi, "probes": probes, "status": 2}
        if state == "hi":
            if m:
                state = "lo"
            else:
                g_lo, g_hi = g_hi, 2.0 * g_hi
        elif state == "lo":
            if not m:
                state = "bisect"
            else:
                g_hi, g_lo = g_lo, 0.5 * g_lo
        else:
            if m:
                g_hi = g
            else:
                g_lo = g
        if state == "bisect" and g_hi - g_lo <= rel * g_hi:
            return {"g_lo": g_lo, "g_hi": g_hi, "probes": probes, "status": 0}
        if probes >= max_probes:
            return {"g_lo": g_lo, "g_hi": g_hi, "probes": probes, "status": 1}
