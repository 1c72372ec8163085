"""Host tests of the bypass geometry (two channels with joined ends, the
paper's closing outlook) and of its plane-Poiseuille resistance ratio."""
import numpy as np
import pytest

from paper_1601_00918_gb300 import workloads as wl


def test_bypass_geometry_and_resistance_ratio():
    """The bypass mask has the branch widths it is built with; the blocked
    variant differs only by the lower branch; every fluid node is connected
    to every other (one periodic loop); the slug fills only the upper
    branch; the resistance ratio is 2."""
    s, b = wl.BypassSpec(), wl.BypassSpec(blocked=True)
    m, mb = wl.bypass_channel(s).mask, wl.bypass_channel(b).mask
    xb0 = s.lm + s.chamber
    assert np.count_nonzero(m[:, 10] == 0) == s.wm
    assert np.count_nonzero(m[:, int(s.x_neck)] == 0) == s.hl + 2 * round(s.h0 - s.amp)
    assert np.count_nonzero(m[1:1 + s.hl, xb0:xb0 + s.branch_len]) == 0
    assert np.all(mb[1:1 + s.hl, xb0:xb0 + s.branch_len] == 1)
    diff = m != mb
    assert np.all(diff[1:1 + s.hl, xb0:xb0 + s.branch_len]) and np.count_nonzero(diff) == s.hl * s.branch_len
    assert wl.bypass_resistance_ratio(s) == pytest.approx(2.0)
    # one connected fluid region (periodic in x), in both variants
    for mm in (m, mb):
        ny, nx = mm.shape
        seen = np.zeros_like(mm, dtype=bool)
        start = tuple(np.argwhere(mm == 0)[0])
        stack = [start]
        seen[start] = True
        while stack:
            y, x = stack.pop()
            for dy, dx in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                yy, xx = y + dy, (x + dx) % nx
                if 0 <= yy < ny and mm[yy, xx] == 0 and not seen[yy, xx]:
                    seen[yy, xx] = True
                    stack.append((yy, xx))
        assert seen.sum() == np.count_nonzero(mm == 0)
    w = wl.bypass_channel(s)
    oil = (w.rho[0] > 0.5) & (m == 0)
    ys, xs = np.nonzero(oil)
    assert ys.min() >= 1 + s.hl + s.island
    assert abs(xs.mean() - s.x_neck) < 1.0
    assert xs.max() - xs.min() + 1 == pytest.approx(s.slug_len_over_lambda * s.lam, abs=2)
