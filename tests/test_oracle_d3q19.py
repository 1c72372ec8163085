"""Pins of the D3Q19 oracle (oracle/d3q19.py, oracle/lbm3d_oracle.c) against
what the lattice, the mathematics and the pinned D2Q9 oracle fix.

* the velocity set: weights sum to 1, odd moments vanish, second moments are
  T0 I and fourth moments isotropic (3 T0^2, T0^2);
* Eq. (feq) on D3Q19: mass, momentum and momentum flux exactly, and the
  third moments D3Q19 can carry (xxy-type) equal
  rho (T0 u_y + u_x^2 u_y - u_z^2 u_y / 2), derived by hand from the four
  lattice edges in the x-y plane;
* a flow that does not depend on z: D3Q19 projected onto the plane (the
  populations summed over c_z) has exactly the D2Q9 weights, and the plain
  BGK step projects onto the D2Q9 step, so a z-extruded channel with walls,
  wall potentials, interaction and body force reproduces the D2Q9 oracle to
  rounding;
* a permutation of the axes commutes with the step (no direction treated
  apart);
* mass conservation with walls in the paper's tube geometry, total momentum
  growing by M g per step in a periodic box, and a uniform mixture under a
  body force moving as one accelerated body (the observables and the
  velocity field carry the half-step force);
* the regularised part is the second-order Hermite projection.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import d3q19
from paper_1601_00918_gb300 import workloads as wl

T0 = 1.0 / 3.0
G = -1.79


def test_lattice_moments():
    c, w = d3q19.lattice()
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.allclose(w @ c, 0.0, atol=1e-16)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", w, c, c), T0 * np.eye(3), atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0.0, atol=1e-16)
    for a in range(3):
        assert np.sum(w * c[:, a] ** 4) == pytest.approx(3 * T0 ** 2, abs=1e-15)
        for b in range(3):
            if a != b:
                assert np.sum(w * c[:, a] ** 2 * c[:, b] ** 2) == pytest.approx(T0 ** 2, abs=1e-15)
    # every velocity has its opposite, and the set is the 19 of |c|^2 <= 2
    assert sorted(map(tuple, c)) == sorted(map(tuple, -c))
    assert sorted(map(tuple, c)) == sorted(v for v in itertools.product((-1, 0, 1), repeat=3)
                                           if sum(x * x for x in v) <= 2)


@pytest.mark.parametrize("order", [2, 3])
@pytest.mark.parametrize("rho,u", [(1.0, (0.0, 0.0, 0.0)), (0.7, (0.11, -0.04, 0.07)),
                                   (0.03, (-0.18, 0.15, -0.09)), (1.3, (0.02, 0.2, -0.12))])
def test_feq_moments(order, rho, u):
    c, _ = d3q19.lattice()
    f = d3q19.feq(rho, *u, order=order)
    u = np.asarray(u)
    assert f.sum() == pytest.approx(rho, rel=1e-14)
    np.testing.assert_allclose(f @ c, rho * u, atol=1e-15)
    np.testing.assert_allclose(np.einsum("i,ia,ib->ab", f, c, c), rho * np.outer(u, u) + T0 * rho * np.eye(3),
                               atol=1e-15)
    # third moments carried by D3Q19: only the four edges (+-1, +-1) in the
    # (a, b) plane have c_a^2 c_b != 0; summing the cubic terms of Eq. (feq)
    # over them (weight 1/36) gives u_a^2 u_b from (c.u)^3 / (6 T0^3) and
    # -u^2 u_b / 2 from -(c.u) u^2 / (2 T0^2), i.e. the Maxwellian's
    # u_a^2 u_b short of u_c^2 u_b / 2 along the third axis c
    for a, b in itertools.permutations(range(3), 2):
        cc = 3 - a - b
        m = np.sum(f * c[:, a] ** 2 * c[:, b])
        ref = rho * (T0 * u[b] + ((u[a] ** 2 - 0.5 * u[cc] ** 2) * u[b] if order == 3 else 0.0))
        assert m == pytest.approx(ref, abs=1e-15), (a, b)


def _project(f3):
    """D3Q19 populations [2, 19, nz, ny, nx] of a z-uniform state -> D2Q9
    populations [2, 9, ny, nx] of one z plane (sum over c_z)."""
    c, _ = d3q19.lattice()
    out = np.zeros((2, 9) + f3.shape[3:])
    for i in range(19):
        k = [j for j in range(9) if oracle.CX[j] == c[i, 0] and oracle.CY[j] == c[i, 1]][0]
        out[:, k] += f3[:, i, 0]
    return out


@pytest.mark.parametrize("eq_order", [2, 3])
def test_z_uniform_flow_reproduces_the_d2q9_oracle(eq_order):
    """A sinusoidal channel with a slug, wall potentials, interaction and a
    body force, extruded over three periodic z planes: after 40 steps every
    z plane of the D3Q19 state, projected, equals the D2Q9 oracle's state to
    1e-14, and the masses and the oil momentum per plane agree."""
    mask2 = wl.sinusoidal_channel(60, 20, 6.0, 3.0, 30.0)
    rho2 = wl.slug(60, 20, 20.0, 42.0)
    kw = dict(tau=(1.0, 0.85), G=G, rho_wall=(0.4, 0.1), eq_order=eq_order)
    P2 = oracle.Problem(mask2, g=(2e-5, -1e-6), periodic=(True, False), **kw)
    f2, h2 = P2.run(P2.init(rho2), 40, history=True)
    nz = 3
    mask3 = np.repeat(mask2[None], nz, axis=0)
    rho3 = np.repeat(rho2[:, None], nz, axis=1)
    P3 = d3q19.Problem3(mask3, g=(2e-5, -1e-6, 0.0), periodic=(True, False, True), **kw)
    f3, h3 = P3.run(P3.init(rho3), 40, history=True)
    for z in range(nz):
        np.testing.assert_allclose(_project(f3[:, :, z:z + 1]), f2, rtol=0, atol=1e-14)
    np.testing.assert_allclose(h3[:, :3] / nz, h2[:, :3], rtol=1e-12, atol=1e-18)


def test_axis_permutation_commutes_with_the_step():
    """A random mixture in a 7 x 6 x 5 periodic box with a body force along
    all three axes, and the same problem with its axes cycled (x -> y -> z
    -> x, the force cycled with them): after 6 steps the densities and
    velocities are the cycled ones, to 1e-14 (a velocity or weight of one
    axis treated apart would break this)."""
    rng = np.random.default_rng(4)
    nz, ny, nx = 5, 6, 7
    rho = 0.5 + 0.4 * rng.random((2, nz, ny, nx))
    g = (3e-5, -2e-5, 1e-5)
    P = d3q19.Problem3(np.zeros((nz, ny, nx), np.uint8), tau=(0.9, 1.2), G=G, g=g)
    r1, u1 = P.fields(P.run(P.init(rho), 6))
    # cycled: new axes (x', y', z') = (z, x, y): array [z', y', x'] = [y, x, z]
    rho_c = np.transpose(rho, (0, 2, 3, 1))
    Pc = d3q19.Problem3(np.zeros(rho_c.shape[1:], np.uint8), tau=(0.9, 1.2), G=G, g=(g[2], g[0], g[1]))
    r2, u2 = Pc.fields(Pc.run(Pc.init(rho_c), 6))
    np.testing.assert_allclose(r2, np.transpose(r1, (0, 2, 3, 1)), rtol=0, atol=1e-14)
    u1c = np.transpose(u1, (0, 2, 3, 1))
    np.testing.assert_allclose(u2, np.stack([u1c[2], u1c[0], u1c[1]]), rtol=0, atol=1e-14)


def test_mass_conservation_in_the_sinusoidal_tube():
    """The paper's geometry (a periodic tube of circular cross sections,
    radius 6 - 2.5 cos(2 pi x / 24)) with an oil slug, wall potentials and
    a body force: each species' mass is conserved to 1e-13 over 60 steps
    (halfway bounce-back returns every population that meets a wall)."""
    mask = wl.sinusoidal_tube(48, 18, 6.0, 2.5, 24.0)
    P = d3q19.Problem3(mask, tau=(1.0, 0.9), G=G, rho_wall=(0.1, 0.4), g=(1e-5, 0.0, 0.0),
                       periodic=(True, False, False), collision="regularized")
    f0 = P.init(wl.tube_slug(48, 18, 14.0, 34.0))
    _, hist = P.run(f0, 60, history=True)
    m0 = np.array([f0[0].sum(), f0[1].sum()])
    np.testing.assert_allclose(hist[:, 0], m0[0], rtol=1e-13)
    np.testing.assert_allclose(hist[:, 1], m0[1], rtol=1e-13)
    assert not hist[:, 4].any()
    assert (mask == 0).sum() > 0.2 * mask.size


def test_total_momentum_grows_by_mass_times_g():
    """Periodic box, random mixture, interaction on: the inter-species forces
    cancel pairwise, so the total momentum (physical velocity) grows by
    exactly (M^o + M^w) g per step."""
    rng = np.random.default_rng(8)
    rho = 0.4 + 0.5 * rng.random((2, 4, 5, 6))
    g = np.array([2e-5, -1e-5, 3e-5])
    P = d3q19.Problem3(np.zeros((4, 5, 6), np.uint8), tau=(0.8, 1.1), G=G, g=tuple(g))
    f = P.run(P.init(rho), 3)
    r0, u0 = P.fields(f)
    r1, u1 = P.fields(P.run(f, 1))
    p0 = np.einsum("xzyk,zyk->x", u0, r0.sum(axis=0))
    p1 = np.einsum("xzyk,zyk->x", u1, r1.sum(axis=0))
    np.testing.assert_allclose(p1 - p0, r0.sum() * g, rtol=1e-9, atol=1e-16)


def test_regularized_part_is_the_hermite_projection():
    """From a spatially uniform random state (the pull is the identity),
    G = 0, g = 0: the regularised non-equilibrium part has no mass and no
    momentum and carries the full non-equilibrium momentum flux, and equals
    w_i Q_i : Pi / (2 T0^2) computed here from the plain part."""
    c, w = d3q19.lattice()
    rng = np.random.default_rng(3)
    f0 = rng.uniform(0.01, 0.1, size=(2, 19))
    tau = 0.8

    def one_step(collision):
        P = d3q19.Problem3(np.zeros((3, 3, 3), np.uint8), tau=(tau, tau), G=0.0, collision=collision)
        f = np.broadcast_to(f0[:, :, None, None, None], (2, 19, 3, 3, 3)).copy()
        out, _ = P.step(f)
        return out[:, :, 1, 1, 1]

    rho = f0.sum(axis=1)
    u = (f0 @ c).sum(axis=0) / rho.sum()
    for a in range(2):
        eq = d3q19.feq(rho[a], *u)
        neq = f0[a] - eq
        fb = (one_step("bgk")[a] - eq) / (1.0 - 1.0 / tau)
        fr = (one_step("regularized")[a] - eq) / (1.0 - 1.0 / tau)
        np.testing.assert_allclose(fb, neq, atol=1e-14)
        Pi = np.einsum("i,ia,ib->ab", neq, c, c)
        Q = np.einsum("ia,ib->iab", c, c) - T0 * np.eye(3)[None]
        ref = w * np.einsum("iab,ab->i", Q, Pi) / (2.0 * T0 * T0)
        np.testing.assert_allclose(fr, ref, atol=1e-14)
        assert abs(fr.sum()) < 1e-14 and np.allclose(fr @ c, 0.0, atol=1e-14)
        np.testing.assert_allclose(np.einsum("i,ia,ib->ab", fr, c, c), Pi, atol=1e-14)


def test_uniformly_accelerated_mixture():
    """A uniform mixture at rest in a periodic box under a body force along
    all three axes moves as one body: the state pulled in step s carries
    velocity s g, and the physical velocity adds half a step of force, so
    the oil momentum observable is M^o (s + 1/2) g_x, max|u| is
    (s + 1/2)|g|, and the velocity field after N steps is (N + 1/2) g at
    every node."""
    n, steps = 4, 30
    g = np.array([3e-5, -2e-5, 4e-5])
    P = d3q19.Problem3(np.zeros((n, n, n), np.uint8), tau=(0.7, 1.4), G=G, g=tuple(g))
    rho = np.empty((2, n, n, n))
    rho[0], rho[1] = 0.7, 0.4
    f, hist = P.run(P.init(rho), steps, history=True)
    s = np.arange(steps)
    mo = 0.7 * n ** 3
    np.testing.assert_allclose(hist[:, 2], mo * (s + 0.5) * g[0], rtol=1e-9)
    np.testing.assert_allclose(hist[:, 3], (s + 0.5) * np.linalg.norm(g), rtol=1e-9)
    _, u = P.fields(f)
    np.testing.assert_allclose(u, np.broadcast_to(((steps + 0.5) * g)[:, None, None, None], u.shape), rtol=1e-9)
