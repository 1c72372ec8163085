"""The oracle's pins catch plausible one-line mistakes in the oracle itself.

Each case below plants one mistake (a dropped term, a flipped sign, a wrong
index or species, a transposed operand) in a copy of oracle/lbm_oracle.c,
compiles the copy into a temporary directory with the oracle's own gcc
flags, points the oracle package at it for the duration of the test, and
runs the fast pins of tests/test_oracle_pins.py: at least one of them has
to fail.  The D3Q19
oracle (oracle/lbm3d_oracle.c) is treated the same way with the pins of
tests/test_oracle_d3q19.py.  A control case
compiles the unchanged source the same way and checks that every pin of the
battery passes, so a failure under a mutation is the mistake's doing and not
the harness's.

Every planted mistake keeps all memory accesses inside their arrays (index
tables stay permutations of 0..8, wrapped indices stay in [0, n)), so a
mutated oracle can give wrong numbers but cannot crash the test process.
"""
import importlib.util
import os
import subprocess

import pytest

import oracle
from oracle import d3q19

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbm_oracle.c")
SRC3 = os.path.join(ROOT, "oracle", "lbm3d_oracle.c")


def _pins(name):
    spec = importlib.util.spec_from_file_location(f"{name}_for_mutations", os.path.join(ROOT, "tests", f"{name}.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


PINS = _pins("test_oracle_pins")
PINS3 = _pins("test_oracle_d3q19")


def _battery():
    """(name, call) of the fast pins, cheapest first (about 10 s in all)."""
    p = PINS
    return [
        ("feq moments", lambda: [p.test_feq_moments(o, r, ux, uy) for o in (2, 3)
                                 for (r, ux, uy) in ((0.7, 0.12, -0.05), (0.03, -0.2, 0.17))]),
        ("rest equilibrium", p.test_feq_rest_is_weights),
        ("open boundary rejected", p.test_oracle_rejects_open_boundary_without_walls),
        ("linear density field force", p.test_force_on_linear_density_field),
        ("species swap", p.test_species_swap_symmetry),
        ("wall potential", p.test_wall_potential_stands_in_for_the_other_species),
        ("closed box at rest", p.test_closed_box_at_rest_stays_at_rest),
        ("momentum balance", lambda: p.test_total_momentum_balance_periodic((1e-4, -3e-5))),
        ("Hermite projection", p.test_regularized_part_is_the_hermite_projection),
        ("step_nodes", lambda: [p.test_step_nodes_equals_step(c) for c in ("periodic_box", "walled_channel")]),
        ("shear wave", p.test_shear_wave_viscosity_single_species),
        ("shear wave, mixture", p.test_shear_wave_mixture_viscosity),
        ("shear wave, regularised", p.test_regularized_shear_wave_keeps_the_viscosity),
        ("mass with walls", p.test_mass_conservation_with_walls),
        ("Poiseuille", p.test_poiseuille_single_species),
        ("bounce-back slip", lambda: p.test_poiseuille_bounce_back_slip_closed_form(0.8)),
        ("uniformly accelerated mixture",
         lambda: p.test_observables_of_a_uniformly_accelerated_mixture((0.7, 1.4))),
        ("instability flag", lambda: [p.test_instability_flag_for_either_species(a) for a in (0, 1)]),
        ("flat interface stress and pressure", p.test_flat_interface_stress_and_equation_of_state),
    ]


# (id, what the mistake is, unique text in lbm_oracle.c, its replacement)
MUTATIONS = [
    ("feq_cubic_sign", "sign of the -(c.u) u^2 / (2 T0^2) term of Eq. (feq)",
     "- cu * uu / (2.0 * T0 * T0)", "+ cu * uu / (2.0 * T0 * T0)"),
    ("feq_drop_u2", "dropped -u^2 / (2 T0) term of Eq. (feq)",
     " - uu / (2.0 * T0);", ";"),
    ("feq_quadratic_power", "T0 instead of T0^2 under (c.u)^2",
     "cu * cu / (2.0 * T0 * T0)", "cu * cu / (2.0 * T0)"),
    ("weight_diagonal", "a diagonal weight 1/9 instead of 1/36",
     "1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0}", "1.0 / 36.0, 1.0 / 9.0, 1.0 / 36.0, 1.0 / 36.0}"),
    ("opp_diagonals", "wrong opposite directions of the diagonals",
     "OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6}", "OPP[9] = {0, 3, 4, 1, 2, 8, 7, 6, 5}"),
    ("bounce_own_direction", "bounce-back returns the direction itself, not its opposite",
     "return fs[fidx(p, a, OPP[i], x, y)];", "return fs[fidx(p, a, i, x, y)];"),
    ("push_instead_of_pull", "streaming source x + c_i instead of x - c_i",
     "int sx = x - CX[i], sy = y - CY[i];", "int sx = x + CX[i], sy = y + CY[i];"),
    ("wrap_off_by_one", "negative indices wrap one node short",
     "return r < 0 ? r + n : r;", "return r < 0 ? r + n - 1 : r;"),
    ("wall_potential_species", "the other species' wall potential at a solid node",
     "if (is_solid(p, solid, x, y)) return p->rho_wall[a];",
     "if (is_solid(p, solid, x, y)) return p->rho_wall[1 - a];"),
    ("force_transposed", "c_y in place of c_x in the force sum of Eq. (comp_interaction)",
     "sx += W[i] * CX[i] * rb;\n        sy += W[i] * CY[i] * rb;\n    }\n    *ax",
     "sx += W[i] * CY[i] * rb;\n        sy += W[i] * CY[i] * rb;\n    }\n    *ax"),
    ("force_own_species", "the force of a species from its own density, not the other's",
     "accel_at(p, rho + (size_t)(1 - a) * n, x, y, &acc[a][0], &acc[a][1]);\n            collide_node",
     "accel_at(p, rho + (size_t)a * n, x, y, &acc[a][0], &acc[a][1]);\n            collide_node"),
    ("force_sign", "the body force subtracted",
     "*ax = p->G * sx + p->g[0];", "*ax = p->G * sx - p->g[0];"),
    ("mixture_velocity_index", "j_x of one species in the mixture's u_y",
     "double uy = (jy[0] + jy[1]) / rt;", "double uy = (jy[0] + jx[1]) / rt;"),
    ("mixture_viscosity_swapped", "the viscosities of the two species swapped in nu_mix",
     "(rho[0] * nu0 + rho[1] * nu1) / rt", "(rho[0] * nu1 + rho[1] * nu0) / rt"),
    ("tau_mix_half", "tau_mix = nu_mix / T0 without the + 1/2",
     "double tau_mix = nu_mix / T0 + 0.5;", "double tau_mix = nu_mix / T0 + 0.25;"),
    ("force_shift_dropped", "the equilibrium velocity shift of Eq. (collision_term) dropped in x",
     "ux + acc[a][0], uy + acc[a][1], feq_s", "ux, uy + acc[a][1], feq_s"),
    ("neq_at_shifted_velocity", "f' taken against the force-shifted equilibrium",
     "oracle_feq(p->eq_order, rho[a], ux, uy, feq_u);",
     "oracle_feq(p->eq_order, rho[a], ux + acc[a][0], uy + acc[a][1], feq_u);"),
    ("relaxation_factor", "f' weighted by 1/tau instead of 1 - 1/tau",
     "(1.0 - 1.0 / tau_mix) * fneq[i]", "(1.0 / tau_mix) * fneq[i]"),
    ("hermite_factor", "the factor 2 of the off-diagonal term of Q_i : Pi dropped",
     "2.0 * qxy * pxy", "qxy * pxy"),
    ("hermite_q_shift", "Q_i = c_i c_i without the - T0 I",
     "double qxx = CX[i] * CX[i] - T0, qyy = CY[i] * CY[i] - T0,",
     "double qxx = CX[i] * CX[i], qyy = CY[i] * CY[i],"),
    ("step_nodes_species", "oracle_step_nodes takes its own species' neighbour densities",
     "double rb = density_at(p, solid, fin, b, x + CX[i], y + CY[i]);",
     "double rb = density_at(p, solid, fin, a, x + CX[i], y + CY[i]);"),
    ("half_force_in_velocity", "half the force left out of the physical velocity u",
     "ux = (jx + 0.5 * (r0 * acc[0][0] + r1 * acc[1][0])) / rt;",
     "ux = jx / rt;"),
    ("init_species", "the initial state of one species filled from the other's densities",
     "W[i] * rho_init[a * n + k];", "W[i] * rho_init[(1 - a) * n + k];"),
    ("accel_field_species", "the acceleration field taken from the species' own density",
     "if (!solid[k]) accel_at(p, rho + (size_t)(1 - a) * n, x, y, &ax, &ay);",
     "if (!solid[k]) accel_at(p, rho + (size_t)a * n, x, y, &ax, &ay);"),
    ("oil_momentum_half_force", "half the force left out of the oil momentum observable",
     "px += mac[2] + 0.5 * r0 * acc[0][0];", "px += mac[2];"),
    ("max_u_component", "max|u| over u_x only",
     "double u2 = ux * ux + uy * uy;", "double u2 = ux * ux;"),
    ("instability_flag_species", "the instability flag watching one species only",
     "if (!(r0 >= 0.0) || !(r1 >= 0.0)) bad = 1.0;", "if (!(r0 >= 0.0)) bad = 1.0;"),
    ("pressure_sign", "the interaction term of the equation of state with the wrong sign",
     "pr = T0 * rt - p->G * T0 * r0 * r1;", "pr = T0 * rt + p->G * T0 * r0 * r1;"),
]


def _compile(source, out_dir, name):
    c = os.path.join(out_dir, f"{name}.c")
    so = os.path.join(out_dir, f"lib{name}.so")
    with open(c, "w") as fh:
        fh.write(source)
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fno-fast-math",
                           "-ffp-contract=off", c, "-o", so, "-lm"])
    return so


def _run_battery(monkeypatch, so, stop_at_first=True, module=oracle, battery=None):
    """Point the oracle module `module` at `so`, run the battery, return the
    names of the pins that failed."""
    monkeypatch.setattr(module, "_lib", None)
    monkeypatch.setattr(module, "build", lambda force=False: so)
    PINS._flat_interface.cache_clear()      # a relaxed state of another build
    failed = []
    for name, call in (battery or _battery)():
        try:
            call()
        except Exception:   # an assertion, or the oracle refusing the run
            failed.append(name)
            if stop_at_first:
                break
    return failed


@pytest.mark.slow
def test_control_unchanged_source_passes_the_battery(tmp_path, monkeypatch):
    with open(SRC) as fh:
        src = fh.read()
    so = _compile(src, str(tmp_path), "control")
    assert _run_battery(monkeypatch, so, stop_at_first=False) == []


@pytest.mark.slow
@pytest.mark.parametrize("mid,what,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_a_planted_mistake_fails_a_pin(tmp_path, monkeypatch, mid, what, old, new):
    with open(SRC) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"mutation {mid}: the text to replace must occur exactly once"
    so = _compile(src.replace(old, new), str(tmp_path), mid)
    failed = _run_battery(monkeypatch, so)
    assert failed, f"no pin caught: {what}"


# ----------------------------------------------------------------------------
# the D3Q19 oracle
# ----------------------------------------------------------------------------
def _battery3():
    """(name, call) of every D3Q19 pin (about 2 s in all)."""
    p = PINS3
    return [
        ("lattice moments", p.test_lattice_moments),
        ("feq moments", lambda: [p.test_feq_moments(o, r, u) for o in (2, 3)
                                 for (r, u) in ((0.7, (0.11, -0.04, 0.07)), (1.3, (0.02, 0.2, -0.12)))]),
        ("axis permutation", p.test_axis_permutation_commutes_with_the_step),
        ("momentum balance", p.test_total_momentum_grows_by_mass_times_g),
        ("Hermite projection", p.test_regularized_part_is_the_hermite_projection),
        ("z-uniform flow = D2Q9", lambda: [p.test_z_uniform_flow_reproduces_the_d2q9_oracle(o) for o in (2, 3)]),
        ("mass in the tube", p.test_mass_conservation_in_the_sinusoidal_tube),
        ("uniformly accelerated mixture", p.test_uniformly_accelerated_mixture),
    ]


MUTATIONS3 = [
    ("weight_z_faces", "the two z faces weighted 1/36 instead of 1/18",
     "(i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0)", "(i <= 4 ? 1.0 / 18.0 : 1.0 / 36.0)"),
    ("feq_cubic_sign", "sign of the -(c.u) u^2 / (2 T0^2) term of Eq. (feq)",
     "- cu * uu / (2.0 * T0 * T0)", "+ cu * uu / (2.0 * T0 * T0)"),
    ("feq_uz_dropped", "u_z left out of u^2 in Eq. (feq)",
     "double uu = ux * ux + uy * uy + uz * uz;", "double uu = ux * ux + uy * uy;"),
    ("force_z_transposed", "c_y in place of c_z in the z force sum",
     "s[2] += weight(i) * CZ[i] * rb;", "s[2] += weight(i) * CY[i] * rb;"),
    ("momentum_z_transposed", "c_y in place of c_z in the z momentum",
     "j[a][2] += CZ[i] * fl[a][i];", "j[a][2] += CY[i] * fl[a][i];"),
    ("pull_z_sign", "streaming source z + c_z instead of z - c_z",
     "node(p, x - CX[i], y - CY[i], z - CZ[i]);", "node(p, x - CX[i], y - CY[i], z + CZ[i]);"),
    ("bounce_own_direction", "bounce-back returns the direction itself, not its opposite",
     "return fs[fidx(p, a, opposite(i), node(p, x, y, z))];", "return fs[fidx(p, a, i, node(p, x, y, z))];"),
    ("hermite_trace_2d", "Q_i = c_i c_i - T0 I with the T0 dropped along z",
     "(r == s ? T0 : 0.0)", "(r == s && r < 2 ? T0 : 0.0)"),
    ("force_own_species", "the force of a species from its own density, not the other's",
     "for (int a = 0; a < 2; a++) accel_at(p, rho + (size_t)(1 - a) * n, x, y, z, acc[a]);",
     "for (int a = 0; a < 2; a++) accel_at(p, rho + (size_t)a * n, x, y, z, acc[a]);"),
    ("force_shift_z_dropped", "the equilibrium velocity shift dropped along z",
     "u[2] + acc[a][2], feq_s", "u[2], feq_s"),
    ("mixture_viscosity_swapped", "the viscosities of the two species swapped in nu_mix",
     "(rho[0] * nu0 + rho[1] * nu1) / rt", "(rho[0] * nu1 + rho[1] * nu0) / rt"),
    ("wall_potential_species", "the other species' wall potential at a solid node",
     "if (solid[k]) return p->rho_wall[a];", "if (solid[k]) return p->rho_wall[1 - a];"),
    ("oil_momentum_half_force", "half the force left out of the oil momentum observable",
     "px += mac[2] + 0.5 * r0 * acc[0][0];", "px += mac[2];"),
    ("fields_half_force", "half the force left out of the physical velocity of the fields",
     "u[d] = (jx[d] + 0.5 * (r0 * acc[0][d] + r1 * acc[1][d])) / (r0 + r1);", "u[d] = jx[d] / (r0 + r1);"),
    ("max_u_without_z", "max|u| over u_x and u_y only",
     "for (int d = 0; d < 3; d++) {\n                    double ud", "for (int d = 0; d < 2; d++) {\n                    double ud"),
]


@pytest.mark.slow
def test_control_unchanged_d3q19_source_passes_the_battery(tmp_path, monkeypatch):
    with open(SRC3) as fh:
        src = fh.read()
    so = _compile(src, str(tmp_path), "control3")
    assert _run_battery(monkeypatch, so, stop_at_first=False, module=d3q19, battery=_battery3) == []


@pytest.mark.slow
@pytest.mark.parametrize("mid,what,old,new", MUTATIONS3, ids=[m[0] for m in MUTATIONS3])
def test_a_planted_mistake_in_the_d3q19_oracle_fails_a_pin(tmp_path, monkeypatch, mid, what, old, new):
    with open(SRC3) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"mutation {mid}: the text to replace must occur exactly once"
    so = _compile(src.replace(old, new), str(tmp_path), mid + "3")
    failed = _run_battery(monkeypatch, so, module=d3q19, battery=_battery3)
    assert failed, f"no pin caught: {what}"
