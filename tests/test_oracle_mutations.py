"""The oracle's pins catch plausible one-line mistakes in the oracle itself.

Each case below plants one mistake (a dropped term, a flipped sign, a wrong
index or species, a transposed operand) in a copy of oracle/lbm_oracle.c,
compiles the copy into a temporary directory with the oracle's own gcc
flags, points the oracle package at it for the duration of the test, and
runs the fast pins of tests/test_oracle_pins.py: at least one of them has
to fail.  The D3Q19 oracle (oracle/lbm3d_oracle.c) is treated the same way
with the pins of tests/test_oracle_d3q19.py, and the Python modules of the
oracle (the planar critical force and the contact angle, the closed forms
and fits, the bisection protocol, the surrogate's FP64 reference) by
replacing their functions with those of a mutated copy of the source.  The
input module (paper_1601_00918_gb300/workloads.py) feeds both the oracle and
the CUDA path, so a mistake in it would pass every parity test: its own pins
are tested the same way.  Control cases compile the unchanged C sources the same way and check that
every pin of their battery passes, so a failure under a mutation is the
mistake's doing and not the harness's.

Every planted mistake keeps all memory accesses inside their arrays (index
tables stay permutations of 0..8, wrapped indices stay in [0, n)), so a
mutated oracle can give wrong numbers but cannot crash the test process.
"""
import importlib
import importlib.util
import os
import subprocess
import sys
import types

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


# ----------------------------------------------------------------------------
# the Python parts of the oracle: closed forms, the planar critical force,
# the contact angle, the bisection protocol and the surrogate's reference
# ----------------------------------------------------------------------------
CAP = _pins("test_oracle_capillary")


def _python_battery():
    """(name, call) of the pins of the Python oracle modules, cheapest first;
    the Laplace law (about 45 s) and the contact-angle symmetry run (about
    15 s) come last, so only mistakes the others miss pay for them.  The
    unchanged modules pass all of these pins in the regular suite."""
    p, c = PINS, CAP
    return [
        ("worked numbers", p.test_worked_numbers_section_3_4),
        ("bisection brackets", lambda: [p.test_bisection_brackets_a_sharp_threshold(*a) for a in
                                        ((1.3e-4, 1e-4, 4e-4), (5e-4, 1e-4, 2e-4), (3e-5, 1e-4, 4e-4))]),
        ("bisection status", p.test_bisection_status_codes),
        ("MLP layout", p.test_mlp_parameter_count_and_layout),
        ("MLP gradient", p.test_mlp_gradient_matches_central_differences),
        ("MLP closed forms", p.test_mlp_closed_forms),
        ("Adam first step", p.test_adam_first_step_is_lr_times_sign),
        ("meniscus", lambda: [c.test_front_meniscus_against_constructed_circle(*a) for a in
                              ((30, 0, 8.0), (55, 20, 6.0), (120, -15, 10.0), (150, 10, 12.0))]),
        ("channel area", c.test_channel_area_is_the_integral_of_twice_the_half_width),
        ("circle fit", c.test_circle_fit_recovers_a_circle),
        ("synthetic contact angle", lambda: [c.test_contact_angle_of_a_synthetic_circular_interface(t)
                                             for t in (35.0, 115.0)]),
        ("droplet radius", lambda: p.test_droplet_radius_of_a_synthetic_tanh_disc(17.3, 64.0, 64.0)),
        ("Laplace fit", p.test_laplace_fit_recovers_a_known_line),
        ("straight channel / symmetric slug",
         lambda: c.test_balance_vanishes_in_a_straight_channel_and_for_symmetric_slugs(60)),
        ("long-wavelength limit", lambda: c.test_long_wavelength_limit_is_the_curvature_difference(50)),
        ("small-amplitude limit", lambda: c.test_small_amplitude_limit_is_the_wall_slope_term(40)),
        ("water-wet slug on a neck", c.test_water_wet_slug_on_a_neck_rests_symmetrically_and_needs_a_push),
        ("loading path", c.test_loading_path_on_a_constructed_balance),
        ("layered Poiseuille", p.test_layered_poiseuille_reduces_to_parabola),
        ("layered Poiseuille, two components", lambda: p.test_layered_poiseuille_two_components(1.5, 1.0)),
        ("shear wave", p.test_shear_wave_viscosity_single_species),
        ("Laplace law", p.test_laplace_law_droplets),
        ("contact-angle symmetries", c.test_oracle_contact_angle_symmetries),
    ]


# (module, id, what the mistake is, unique text in the module, its replacement)
PY_MUTATIONS = [
    ("capillary", "wall_slope", "h'(x) without its 2 pi / lam",
     "return np.arctan(amp * k * np.sin(k * np.asarray(x, dtype=np.float64)))",
     "return np.arctan(amp * np.sin(k * np.asarray(x, dtype=np.float64)))"),
    ("capillary", "meniscus_phi_sign", "the wall angle entering the front and rear menisci swapped",
     "alpha = 0.5 * math.pi + (phi if front else -phi) - theta",
     "alpha = 0.5 * math.pi + (-phi if front else phi) - theta"),
    ("capillary", "segment_area", "the circular segment without its chord triangle",
     "(a - np.sin(a) * np.cos(a))", "(a - np.sin(a))"),
    ("capillary", "channel_area_k", "the integral of the cosine with k in place of 1 / k",
     "return 2.0 * (h0 * (b - a) - amp / k * (math.sin(k * b) - math.sin(k * a)))",
     "return 2.0 * (h0 * (b - a) - amp * k * (math.sin(k * b) - math.sin(k * a)))"),
    ("capillary", "oil_area_rear_segment", "the rear segment subtracted from the oil area",
     "return between + sr + sf", "return between - sr + sf"),
    ("capillary", "balance_sign", "rear minus front curvature",
     "return kf - kr", "return kr - kf"),
    ("capillary", "jump_length", "a slug counted as moving only after a jump of a whole wavelength",
     "jump = 0.5 * lam if jump is None else jump", "jump = lam if jump is None else jump"),
    ("capillary", "contact_half_width", "the half width between the outermost fluid rows, not the walls",
     "y0 = 0.5 * (y_hi - y_lo + 1)", "y0 = 0.5 * (y_hi - y_lo)"),
    ("capillary", "contact_side", "the angle taken through oil instead of water",
     "return acute if centre_on_oil else 180.0 - acute", "return 180.0 - acute if centre_on_oil else acute"),
    ("analytic", "layered_core_continuity", "the wall layer's velocity at the interface with the core viscosity",
     "+ f * (a * a - b * b) / (2.0 * mu_out)\n", "+ f * (a * a - b * b) / (2.0 * mu_core)\n"),
    ("analytic", "bond_without_d", "the Bond number without the neck half-width",
     "return rho * g * length * d / sigma", "return rho * g * length / sigma"),
    ("analytic", "droplet_diameter", "the droplet's diameter taken for its radius",
     "radii.append(0.5 * (pos[1] - pos[0]))", "radii.append(pos[1] - pos[0])"),
    ("analytic", "tanh_shift_sign", "the interface position entering Eq. (den-fitting) with the wrong sign",
     "return c1 * np.tanh(c2 * (x - c3)) + c4", "return c1 * np.tanh(c2 * (x + c3)) + c4"),
    ("analytic", "laplace_inverse_diameter", "dP fitted against 2 / R",
     "inv_r = 1.0 / np.asarray(radii, dtype=np.float64)", "inv_r = 2.0 / np.asarray(radii, dtype=np.float64)"),
    ("bisect", "arithmetic_first_probe", "the bracket check skipped: the first probe bisects",
     'state = "hi" if check_bracket else "bisect"', 'state = "bisect"'),
    ("bisect", "stop_rule", "the stopping rule relative to g_lo",
     "if state == \"bisect\" and g_hi - g_lo <= rel * g_hi:", "if state == \"bisect\" and g_hi - g_lo <= rel:"),
    ("bisect", "widening", "a failed upper bracket not widened",
     "g_lo, g_hi = g_hi, 2.0 * g_hi", "g_lo, g_hi = g_hi, g_hi"),
    ("mlp", "dsilu", "the SiLU derivative without the z s (1 - s) term",
     "return s * (1.0 + z * (1.0 - s))", "return s * (1.0 + z * s)"),
    ("mlp", "dloss_ds", "dL/ds without its 1/2",
     "d[:, 1] = 0.5 * (1.0 - e * r * r) / B", "d[:, 1] = (1.0 - e * r * r) / B"),
    ("mlp", "adam_bias_correction", "Adam's second moment without its bias correction",
     "vh = v / (1 - b2 ** t)", "vh = v"),
    ("mlp", "unpack_transposed", "weights read as [fan_in, fan_out]",
     "W = theta[o:o + fan_out * fan_in].reshape(fan_out, fan_in)",
     "W = theta[o:o + fan_out * fan_in].reshape(fan_in, fan_out).T"),
]


def _mutate_python(monkeypatch, modname, old, new):
    """Replace every function of oracle.<modname> (or of the module of that
    dotted name) by its counterpart from a copy of the module's source with
    `old` replaced by `new`."""
    real = importlib.import_module(modname if "." in modname else f"oracle.{modname}")
    with open(real.__file__) as fh:
        src = fh.read()
    assert src.count(old) == 1, f"{modname}: the text to replace must occur exactly once"
    mut = types.ModuleType(f"{real.__name__}_mutated")
    mut.__file__ = real.__file__
    monkeypatch.setitem(sys.modules, mut.__name__, mut)      # dataclasses look their module up
    exec(compile(src.replace(old, new), real.__file__, "exec"), mut.__dict__)
    for name, value in vars(mut).items():
        if callable(value) and getattr(value, "__module__", None) == mut.__name__:
            monkeypatch.setattr(real, name, value)


@pytest.mark.slow
@pytest.mark.parametrize("modname,mid,what,old,new", PY_MUTATIONS, ids=[m[1] for m in PY_MUTATIONS])
def test_a_planted_mistake_in_the_python_oracle_fails_a_pin(monkeypatch, modname, mid, what, old, new):
    _mutate_python(monkeypatch, modname, old, new)
    failed = []
    for name, call in _python_battery():
        try:
            call()
        except Exception:
            failed.append(name)
            break
    assert failed, f"no pin caught: {what}"


# ----------------------------------------------------------------------------
# the input module (workloads.py): it feeds both the oracle and the CUDA path,
# so a mistake in it would pass every parity test; its own pins must fail
# ----------------------------------------------------------------------------
CAPI = _pins("test_capi_host")
WETTING = _pins("test_wetting_host")


def _input_battery():
    c, w, p = CAPI, WETTING, PINS
    return [
        ("channel rows", c.test_sinusoidal_channel_rows),
        ("droplet and slug profiles", c.test_droplet_and_slug_profiles),
        ("layered channel rows", c.test_layered_channel_rows),
        ("tube cross sections", c.test_sinusoidal_tube_cross_sections),
        ("channel geometry = library", lambda: [w.test_channel_geometry_is_the_input_module_channel(*a) for a in
                                                ((32, 0.2, 1.0, 4), (48, 0.37, 1.3, 3))]),
        ("flat-interface coexistence", p.test_flat_interface_coexistence_at_the_chosen_g),
    ]


WL = "paper_1601_00918_gb300.workloads"
INPUT_MUTATIONS = [
    ("half_width_sign", "h(x) = h0 + A cos: bulges where the necks are",
     "return h0 - amp * np.cos(2.0 * np.pi", "return h0 + amp * np.cos(2.0 * np.pi"),
    ("channel_centre", "the channel centred on ny / 2 instead of (ny - 1) / 2",
     "        yc = (ny - 1) / 2.0\n", "        yc = ny / 2.0\n"),
    ("tube_centre", "the tube's axis off the middle of its cross section",
     "    c = (n_cross - 1) / 2.0\n", "    c = n_cross / 2.0\n"),
    ("layered_rows", "the wetting layers one row short",
     "core = (y >= 1 + outer) & (y <= width - outer)", "core = (y >= outer) & (y <= width - outer)"),
    ("droplet_inside_out", "species o outside the droplet instead of inside",
     "s = _step(radius - r)", "s = _step(r - radius)"),
    ("tanh_width", "interfaces of width 1 instead of 2",
     "np.tanh(np.asarray(d, dtype=np.float64) / 2.0)", "np.tanh(np.asarray(d, dtype=np.float64))"),
    ("slug_front", "the slug's front end reversed",
     "s = _step(x - x_rear) - _step(x - x_front)\n    ro = rho_lo + (rho_hi - rho_lo) * s\n    return np.stack([ro, rho_hi + rho_lo - ro])\n\n\ndef uniform",
     "s = _step(x - x_rear) - _step(x_front - x)\n    ro = rho_lo + (rho_hi - rho_lo) * s\n    return np.stack([ro, rho_hi + rho_lo - ro])\n\n\ndef uniform"),
    ("first_slug_neck", "the first slug centred one neck too far",
     "first = float(spec.lam * (spec.n_periods // (2 * k)))", "first = float(spec.lam * (spec.n_periods // k))"),
    ("flat_band", "the oil band of the flat interface half as wide",
     "s = _step(x - nx / 4.0) - _step(x - 3.0 * nx / 4.0)", "s = _step(x - nx / 4.0) - _step(x - nx / 2.0)"),
]


@pytest.mark.slow
@pytest.mark.parametrize("mid,what,old,new", INPUT_MUTATIONS, ids=[m[0] for m in INPUT_MUTATIONS])
def test_a_planted_mistake_in_the_input_module_fails_a_pin(monkeypatch, mid, what, old, new):
    _mutate_python(monkeypatch, WL, old, new)
    PINS._flat_interface.cache_clear()
    failed = []
    for name, call in _input_battery():
        try:
            call()
        except Exception:
            failed.append(name)
            break
    PINS._flat_interface.cache_clear()
    assert failed, f"no pin caught: {what}"
