"""Where the FP32 and 16-bit errors of the step come from (the FP32
contract: relative L-infinity <= 1e-5 on rho and u after 1000 steps, mass
drift <= 1e-6).

The numpy emulation of tests/precision_emulation.py steps the static droplet
(128 x 128 periodic, R = 20, tau = 1) and the sinusoidal channel of the GPU
parity tests (300 x 40, walls, wall potentials, body force, tau = (1, 0.9),
plain BGK and regularised) with each stage in a chosen precision, and is
compared with the FP64 oracle after 1000 steps (u, relative L-infinity):

| form                                                        | droplet | channel BGK / reg. |
|-------------------------------------------------------------|---------|--------------------|
| FP32 storage, FP64 arithmetic                                | 3.0e-6  |                    |
| plain FP32 (weights summing to 1, rest population by mass)  | 1.7e-5  | 2.0e-5 / 1.7e-5    |
| compensated: density sums exact, w_i rho exact, one rounding | 3.3e-6  | 7.7e-6 / 6.3e-6    |
| the same, deviation written with a rounded T0                | 1.4e-5  |                    |
| the same, exact density rounded once (its low part dropped)  | 6.3e-6  |                    |

The GPU's two FP32 forms measure u 1.4e-5 to 2.2e-5 (plain) and 3.5e-6 to
4.6e-6 (compensated) on the same cases.  So the storage is not the limit;
plain FP32 arithmetic is, through the density sums and the composition
f*_i = w_i rho (1 + D_i) + (1 - 1/tau) f'_i; with both exact and the
deviation D_i written with constants exact in binary, FP32 meets the
contract.  Correctly rounded FP32 weights sum to 1 + 2^-27 and create that
fraction of mass every step unless the rest population closes the mass.
"""
import numpy as np
import pytest

import oracle
from paper_1601_00918_gb300 import workloads as wl

import precision_emulation as em

pytestmark = pytest.mark.slow

G = -1.79
N, STEPS = 128, 1000
# the two FP32 forms of the CUDA library, as emulation options
PLAIN = dict(weight_kind="sum_to_one", rest="by_mass")
COMPENSATED = dict(density="exact", compose="single_rounding", weight_kind="sum_to_one", rest="by_mass")
CHANNEL = dict(tau=(1.0, 0.9), rho_wall=(0.3, 0.1), g=(2e-5, 0.0))


def channel_geometry():
    nx, ny = 300, 40
    return wl.sinusoidal_channel(nx, ny, 12.0, 5.0, 100.0), wl.slug(nx, ny, 0.3 * nx, 0.7 * nx)


@pytest.fixture(scope="module")
def droplet():
    rho0 = wl.droplet(N, N, 20.0, N / 2.0, N / 2.0)
    P = oracle.Problem(wl.periodic_box(N, N), tau=(1.0, 1.0), G=G)
    rho_r, u_r, _ = P.fields(P.run(P.init(rho0), STEPS))
    return rho0, P, rho_r, u_r


def errors(case, f):
    """(rho, u) relative L-infinity errors and the per-species mass drift."""
    rho0, P, rho_r, u_r = case
    rho, u, _ = P.fields(np.asarray(f, dtype=np.float64))
    fluid = P.mask == 0
    m0 = rho0[:, fluid].sum(axis=1)
    m = np.asarray(f, dtype=np.float64).reshape(2, 9, -1).sum(axis=(1, 2))
    return (np.max(np.abs(rho - rho_r)[:, fluid]) / np.max(rho_r[:, fluid]),
            np.max(np.abs(u - u_r)) / np.max(np.abs(u_r)), np.abs(m - m0) / m0)


def test_the_emulation_in_fp64_is_the_oracle():
    """The emulation is a statement of the same step: in FP64 it gives the
    oracle's state to rounding on the droplet (100 steps) and on the walled
    channel with wall potentials, body force and mixed tau, plain BGK and
    regularised (50 steps)."""
    rho0 = wl.droplet(N, N, 20.0, N / 2.0, N / 2.0)
    P = oracle.Problem(wl.periodic_box(N, N), tau=(1.0, 1.0), G=G)
    f = em.run(rho0, 100, G, store=np.float64, work=np.float64)
    np.testing.assert_allclose(f, P.run(P.init(rho0), 100), rtol=0, atol=1e-13)
    mask, rho = channel_geometry()
    for collision in ("bgk", "regularized"):
        P = oracle.Problem(mask, G=G, periodic=(True, False), collision=collision, **CHANNEL)
        for rest in ("equilibrium", "by_mass"):
            f = em.run(rho, 50, G, store=np.float64, work=np.float64, mask=mask, rest=rest,
                       regularized=collision == "regularized", **CHANNEL)
            np.testing.assert_allclose(f, P.run(P.init(rho), 50), rtol=0, atol=1e-13)


def test_fp32_weights():
    """Each of the nine weights correctly rounded to FP32, they add up to
    1 + 2^-27; with 1/36 one unit in the last place lower they add up to
    exactly 1."""
    assert em.weights(np.float32).astype(np.float64).sum() == 1.0 + 2.0 ** -27
    assert em.weights(np.float32, "sum_to_one").astype(np.float64).sum() == 1.0


def test_fp32_storage_alone_meets_the_contract(droplet):
    err_rho, err_u, drift = errors(droplet, em.run(droplet[0], STEPS, G, work=np.float64))
    assert err_rho < 1e-6 and err_u < 5e-6, (err_rho, err_u)
    assert np.all(drift < 1e-6)


def test_correctly_rounded_weights_create_mass(droplet):
    """All stages in FP32 with correctly rounded weights and the rest
    population from its equilibrium: the mass grows by 2^-27 per step
    (7.5e-6 after 1000 steps), more than the contract allows."""
    err_rho, _, drift = errors(droplet, em.run(droplet[0], STEPS, G))
    assert np.all(np.abs(drift - STEPS * 2.0 ** -27) < 0.1 * STEPS * 2.0 ** -27), drift
    assert err_rho > 1e-5


def test_plain_fp32_arithmetic_misses_the_velocity_bound(droplet):
    """The plain FP32 form (weights summing to 1, the rest population closing
    the mass): mass and rho within the contract, u not (1.7e-5)."""
    err_rho, err_u, drift = errors(droplet, em.run(droplet[0], STEPS, G, **PLAIN))
    assert np.all(drift < 1e-6) and err_rho < 5e-6, (drift, err_rho)
    assert err_u > 1.2e-5, err_u


def test_compensated_fp32_meets_the_contract(droplet):
    """Density sums and w_i rho exact, each stored population rounded once,
    everything else FP32: u 3.3e-6.  Written with a rounded T0 instead of
    exact constants the deviation alone puts u back above the contract
    (1.4e-5); rounding the exact density once, so that its low part never
    reaches the stored populations, about doubles the error (6.3e-6)."""
    err_rho, err_u, drift = errors(droplet, em.run(droplet[0], STEPS, G, **COMPENSATED))
    assert err_rho < 1e-6 and err_u < 5e-6, (err_rho, err_u)
    assert np.all(drift < 1e-6)
    _, err_u_t0, _ = errors(droplet, em.run(droplet[0], STEPS, G, **dict(COMPENSATED, dev="rounded_t0")))
    assert err_u_t0 > 1e-5, err_u_t0
    _, err_u_hi, _ = errors(droplet, em.run(droplet[0], STEPS, G, **dict(COMPENSATED, density="exact_rounded")))
    assert err_u_hi > 1.5 * err_u, (err_u_hi, err_u)


@pytest.mark.parametrize("collision", ["bgk", "regularized"])
def test_the_two_fp32_forms_on_the_channel(collision):
    """The channel of the GPU parity tests after 1000 steps: the plain form
    misses the velocity bound (BGK 2.0e-5, regularised 1.7e-5), the
    compensated one meets it (7.7e-6, 6.3e-6); both keep rho and the mass
    within the contract."""
    mask, rho = channel_geometry()
    P = oracle.Problem(mask, G=G, periodic=(True, False), collision=collision, **CHANNEL)
    rho_r, u_r, _ = P.fields(P.run(P.init(rho), STEPS))
    case = (rho, P, rho_r, u_r)
    reg = collision == "regularized"
    err_rho, err_u, drift = errors(case, em.run(rho, STEPS, G, mask=mask, regularized=reg, **CHANNEL, **PLAIN))
    assert err_rho < 1e-5 and np.all(drift < 1e-6), (err_rho, drift)
    assert err_u > 1.2e-5, err_u
    err_rho, err_u, drift = errors(case, em.run(rho, STEPS, G, mask=mask, regularized=reg, **CHANNEL,
                                                **COMPENSATED))
    assert err_rho < 5e-6 and err_u < 1e-5 and np.all(drift < 1e-6), (err_rho, err_u, drift)


# ----------------------------------------------------------------------------
# 16-bit storage: which reference the stored part is shifted by
# ----------------------------------------------------------------------------
def test_16bit_rounding_is_the_formats_own():
    """to16 rounds to nearest with ties to even exactly as numpy's float16
    and torch's bfloat16 conversions do, subnormal FP16 values included."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.normal(0, 1, 20000), rng.normal(0, 1e-4, 20000), rng.normal(0, 1e-7, 20000),
                        np.arange(-500, 500) * 2.0 ** -10 + 2.0 ** -11,
                        np.arange(-500, 500) * 2.0 ** -7 + 2.0 ** -8]).astype(np.float32)
    ref16 = x.astype(np.float16).astype(np.float32)
    np.testing.assert_array_equal(em.to16(x, "fp16").view(np.uint32), ref16.view(np.uint32))
    refb = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(em.to16(x, "bf16").view(np.uint32), refb.view(np.uint32))


@pytest.fixture(scope="module")
def shifted16(droplet):
    """Errors (rho, u) of the droplet after 1000 steps with 16-bit storage,
    FP32 arithmetic and weights summing to 1, for the node shift (FP16,
    BF16) and the destination shift (FP16); the constant shift after 200
    steps."""
    rho0, P, _, _ = droplet
    out = {}
    for fmt, shift in (("fp16", "node"), ("fp16", "destination"), ("bf16", "node")):
        out[fmt, shift] = errors(droplet, em.run16(rho0, STEPS, G, fmt=fmt, shift=shift,
                                                   weight_kind="sum_to_one"))[:2]
    rho_r, u_r, _ = P.fields(P.run(P.init(rho0), 200))
    rho, u, _ = P.fields(em.run16(rho0, 200, G, fmt="fp16", shift="constant", weight_kind="sum_to_one"))
    out["fp16", "constant"] = (np.max(np.abs(rho - rho_r)) / np.max(rho_r), np.max(np.abs(u - u_r)) / np.max(np.abs(u_r)))
    return out


def test_node_shifted_16bit_storage_within_the_gpu_bounds(shifted16):
    """The node shift the library stores (s_i = f*_i - w_i rhohat of the
    storing node): emulated FP16 rho 2.7e-4, u 3.4e-3 and BF16 rho 2.9e-3,
    u 2.8e-2, the errors the GPU shows on the same droplet (FP16 3.4e-4 /
    3.1e-3, BF16 3.2e-3 / 3e-2) and inside the bounds its 1000-step test
    holds it to."""
    r, u = shifted16["fp16", "node"]
    assert r < 5e-4 and u < 8e-3, (r, u)
    r, u = shifted16["bf16", "node"]
    assert r < 2.5e-2 and u < 0.12, (r, u)


def test_destination_shift_is_no_better(shifted16):
    """Shifting each stored part by the density of the node that pulls it
    next (which cancels the force-shifted first-order part at a static
    interface in the continuum) gives larger velocity errors (FP16 6.2e-3
    against 3.4e-3; BF16, not run here, 4.0e-2 against 2.8e-2): the
    interfaces are four nodes wide, far from the continuum limit."""
    assert shifted16["fp16", "destination"][1] > 1.2 * shifted16["fp16", "node"][1]


def test_constant_shift_fails_at_the_interface(shifted16):
    """A shift by each species' mean density leaves the minority species'
    stored part as large as the majority density across the interface:
    percent-level density errors within 200 steps (FP16 1.1 % on rho,
    11 % on u), far above the node shift's after 1000."""
    assert shifted16["fp16", "constant"][0] > 30 * shifted16["fp16", "node"][0]
