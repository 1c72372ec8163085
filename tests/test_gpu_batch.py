"""GPU tests of the batched path: many uneven channels in one launch per step,
and the device-side bisection of the critical body force (Section 3.4)."""
import numpy as np
import pytest

import oracle
from oracle.bisect import bisect_critical
from paper_1601_00918_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

G = -1.79


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    from paper_1601_00918_gb300 import build
    build.build()
    from paper_1601_00918_gb300 import lbm as mod
    mod.library()
    return mod


def channel_instance(lam, periods, h0, amp, slug_len, tau=(1.0, 1.0), rho_wall=(0.3, 0.1), g=0.0):
    nx = int(lam * periods)
    ny = 2 * int(np.ceil(h0 + amp)) + 2
    mask = wl.sinusoidal_channel(nx, ny, h0, amp, float(lam))
    centre = lam * (periods // 2)
    rho = wl.slug(nx, ny, centre - slug_len / 2, centre + slug_len / 2)
    return dict(mask=mask, rho_init=rho, tau=tau, G=G, rho_wall=rho_wall, g=(g, 0.0), periodic=(True, False),
                disp_threshold=lam / 2.0)


def uneven_instances():
    return [channel_instance(32, 3, 6.0, 2.0, 24.0, tau=(1.0, 0.9)),
            channel_instance(48, 3, 9.0, 4.0, 40.0, rho_wall=(0.1, 0.4), g=2e-5),
            channel_instance(100, 3, 12.0, 5.0, 90.0, tau=(0.9, 1.2), g=-1e-5),
            channel_instance(20, 2, 4.0, 1.0, 12.0)]


def test_batch_steps_match_single_grids(lbm):
    """Four channels of different sizes (one narrower than a tile, one with
    a ragged last tile) stepped together agree with each one stepped alone
    through lbm_create / lbm_step (FP64: to rounding)."""
    inst = uneven_instances()
    b = lbm.Batch(inst, precision="fp64")
    try:
        b.step(40)
        got = [b.save(i) for i in range(len(inst))]
        obs = b.observables()
    finally:
        b.close()
    for d, f_b, o in zip(inst, got, obs):
        sim = lbm.Simulation(d["mask"], d["rho_init"], tau=d["tau"], G=d["G"], rho_wall=d["rho_wall"],
                             g=d["g"], periodic=d["periodic"], precision="fp64", variant="simple")
        try:
            sim.step(40)
            f_s = sim.save()
            o_s = sim.observables()
        finally:
            sim.close()
        np.testing.assert_allclose(f_b, f_s, rtol=0, atol=1e-13)
        assert o["step"] == 40
        np.testing.assert_allclose(o["mass"], o_s["mass"], rtol=1e-13)
        np.testing.assert_allclose(o["oil_disp_x"], o_s["oil_disp_x"], rtol=1e-9, atol=1e-13)


def test_batch_regularized_matches_oracle(lbm):
    """Instances may use the regularised collision (Eq. Regualize), each its
    own choice: a mixed batch stepped together matches the FP64 oracle."""
    inst = uneven_instances()[:2]
    inst[0]["collision"] = "regularized"
    inst[0]["tau"] = (1.0, 0.65)
    b = lbm.Batch(inst, precision="fp64")
    try:
        b.step(40)
        got = [b.save(i) for i in range(len(inst))]
    finally:
        b.close()
    for d, f_b in zip(inst, got):
        P = oracle.Problem(d["mask"], tau=d["tau"], G=d["G"], rho_wall=d["rho_wall"], g=d["g"],
                           periodic=d["periodic"], collision=d.get("collision", "bgk"))
        np.testing.assert_allclose(f_b, P.run(P.init(d["rho_init"]), 40), rtol=0, atol=1e-12)


@pytest.mark.parametrize("precision", ["fp32", "fp32c"])
def test_batch_steps_fp32_match_oracle(lbm, precision):
    inst = uneven_instances()[:2]
    b = lbm.Batch(inst, precision=precision)
    try:
        b.step(30)
        got = [b.save(i) for i in range(len(inst))]
    finally:
        b.close()
    for d, f_b in zip(inst, got):
        P = oracle.Problem(d["mask"], tau=d["tau"], G=d["G"], rho_wall=d["rho_wall"], g=d["g"],
                           periodic=d["periodic"])
        f_r = P.run(P.init(d["rho_init"]), 30)
        np.testing.assert_allclose(f_b, f_r, rtol=0, atol=2e-5)


@pytest.mark.parametrize("rows", [None, 1, 3, 8, 64])
@pytest.mark.parametrize("precision,atol", [("fp32", 2e-5), ("fp32c", 2e-5), ("fp16s", 2e-3)])
def test_staged_batch_tiles_match_oracle(lbm, rows, precision, atol, monkeypatch):
    """FP32 and FP16-shifted batches step with the staged (TMA) march over
    tiles of 128 columns x R rows holding fluid: with R chosen by the
    library or pinned (strips of 1, 3, 8 and 64 rows), four uneven channels
    and an all-solid one (a single empty tile) stepped together agree with
    the FP64 oracle; so does a droplet in a box periodic in both directions
    (rows wrap in y inside the march); every instance counts its steps."""
    if rows is None:
        monkeypatch.delenv("GB300LBM_BATCH_ROWS", raising=False)
    else:
        monkeypatch.setenv("GB300LBM_BATCH_ROWS", str(rows))
    inst = uneven_instances()
    inst.append(dict(mask=wl.periodic_box(150, 40), rho_init=wl.droplet(150, 40, 12.0, 70.0, 18.0),
                     tau=(1.0, 1.0), G=G, rho_wall=(0.0, 0.0), g=(1e-5, 0.0), periodic=(True, True),
                     disp_threshold=10.0))
    solid = dict(inst[3], mask=np.ones_like(inst[3]["mask"]))
    inst.append(solid)
    b = lbm.Batch(inst, precision=precision)
    try:
        info = b.kernel_info()
        b.step(30)
        got = [b.save(i) for i in range(len(inst) - 1)]
        obs = b.observables()
    finally:
        b.close()
    assert info["variant"] == "staged"
    if rows is not None:
        assert info["strip_rows"] == rows
    assert 8 <= info["strip_rows"] <= 64 or rows is not None
    assert all(o["step"] == 30 and o["timeout_flag"] == 0 for o in obs)
    assert tuple(obs[-1]["mass"]) == (0.0, 0.0)
    for d, f_b in zip(inst, got):
        P = oracle.Problem(d["mask"], tau=d["tau"], G=d["G"], rho_wall=d["rho_wall"], g=d["g"],
                           periodic=d["periodic"])
        np.testing.assert_allclose(f_b, P.run(P.init(d["rho_init"]), 30), rtol=0, atol=atol)


def test_batch_autotune_keeps_the_state_and_tiling_changes_no_bit(lbm, monkeypatch):
    """The strip-row autotuner steps the batch at create time: afterwards
    the state and the observables are those of creation (step 0, the
    initial populations).  The tiling changes no population: every node's
    density is pulled and summed in the same order in any tile, so 20 steps
    with the timed choice and with strips of 3 rows agree bit for bit; the
    observables are sums reduced tile by tile, so they agree to rounding
    (the oil displacement of these near-static slugs is a difference of
    opposite momenta, ~1e-8 lattice units)."""
    inst = uneven_instances()
    monkeypatch.delenv("GB300LBM_BATCH_ROWS", raising=False)
    a = lbm.Batch(inst, precision="fp32")
    monkeypatch.setenv("GB300LBM_BATCH_ROWS", "3")
    b = lbm.Batch(inst, precision="fp32")
    try:
        assert a.kernel_info()["strip_rows"] != 3
        assert all(o["step"] == 0 and o["oil_disp_x"] == 0.0 for o in a.observables())
        for i, d in enumerate(inst):
            P = oracle.Problem(d["mask"], tau=d["tau"], G=d["G"], rho_wall=d["rho_wall"], g=d["g"],
                               periodic=d["periodic"])
            np.testing.assert_allclose(a.save(i), P.init(d["rho_init"]), rtol=0, atol=1e-6)
        a.step(20)
        b.step(20)
        for i in range(len(inst)):
            np.testing.assert_array_equal(a.save(i), b.save(i))
        oa, ob = a.observables(), b.observables()
        for x, y in zip(oa, ob):
            assert x["step"] == y["step"] == 20
            np.testing.assert_allclose(x["mass"], y["mass"], rtol=1e-6)
            assert abs(x["oil_disp_x"] - y["oil_disp_x"]) < 1e-6
    finally:
        a.close()
        b.close()


def test_batch_kernel_choice(lbm):
    """FP64 batches keep the register-pull march (their step is arithmetic-
    bound); BF16-shifted ones run staged."""
    inst = uneven_instances()[:1]
    for precision, variant in (("fp64", "register-pull"), ("bf16s", "staged")):
        b = lbm.Batch(inst, precision=precision)
        try:
            assert b.kernel_info()["variant"] == variant
        finally:
            b.close()


def gpu_moving(lbm, d, f_eq, t_obs, precision="fp64"):
    """One probe through the single-grid ABI: restart from f_eq at g."""
    def moving(g):
        sim = lbm.Simulation(d["mask"], d["rho_init"], tau=d["tau"], G=d["G"], rho_wall=d["rho_wall"],
                             g=(g, 0.0), periodic=d["periodic"], precision=precision, variant="simple")
        try:
            sim.load(f_eq)
            sim.step(t_obs)
            o = sim.observables(check=False)
        finally:
            sim.close()
        if o["nan_flag"]:
            return None
        return abs(o["oil_disp_x"]) > d["disp_threshold"]
    return moving


def test_device_bisection_follows_the_protocol(lbm):
    """The device bisection (all instances in lockstep, decisions in FP64 on
    the GPU) returns the same brackets as the host statement of the protocol
    driving single-grid probes from the same equilibrated state."""
    inst = [channel_instance(32, 2, 6.0, 3.0, 24.0), channel_instance(40, 2, 7.0, 2.0, 30.0, tau=(1.0, 0.9))]
    t_eq, t_obs = 600, 1500
    g_lo = np.array([2e-5, 2e-5])
    g_hi = np.array([4e-4, 4e-4])
    b = lbm.Batch(inst, precision="fp64")
    try:
        res = b.critical_pressure(g_lo, g_hi, rel_bracket=0.05, t_eq=t_eq, t_obs=t_obs, max_probes=16)
    finally:
        b.close()
    for k, d in enumerate(inst):
        sim = lbm.Simulation(d["mask"], d["rho_init"], tau=d["tau"], G=d["G"], rho_wall=d["rho_wall"],
                             g=(0.0, 0.0), periodic=d["periodic"], precision="fp64", variant="simple")
        try:
            sim.step(t_eq)
            f_eq = sim.save()
        finally:
            sim.close()
        ref = bisect_critical(gpu_moving(lbm, d, f_eq, t_obs), g_lo[k], g_hi[k], rel=0.05, max_probes=16)
        assert res[k]["status"] == ref["status"]
        assert res[k]["probes"] == ref["probes"]
        np.testing.assert_allclose([res[k]["g_lo"], res[k]["g_hi"]], [ref["g_lo"], ref["g_hi"]], rtol=1e-12)


def test_bisection_matches_oracle_bracket(lbm):
    """End to end on a small channel (64 x 20, lambda = 32): the GPU batch
    bisection (FP32) and the FP64 oracle running the same protocol end with
    brackets that overlap or touch (one 5 % bracket)."""
    d = channel_instance(32, 2, 6.0, 3.0, 24.0)
    t_eq, t_obs = 600, 1500
    b = lbm.Batch([d], precision="fp32")
    try:
        res = b.critical_pressure([2e-5], [4e-4], rel_bracket=0.05, t_eq=t_eq, t_obs=t_obs, max_probes=16)[0]
    finally:
        b.close()
    P = oracle.Problem(d["mask"], tau=d["tau"], G=d["G"], rho_wall=d["rho_wall"], g=(0.0, 0.0),
                       periodic=d["periodic"])
    f_eq = P.run(P.init(d["rho_init"]), t_eq)

    def moving(g):
        Pg = oracle.Problem(d["mask"], tau=d["tau"], G=d["G"], rho_wall=d["rho_wall"], g=(g, 0.0),
                            periodic=d["periodic"])
        _, hist = Pg.run(f_eq, t_obs, history=True)
        if hist[:, 4].any():
            return None
        return abs(np.sum(hist[:, 2] / hist[:, 0])) > d["disp_threshold"]

    ref = bisect_critical(moving, 2e-5, 4e-4, rel=0.05, max_probes=16)
    assert res["status"] == 0 and ref["status"] == 0
    assert res["g_lo"] <= ref["g_hi"] * (1 + 1e-12) and ref["g_lo"] <= res["g_hi"] * (1 + 1e-12)


def test_bisection_status_paths(lbm):
    """max_probes reached -> status 1; a bracket below the critical force is
    expanded upwards until g_hi moves."""
    d = channel_instance(32, 2, 6.0, 3.0, 24.0)
    b = lbm.Batch([d, d], precision="fp32")
    try:
        res = b.critical_pressure([2e-5, 1e-6], [4e-4, 2e-6], rel_bracket=1e-6, t_eq=300, t_obs=800,
                                  max_probes=6)
    finally:
        b.close()
    assert res[0]["status"] == 1 and res[0]["probes"] == 6
    assert res[1]["g_hi"] > 2e-6          # expanded


def test_device_wait_gives_up_and_the_context_stays_usable(lbm):
    """Failure handling of the device waits: the bounded mbarrier wait of the
    step kernels, run on a barrier nothing ever completes, gives up within a
    few seconds and the host sees LBM_ETIMEOUT; the CUDA context still works
    (a batch steps normally right after)."""
    rc, sec = lbm.lbm_wait_selftest()
    assert rc == lbm.LBM_ETIMEOUT, (rc, lbm.library().lbm_last_error(None))
    assert 0.05 < sec < 10.0, sec
    b = lbm.Batch([channel_instance(32, 2, 6.0, 3.0, 24.0)], precision="fp32")
    try:
        b.step(10)
        obs = b.observables()
    finally:
        b.close()
    assert obs[0]["step"] == 10 and obs[0]["nan_flag"] == 0 and obs[0]["timeout_flag"] == 0
