"""Host-side checks of the C-ABI library and the input generators (no GPU).

The library is compiled for sm_103a here (nvcc cross-compiles) and loaded;
only calls that fail validation before touching the device are made.
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1601_00918_gb300 import build, lbm, workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbm.library()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lbm[0-9a-z]*_[a-z0-9_]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert {"lbm_create", "lbm_step", "lbm_observables", "lbm_destroy"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert set(lbm.EXPORTS) <= names


def test_workspace_size_formula(lib):
    """Two population buffers with 8 ghost columns a side (pitch = nx + 16
    rounded up to 32), the link words, one fluid-row range per 128 columns,
    parameters, two accumulator and two observable blocks, each 256-aligned."""
    p = lbm.make_params(100, 30, precision="fp32")
    pitch = 128
    buf = 18 * 30 * pitch * 4
    buf = (buf + 255) // 256 * 256
    links = (30 * pitch * 2 + 255) // 256 * 256
    assert lbm.lbm_workspace_size(p) == 2 * buf + links + 256 + 256 + 2 * 256 + 2 * 256
    p = lbm.make_params(113, 30, precision="fp32")          # 113 + 16 > 128: pitch 160
    buf = (18 * 30 * 160 * 4 + 255) // 256 * 256
    links = (30 * 160 * 2 + 255) // 256 * 256
    assert lbm.lbm_workspace_size(p) == 2 * buf + links + 256 + 256 + 2 * 256 + 2 * 256
    assert lbm.lbm_workspace_size(lbm.make_params(100, 30, precision="fp16s")) < \
        lbm.lbm_workspace_size(p)


def test_too_large_grid_rejected(lib):
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_workspace_size(lbm.make_params(1 << 16, 1 << 12))
    assert e.value.code == lbm.LBM_EINVAL


@pytest.mark.parametrize("bad", [
    dict(tau=(0.5, 1.0)),
    dict(tau=(1.0, 0.3)),
    dict(eq_order=4),
    dict(precision=9),
    dict(periodic=(True, False)),            # open in y without solid rows
    dict(variant=6),                         # 5 = persistent is the last kernel
    dict(collision=2),
])
def test_create_rejects_bad_parameters(lib, bad):
    kw = dict(nx=16, ny=8)
    p = lbm.make_params(**kw, **bad)
    mask = wl.periodic_box(16, 8)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_create(mask, wl.uniform(16, 8, 1.0, 0.1), p)
    assert e.value.code == lbm.LBM_EINVAL
    assert lbm.lbm_last_error(None)


def test_create_with_bad_densities_fails_with_a_status(lib):
    """The initial densities are checked on the device after the upload
    (LBM_EINVAL; the GPU suite tests that).  Without a device the call must
    still fail with a status and a message, not crash."""
    import torch
    p = lbm.make_params(16, 8)
    for rho in (wl.uniform(16, 8, 1.0, 0.1), wl.uniform(16, 8, 0.0, 0.0)):
        rho[0, 3, 3] = -0.1
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create(wl.periodic_box(16, 8), rho, p)
        if torch.cuda.is_available():
            assert e.value.code == lbm.LBM_EINVAL
        else:
            assert e.value.code in (lbm.LBM_ENOMEM, lbm.LBM_ECUDA)
        assert lbm.lbm_last_error(None)


@pytest.mark.parametrize("bad", ["negative", "nan", "empty", "tau", "collision", "open_y"])
def test_batch_create_checks_every_instance_on_the_host(lib, bad):
    """lbm_batch_create validates each instance before touching the device:
    the densities at fluid nodes (finite, >= 0, positive total), tau > 1/2,
    the collision option and solid boundary lines of an open direction."""
    mask = wl.sinusoidal_channel(64, 24, 6.0, 2.0, 32.0)
    good = dict(mask=mask, rho_init=wl.slug(64, 24, 16.0, 40.0), tau=(1.0, 1.0), G=-1.79,
                periodic=(True, False), disp_threshold=16.0)
    d = dict(good, rho_init=good["rho_init"].copy())
    y, x = np.argwhere(mask == 0)[5]
    if bad == "negative":
        d["rho_init"][1, y, x] = -1e-3
    elif bad == "nan":
        d["rho_init"][0, y, x] = np.nan
    elif bad == "empty":
        d["rho_init"][:, y, x] = 0.0
    elif bad == "tau":
        d["tau"] = (0.5, 1.0)
    elif bad == "collision":
        d["collision"] = 2
    else:
        d["mask"] = np.zeros_like(mask)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_create([good, d])
    assert e.value.code == lbm.LBM_EINVAL
    assert "instance 1" in str(e.value)


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.lbm_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_observables(None, None) == lbm.LBM_EINVAL
    lib.lbm_destroy(None)


@pytest.mark.parametrize("bad,needle", [
    (dict(precision="fp64"), "LBM_FP32"),
    (dict(nx=2048, ny=1025), "2097152"),
    (dict(nx=0, ny=8), "2097152"),
    (dict(eq_order=4), "eq_order"),
    (dict(collision=2), "collision"),
    (dict(tau=(0.5, 1.0)), "tau"),
    (dict(tau=(1.0, float("inf"))), "tau"),
    (dict(G=float("nan")), "finite"),
    (dict(g=(float("inf"), 0.0)), "finite"),
    (dict(rho_wall=(0.1, float("nan"))), "finite"),
])
def test_noalloc_step_checks_its_arguments_on_the_host(lib, bad, needle):
    """The allocation-free step rejects every argument it cannot step with
    (LBM_EINVAL and a message naming it) before it touches the device; the
    pointers here are host buffers it never reads."""
    kw = dict(nx=16, ny=8)
    kw.update(bad)
    p = lbm.make_params(**kw)
    buf = (ctypes.c_float * 16)()
    mask = (ctypes.c_uint8 * 16)()
    rc = lib.lbm_step_noalloc(ctypes.addressof(mask), ctypes.addressof(buf), ctypes.addressof(buf), None,
                              ctypes.byref(p))
    assert rc == lbm.LBM_EINVAL
    assert needle in lbm.lbm_last_error(None)


def test_every_handle_call_rejects_a_null_handle(lib):
    """Each call that takes a handle returns LBM_EINVAL for NULL (as the
    header states) before it touches a device, and every destroy ignores
    NULL; the error text of the NULL handle is readable afterwards."""
    d = ctypes.c_double
    calls = [
        lambda: lib.lbm_get_fields(None, None, None, None),
        lambda: lib.lbm_set_body_force(None, d(0.0), d(0.0)),
        lambda: lib.lbm_save(None, None),
        lambda: lib.lbm_load(None, None),
        lambda: lib.lbm_kernel_info(None, None),
        lambda: lib.lbm_batch_step(None, ctypes.c_int64(1)),
        lambda: lib.lbm_batch_observables(None, None),
        lambda: lib.lbm_batch_kernel_info(None, None),
        lambda: lib.lbm_batch_set_body_force(None, None),
        lambda: lib.lbm_batch_save(None, 0, None),
        lambda: lib.lbm_critical_pressure_batch(None, None, None, None, None),
        lambda: lib.lbm3d_step(None, ctypes.c_int64(1)),
        lambda: lib.lbm3d_observables(None, None),
        lambda: lib.lbm3d_get_fields(None, None, None),
        lambda: lib.lbm3d_save(None, None),
        lambda: lib.lbm3d_load(None, None),
        lambda: lib.lbm_mlp_params(None, None, None),
        lambda: lib.lbm_mlp_forward(None, None, 1, None),
        lambda: lib.lbm_mlp_loss_grad(None, None, None, 1, None, None),
        lambda: lib.lbm_mlp_adam(None, ctypes.c_float(1e-3)),
        lambda: lib.lbm_critical_pressure_channels(None, 1, None, None),
        lambda: lib.lbm_step_noalloc(None, None, None, None, None),
    ]
    for k, call in enumerate(calls):
        assert call() == lbm.LBM_EINVAL, k
    lib.lbm_batch_destroy(None)
    lib.lbm3d_destroy(None)
    lib.lbm_mlp_destroy(None)
    for fn in (lib.lbm_last_error, lib.lbm_batch_last_error, lib.lbm3d_last_error):
        fn.restype = ctypes.c_char_p
        assert isinstance(fn(None), bytes)


# ----------------------------------------------------------------------------
# input generators
# ----------------------------------------------------------------------------
def test_sinusoidal_channel_rows():
    """1024 x 146 channel, h(x) = 48 - 24 cos(2 pi x / 256), y_c = 72.5: rows
    1..144 are fluid at a bulge, rows 49..96 (48 rows) at a neck."""
    w = wl.sinusoidal_slug(scale=1)
    assert w.mask.shape == (146, 1024)
    bulge = np.nonzero(w.mask[:, 128] == 0)[0]
    neck = np.nonzero(w.mask[:, 0] == 0)[0]
    assert (bulge.min(), bulge.max()) == (1, 144)
    assert (neck.min(), neck.max(), len(neck)) == (49, 96, 48)
    assert np.all(w.mask[0] == 1) and np.all(w.mask[-1] == 1)
    big = wl.sinusoidal_slug(scale=8)
    assert big.mask.shape == (1170, 8192)
    rows = np.nonzero(big.mask[:, 1024] == 0)[0]
    assert (rows.min(), rows.max()) == (9, 1160)


def test_droplet_and_slug_profiles():
    """Section 3.1's droplet: 1.0 inside, 0.03 outside, the total 1.03
    everywhere, the interface a tanh of width 2 centred on the radius (half
    way at r = R, a fraction (1 - tanh 1) / 2 of the jump one width out);
    a slug fills the channel between its ends."""
    r = wl.droplet(64, 64, 10.0, 32.0, 32.0)
    assert r[0, 32, 32] == pytest.approx(1.0, abs=1e-3)
    assert r[0, 0, 0] == pytest.approx(0.03, abs=1e-6)
    np.testing.assert_allclose(r.sum(axis=0), 1.03)
    assert r[0, 32, 42] == pytest.approx(0.515, abs=1e-12)                  # r = R
    assert r[0, 32, 44] == pytest.approx(0.03 + 0.97 * (1 - np.tanh(1.0)) / 2, abs=1e-12)   # r = R + 2
    s = wl.slug(100, 10, 30.0, 70.0)
    assert s[0, 5, 50] == pytest.approx(1.0, abs=1e-6)
    assert s[1, 5, 5] == pytest.approx(1.0, abs=1e-6)


def test_sweep_specs_are_seeded():
    a = wl.sweep_specs(16, seed=3)
    b = wl.sweep_specs(16, seed=3)
    assert a == b
    for s in a:
        assert s.lam in (128, 192, 256, 384, 512)
        assert 0.2 <= s.amp_ratio <= 0.6 and 20 <= s.theta_deg <= 160
        assert 0.2 <= s.visc_ratio <= 10
        w = wl.channel_instance(s)
        assert w.mask.shape == (s.ny, s.nx)


@pytest.mark.parametrize("bad,needle", [
    (dict(nz=0), "nx, ny, nz"),
    (dict(precision=2), "precision"),
    (dict(eq_order=1), "eq_order"),
    (dict(collision=3), "collision"),
    (dict(tau=(1.0, 0.5)), "tau"),
    (dict(G=float("inf")), "finite"),
    (dict(g=(0.0, 0.0, float("nan"))), "finite"),
    (dict(periodic=(1, 1, 0)), "boundary plane"),
    (dict(rho_bad=-0.1), "rho_init"),
    (dict(rho_bad=float("nan")), "rho_init"),
])
def test_d3q19_create_checks_its_arguments_on_the_host(lib, bad, needle):
    """lbm3d_create rejects sizes, parameters, an open direction with fluid
    on its boundary planes and bad initial densities with LBM_EINVAL and a
    message, on the host, before any device work."""
    from paper_1601_00918_gb300.lbm import Params3
    kw = dict(nx=6, ny=5, nz=4, precision=0, eq_order=3, collision=0, tau=(1.0, 1.0), G=-1.79,
              g=(0.0, 0.0, 0.0), periodic=(1, 1, 1))
    rho_bad = bad.pop("rho_bad", None)
    kw.update(bad)
    n = 6 * 5 * 4
    mask = np.zeros(n, np.uint8)
    rho = np.full(2 * n, 0.5)
    if rho_bad is not None:
        rho[7] = rho_bad
    p = Params3(kw["nx"], kw["ny"], kw["nz"], (ctypes.c_int32 * 3)(*kw["periodic"]),
                (ctypes.c_double * 2)(*kw["tau"]), kw["G"], (ctypes.c_double * 2)(0.0, 0.0),
                (ctypes.c_double * 3)(*kw["g"]), kw["precision"], kw["eq_order"], kw["collision"], None)
    h = ctypes.c_void_p()
    rc = lib.lbm3d_create(mask.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                          rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(p), ctypes.byref(h))
    assert rc == lbm.LBM_EINVAL and not h.value
    lib.lbm3d_last_error.restype = ctypes.c_char_p
    assert needle in lib.lbm3d_last_error(None).decode()


def _shape(lib, **kw):
    spec = dict(lam=64, amp_ratio=0.5, slug_len_over_lambda=1.5, theta_deg=60.0, visc_ratio=1.0, n_periods=0,
                n_slugs=0)
    spec.update(kw)
    cs = lbm.ChannelSpec(spec["lam"], spec["amp_ratio"], spec["slug_len_over_lambda"], spec["theta_deg"],
                         spec["visc_ratio"], spec["n_periods"], spec["n_slugs"])
    nx, ny = ctypes.c_int32(), ctypes.c_int32()
    rc = lib.lbm_channel_shape(ctypes.byref(cs), ctypes.byref(nx), ctypes.byref(ny))
    return rc, nx.value, ny.value


@pytest.mark.parametrize("bad", [
    dict(lam=4), dict(lam=70000), dict(n_periods=1), dict(n_periods=65), dict(n_periods=-2),
    dict(n_periods=4, n_slugs=3), dict(n_slugs=-1), dict(amp_ratio=-0.1), dict(amp_ratio=0.96),
    dict(amp_ratio=float("nan")), dict(slug_len_over_lambda=0.0), dict(slug_len_over_lambda=3.01),
    dict(n_slugs=2, slug_len_over_lambda=1.76), dict(theta_deg=0.0), dict(theta_deg=180.0),
    dict(visc_ratio=0.0), dict(visc_ratio=float("inf")),
])
def test_channel_spec_ranges(lib, bad):
    """A channel description outside the ranges the header states is
    rejected with LBM_EINVAL (host, no GPU)."""
    assert _shape(lib, **bad)[0] == lbm.LBM_EINVAL


def test_channel_spec_defaults_and_limits(lib):
    """0 periods and 0 slugs select 4 and 1; the longest slugs the header
    admits (n_periods - 1 wavelengths for one slug, n_periods / n_slugs - 1/4
    for several) are accepted; the lattice is lambda n_periods by
    2 ceil(h0 + A) + 2 with h0 = 0.1875 lambda."""
    assert _shape(lib) == (lbm.LBM_OK, 256, 2 * 18 + 2)
    assert _shape(lib, n_periods=4, n_slugs=1)[1:] == (256, 38)
    assert _shape(lib, slug_len_over_lambda=3.0)[0] == lbm.LBM_OK
    assert _shape(lib, n_slugs=2, slug_len_over_lambda=1.75)[0] == lbm.LBM_OK
    assert _shape(lib, lam=128, n_periods=6, amp_ratio=0.2)[1:] == (768, 2 * 29 + 2)


def test_binding_checks_host_array_shapes(lib):
    """The binding refuses host arrays whose shape does not match what the C
    call will read (it reads both species' planes, or n table entries),
    instead of letting the call read past their end."""
    good = np.ones((2, 12, 20))
    with pytest.raises(ValueError):
        lbm.lbm_contact_angle(np.ones((1, 12, 20)), 1, 10)
    with pytest.raises(ValueError):
        lbm.lbm_meniscus_angles(np.ones((12, 20)), 4.0, 1.0, 20.0)
    with pytest.raises(ValueError):
        lbm.lbm_slug_area(good, np.zeros((12, 21), np.uint8))
    with pytest.raises(ValueError):
        lbm.lbm_wall_potentials(np.array([-0.4, 0.0, 0.4]), np.array([135.0, 90.0]), 60.0)
    assert lbm.lbm_slug_area(good * np.array([1.0, 0.0])[:, None, None], np.zeros((12, 20), np.uint8))[0] == 240
    inst = dict(mask=wl.periodic_box(8, 6), rho_init=np.ones((2, 6, 9)))
    with pytest.raises(ValueError):
        lbm.lbm_batch_create([inst])
    with pytest.raises(ValueError):
        lbm.lbm_load(None, np.zeros((2, 9, 6, 7)), 8, 6)
    with pytest.raises(ValueError):
        lbm.lbm_critical_pressure_batch(None, [1e-5, 2e-5], [4e-5, 8e-5], n=3)
    with pytest.raises(ValueError):
        lbm.lbm_critical_pressure_batch(None, [1e-5, 2e-5], [4e-5])
    with pytest.raises(ValueError):
        lbm.lbm_batch_set_body_force(None, [1e-5], n=2)


def test_surrogate_binding_checks_shapes(lib):
    """Parameter vectors, features and targets are checked against what the
    lbm_mlp_* calls read before any device work (a handle-less object is
    enough to reach the checks)."""
    s = object.__new__(lbm.Surrogate)
    s.h = None
    with pytest.raises(ValueError):
        s.set_params(np.zeros(lbm.MLP_PARAMS - 1, np.float32))
    with pytest.raises(ValueError):
        s.forward(np.zeros((4, 4), np.float32))
    with pytest.raises(ValueError):
        s.loss_grad(np.zeros((4, 5), np.float32), np.zeros(3, np.float32))
    with pytest.raises(ValueError):
        s.train(np.zeros((0, 5), np.float32), np.zeros(0, np.float32), 1)
    with pytest.raises(ValueError):
        lbm.Surrogate(params=np.zeros(10, np.float32))


def test_sinusoidal_tube_cross_sections():
    """The paper's tube (Section 3.4) as the input module builds it: every
    cross section is a lattice disc about the centre line, symmetric under
    the swap and the reflections of y and z, whose node count N lies within
    the bounds a disc of radius r = h(x) = h0 - A cos(2 pi x / lam) fixes,
    pi (r - sqrt(2)/2)^2 <= N <= pi (r + sqrt(2)/2)^2 (the unit squares of
    its nodes lie inside the disc of radius r + sqrt(2)/2 and cover the one
    of radius r - sqrt(2)/2); the narrowest section is at x = 0 and the
    widest at lam / 2; the mask repeats with the wavelength; the boundary
    planes are solid."""
    nx, n, h0, amp, lam = 96, 22, 8.0, 3.0, 48.0
    m = wl.sinusoidal_tube(nx, n, h0, amp, lam)
    assert m.shape == (n, n, nx)
    fluid = (m == 0)
    counts = fluid.sum(axis=(0, 1))
    for x in range(nx):
        sl = fluid[:, :, x]
        assert np.array_equal(sl, sl.T) and np.array_equal(sl, sl[::-1]) and np.array_equal(sl, sl[:, ::-1])
        r = h0 - amp * np.cos(2 * np.pi * x / lam)
        assert np.pi * (r - 0.5 ** 0.5) ** 2 <= counts[x] <= np.pi * (r + 0.5 ** 0.5) ** 2, (x, counts[x], r)
    assert counts[0] == counts.min() and counts[int(lam) // 2] == counts.max()
    assert np.array_equal(m[:, :, :int(lam)], m[:, :, int(lam):2 * int(lam)])
    assert m[0].all() and m[-1].all() and m[:, 0].all() and m[:, -1].all()


def test_layered_channel_rows():
    """The two-component Hagen-Poiseuille set-up (Section 3.2): a straight
    channel of 64 fluid rows between two solid rows, 256 long; rows 1-12 and
    53-64 hold the wetting species, rows 13-52 the core species (sharp
    interfaces), with either species in the core."""
    m = wl.straight_channel(256, 64)
    assert m.shape == (66, 256) and m[0].all() and m[65].all() and not m[1:65].any()
    for core in (0, 1):
        r = wl.layered_channel(256, 64, 12, core_species=core)
        assert r.shape == (2, 66, 256)
        rows_core = np.nonzero(r[core, :, 0] == r[core].max())[0]
        assert rows_core.min() == 13 and rows_core.max() == 52 and len(rows_core) == 40
        assert np.all(r[1 - core, 1:13] == r[1 - core].max()) and np.all(r[1 - core, 53:65] == r[1 - core].max())
        np.testing.assert_allclose(r.sum(axis=0), r.sum(axis=0)[0, 0])      # total density uniform
