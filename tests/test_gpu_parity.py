"""GPU parity: liblbm's kernels against the FP64 CPU oracle, through the C ABI.

* FP64 reference kernels: bit-identical distributions (np.array_equal) to the
  oracle, which evaluates the step in the same canonical order.
* FP32 fused kernel: max relative density error <= 1e-4 after 1000 steps on
  the 400 x 200 single-droplet workload (the FP32 tolerance of the target),
  and on small ragged / variant grids after a few steps.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1501_05430_gb300 import inputs as I
from paper_1501_05430_gb300 import lbm as L

from helpers import Case, Pair, droplet_pair

pytestmark = pytest.mark.gpu

REF, FUSED = L.LBM_KERNEL_REFERENCE, L.LBM_KERNEL_FUSED


def _rel(a, b, mask=None):
    d = np.abs(a - b) / np.maximum(np.abs(b), 1e-30)
    return d[mask].max() if mask is not None else d.max()


def _fluid(ny, walls=True):
    m = np.ones(ny, bool)
    if walls:
        m[0] = m[-1] = False
    return m


# ---------------------------------------------------------------------------
# FP64: bit-exact
# ---------------------------------------------------------------------------

def test_fp64_plain_workload_bit_exact():
    """100 x 60 droplet, CS T/Tc = 0.8, tau = 1, theta = 90 deg: identical f
    after 1, 10 and 2000 steps; mass conserved to 1e-13."""
    w = I.plain_fp64()
    p = droplet_pair(w, precision=64, kernel=REF)
    assert np.array_equal(p.gpu.f(), p.orc.get_f())
    m0 = p.orc.mass()
    done = 0
    for n in (1, 9, 1990):
        assert p.step(n) == 0
        done += n
        fg, fo = p.gpu.f(), p.orc.get_f()
        assert np.array_equal(fg, fo), f"first mismatch after {done} steps: max |d| = {np.abs(fg - fo).max()}"
    assert abs(p.gpu.mass() - m0) / m0 < 5e-13
    assert p.gpu.status() == 0
    p.close()


VARIANTS = {
    "geometric_random_theta": dict(theta="random"),
    "geometric_eq19_only": dict(theta="random", n_iter=0),
    "geometric_8_iterations": dict(theta="random", n_iter=8),
    "martys_chen": dict(wetting=1, G_w=-0.2),
    "periodic_box": dict(walls=False),
    "piecewise_eos_ratio10": dict(eos="pw", pw=(0.25, -0.02, 0.3, 1.1216073327407194, 9.540106186999981)),
    "mrt_rates_kappa": dict(rates=dict(s_e=0.8, s_eps=0.9, s_j=1.0, s_q=1.1), kappa=0.9, A=-0.3),
    "low_T": dict(t_over_tc=0.5, tau=0.6, rates=dict(s_e=0.8, s_eps=0.8, s_j=1.0, s_q=1.1)),
    # the remaining (collision, wetting, EOS) combinations the fused kernel is
    # specialised on: general rates with Martys-Chen, and the piecewise EOS with
    # general rates and with Martys-Chen (unit and general rates)
    "martys_chen_mrt_rates": dict(wetting=1, G_w=-0.2, rates=dict(s_e=0.8, s_eps=0.9, s_j=1.0, s_q=1.1)),
    "piecewise_mrt_rates": dict(eos="pw", pw=(0.25, -0.02, 0.3, 1.1216073327407194, 9.540106186999981),
                                rates=dict(s_e=0.8, s_eps=0.9, s_j=1.0, s_q=1.1)),
    "piecewise_martys_chen": dict(eos="pw", pw=(0.25, -0.02, 0.3, 1.1216073327407194, 9.540106186999981),
                                  wetting=1, G_w=-0.1),
    "piecewise_martys_chen_tau08": dict(eos="pw", pw=(0.25, -0.02, 0.3, 1.1216073327407194, 9.540106186999981),
                                        wetting=1, G_w=-0.1, tau=0.8),
}


def _variant_pair(name, nx, ny, precision, kernel, seed=5):
    kw = dict(VARIANTS[name])
    rng = np.random.default_rng(seed)
    if kw.get("theta") == "random":
        kw["theta"] = rng.uniform(np.deg2rad(20), np.deg2rad(160), (ny, nx))
    p = Pair(nx, ny, precision=precision, kernel=kernel, **kw)
    walls = kw.get("walls", True)
    drops = [(nx * 0.3, ny * 0.35, 0), (nx * 0.75, ny * 0.3, 1)] if walls else [(nx * 0.4, ny * 0.25, ny * 0.5)]
    rho = I.droplet_field(nx, ny, drops, p.rho_v, p.rho_l)
    p.set_f(I.random_distributions(rho, seed, walls=walls))
    return p, walls


@pytest.mark.parametrize("nx,ny", [(28, 16), (4, 5)])
@pytest.mark.parametrize("name", list(VARIANTS))
def test_fp64_variants_bit_exact(name, nx, ny):
    """Every model variant, and the smallest grid the library takes (4 x 5:
    three fluid rows, both ghost rules reading row 2)."""
    p, walls = _variant_pair(name, nx, ny, 64, REF)
    for _ in range(3):
        assert p.step(2) == 0
        assert np.array_equal(p.gpu.f(), p.orc.get_f())
    p.close()


@pytest.mark.parametrize("name", ["geometric_random_theta", "martys_chen", "periodic_box", "piecewise_eos_ratio10"])
def test_fp64_fields_bit_exact(name):
    """rho, psi, U (ghost rows included), force and Eq. 17 tensor."""
    p, walls = _variant_pair(name, 20, 12, 64, REF, seed=9)
    p.step(1)
    g, o = p.gpu.fields(), p.orc.fields()
    for k in ("rho", "psi", "U", "Fx", "Fy", "Qxx", "Qyy", "Qxy"):
        assert np.array_equal(g[k], o[k]), k
    ux, uy = p.gpu.u()
    _, oux, ouy = p.orc.macro()
    assert np.array_equal(ux, oux) and np.array_equal(uy, ouy)
    p.close()


# ---------------------------------------------------------------------------
# FP32 fused kernel
# ---------------------------------------------------------------------------

def test_fp32_fused_single_droplet_1000_steps():
    """400 x 200, CS T/Tc = 0.6, tau = 0.8, theta = 60 deg: max relative density
    error <= 1e-4 after 1000 steps."""
    w = I.single_droplet(60.0)
    p = droplet_pair(w, precision=32, kernel=FUSED)
    assert p.gpu.info.kernel_in_use == FUSED
    assert p.step(1000) == 0
    rg, ro = p.gpu.rho(), p.orc.rho()
    fl = _fluid(w.ny)
    err = _rel(rg, ro, np.broadcast_to(fl[:, None], rg.shape))
    assert err <= 1e-4, err
    assert p.gpu.status() == 0
    p.close()


@pytest.mark.parametrize("nx,ny", [(100, 40), (260, 24), (8, 9), (132, 7), (4, 5), (800, 10)])
@pytest.mark.parametrize("name", list(VARIANTS))
def test_fp32_fused_variants(name, nx, ny):
    """Ragged strips (nx not a multiple of 128), tiny grids down to the
    smallest the library takes (4 x 5: one 4-column strip whose halo boxes
    wrap onto itself), a strip away from the x wrap (800 wide: the middle
    strip's interior rows take the single-address store path, in a walled and
    a fully periodic box) and every model variant: FP32 fused vs FP64 oracle
    after 12 steps."""
    p, walls = _variant_pair(name, nx, ny, 32, FUSED, seed=nx + ny)
    assert p.gpu.info.kernel_in_use == FUSED
    assert p.step(12) == 0
    rg, ro = p.gpu.rho(), p.orc.rho()
    fl = np.broadcast_to(_fluid(ny, walls)[:, None], rg.shape)
    assert _rel(rg, ro, fl) < 2e-5
    fg, fo = p.gpu.f(), p.orc.get_f()
    scale = np.abs(fo).max()
    assert np.abs(fg - fo).max() < 2e-5 * scale
    p.close()


def test_fp32_fused_matches_fp32_reference_kernels():
    w = I.single_droplet(120.0)
    a = droplet_pair(w, precision=32, kernel=FUSED)
    b = droplet_pair(w, precision=32, kernel=REF)
    a.gpu.step(50)
    b.gpu.step(50)
    assert _rel(a.gpu.rho(), b.gpu.rho(), np.broadcast_to(_fluid(w.ny)[:, None], (w.ny, w.nx))) < 1e-5
    a.close()
    b.close()


@pytest.mark.parametrize("recipe", ["throughput_cs", "throughput"])
def test_fp32_fused_full_size_throughput_workload(recipe):
    """The two 4096 x 2048 benchmark workloads (Carnahan-Starling with MRT
    rates: the general-rate kernel; Table 1 with all rates 1: the unit-rate
    kernel) in the benchmark's launch configuration: every node against the
    oracle after 2 steps."""
    w = getattr(I, recipe)()
    p = droplet_pair(w, precision=32, kernel=FUSED)
    assert p.gpu.info.kernel_in_use == L.LBM_KERNEL_FUSED
    assert (w.tau == 1.0 and not w.rates) == (recipe == "throughput")  # unit rates only for Table 1
    before = p.gpu.launches()
    assert p.step(2) == 0
    assert p.gpu.launches() - before == 2
    rg, ro = p.gpu.rho(), p.orc.rho()
    fl = np.broadcast_to(_fluid(w.ny)[:, None], rg.shape)
    assert _rel(rg, ro, fl) < 1e-5
    p.close()


@pytest.mark.parametrize("kernel", [FUSED, REF])
def test_zero_steps_change_nothing(kernel):
    """lbm_step(ctx, 0) launches nothing and leaves the state as it was."""
    p, _ = _variant_pair("geometric_random_theta", 16, 9, 32, kernel)
    f0, l0 = p.gpu.f(), p.gpu.launches()
    p.gpu.step(0)
    assert p.gpu.launches() == l0 and p.gpu.info.steps_done == 0
    assert np.array_equal(p.gpu.f(), f0)
    p.close()


@pytest.mark.parametrize("recipe", ["throughput_cs", "throughput"])
def test_fp32_fused_at_the_32_bit_offset_limit(recipe):
    """The largest grid the fused kernel takes (9 nx ny just below 2^31, where
    its 32-bit element offsets end): 32768 x 7281, 17 GB of distributions,
    with each benchmark recipe (general-rate and unit-rate kernels).  The
    initial state and the wall angles repeat every 256 columns, so after 2
    steps every 256-column window equals the oracle run on a 256-wide periodic
    domain (x translation symmetry holds at any size); three windows are
    compared node by node."""
    tile, reps, ny = 256, 128, 7281
    nx = tile * reps
    assert 9 * nx * ny < 2 ** 31 <= 9 * nx * (ny + 1)
    w = getattr(I, recipe)(nx=tile, ny=ny)
    c = Case(tile, ny, t_over_tc=w.t_over_tc, tau=w.tau, theta=w.theta, rates=w.rates, precision=32,
             eos=w.eos, A=w.A, kappa=w.kappa, kernel=FUSED)
    rho_tile = I.droplet_field(tile, ny, w.droplets, c.rho_v, c.rho_l, w.width)
    c.orc.set_rho(rho_tile)
    assert c.orc.step(2) == 0
    ro = c.orc.rho()
    g = L.Lbm(nx, ny, c.geos, c.T, c.tau, theta=np.tile(c.theta, (1, reps)), params=c.params, torch_state=False)
    try:
        assert g.info.kernel_in_use == FUSED
        g.set_rho(np.tile(rho_tile, (1, reps)))
        g.step(2)
        assert g.status() == 0
        rg = g.rho()
    finally:
        g.close()
        c.orc.close()
    fl = np.broadcast_to(_fluid(ny)[:, None], ro.shape)
    for k in (0, reps // 2, reps - 1):
        win = rg[:, k * tile:(k + 1) * tile]
        assert _rel(win, ro, fl) < 1e-5, k


# ---------------------------------------------------------------------------
# measurement, reductions, checkpoints, errors
# ---------------------------------------------------------------------------

def _cap(nx, ny, R, theta, rv, rl, wall=0, xc=None):
    xc = nx / 2 - 0.4 if xc is None else xc
    base = 1.0 if wall == 0 else ny - 2.0
    yc = base - R * math.cos(theta) if wall == 0 else base + R * math.cos(theta)
    return I.droplet_field(nx, ny, [(xc, R, yc)], rv, rl)


@pytest.mark.parametrize("theta_deg", [30, 90, 150])
@pytest.mark.parametrize("wall", [0, 1])
def test_contact_angle_matches_oracle_measurement(theta_deg, wall):
    # the measurement kernel's arithmetic bit for bit: both sides interpolate
    # the same contour (the oracle's rho_mid), then the library's own contour
    p = Pair(240, 200, precision=64, kernel=REF, oracle_bounds=True)
    rho = _cap(240, 200, 40.0, math.radians(theta_deg), p.rho_v, p.rho_l, wall)
    p.set_rho(rho)
    th, H, L_ = p.gpu.contact_angle(wall, 20, 220)
    assert np.array_equal(p.gpu.rho(), p.orc.rho())
    ot, oH, oL, _ = O.contact_angle_field(p.orc.rho(), wall, 20, 220, p.rho_mid)
    assert th == pytest.approx(ot, rel=1e-13) and H == oH and L_ == oL
    with L.Lbm(240, 200, p.geos, p.T, p.tau, params=L.lbm_params_default(precision=64), torch_state=False) as own:
        assert own.info.rho_mid == pytest.approx(p.rho_mid, rel=1e-12)
        own.set_rho(rho)
        th2, H2, L2 = own.contact_angle(wall, 20, 220)
        assert th2 == pytest.approx(ot, rel=1e-10) and H2 == pytest.approx(oH, rel=1e-10)
        assert L2 == pytest.approx(oL, rel=1e-10)
    assert abs(math.degrees(th) - theta_deg) < 0.6
    with pytest.raises(L.LbmError) as e:
        p.gpu.contact_angle(wall, 0, 30)
    assert e.value.status == L.LBM_ENOCONTACT
    p.close()


def test_mass_and_max_speed_match_oracle():
    p, _ = _variant_pair("geometric_random_theta", 64, 32, 64, REF, seed=3)
    p.step(5)
    assert p.gpu.mass() == pytest.approx(p.orc.mass(), rel=1e-14)
    _, ux, uy = p.orc.macro()
    assert p.gpu.max_speed() == pytest.approx(np.hypot(ux, uy)[1:-1].max(), rel=1e-14)
    p.close()


def test_fp32_mass_drift_small():
    w = I.single_droplet(60.0)
    p = droplet_pair(w, precision=32, kernel=FUSED)
    m0 = p.gpu.mass()
    p.gpu.step(2000)
    assert abs(p.gpu.mass() - m0) / m0 < 1e-5
    p.close()


def test_init_droplets_matches_input_recipe():
    w = I.throughput(nx=512, ny=256, per_wall=4)
    p = Pair(w.nx, w.ny, t_over_tc=0.5, precision=64, kernel=REF)
    xc = [d[0] for d in w.droplets]
    r = [d[1] for d in w.droplets]
    wall = [d[2] for d in w.droplets]
    p.gpu.init_droplets(xc, r, wall, 3.0)
    ref = I.droplet_field(w.nx, w.ny, w.droplets, p.rho_v, p.rho_l)
    got = p.gpu.rho()
    assert np.allclose(got[1:-1], ref[1:-1], rtol=1e-13, atol=0)
    p.close()


@pytest.mark.parametrize("precision,kernel", [(64, REF), (32, FUSED)])
def test_checkpoint_resume_is_bitwise(precision, kernel):
    w = I.single_droplet(45.0)
    a = droplet_pair(w, precision=precision, kernel=kernel)
    a.gpu.step(20)
    img = a.gpu.save()
    a.gpu.step(20)
    b = droplet_pair(w, precision=precision, kernel=kernel)
    b.gpu.load(img)
    b.gpu.step(20)
    assert np.array_equal(a.gpu.f(), b.gpu.f())
    assert b.gpu.info.steps_done == 40
    a.close()
    b.close()


def test_invalid_arguments():
    eos = L.carnahan_starling()
    T = 0.8 * L.lbm_eos_critical(eos)[0]
    for args in [(3, 10, eos, T, 1.0), (10, 4, eos, T, 1.0), (10, 10, eos, T, 0.5), (10, 10, eos, 1.0, 1.0)]:
        with pytest.raises(L.LbmError) as e:
            L.lbm_create(*args)
        assert e.value.status == L.LBM_EINVAL
    mask = np.zeros((10, 12), np.uint8)
    mask[0] = 1  # one wall only
    import ctypes
    out = ctypes.c_void_p()
    st = L.load().lbm_create(12, 10, ctypes.byref(eos), T, 1.0, None, mask.ctypes.data_as(ctypes.c_void_p), None,
                             None, ctypes.byref(out))
    assert st == L.LBM_EUNSUPPORTED
    p64 = L.lbm_params_default(precision=64, kernel=FUSED)
    with pytest.raises(L.LbmError) as e:
        L.lbm_create(16, 10, eos, T, 1.0, params=p64)
    assert e.value.status == L.LBM_EUNSUPPORTED
    ctx = L.lbm_create(16, 10, eos, T, 1.0)
    rho = np.full((10, 16), 0.2)
    rho[0, 3] = rho[9, 5] = -1.0  # wall rows are ignored
    L.lbm_set_rho(ctx, rho)
    f0 = L.lbm_get_f(ctx)
    for bad in (-1.0, 0.0, np.nan, np.inf):
        r = rho.copy()
        r[4, 4] = bad
        with pytest.raises(L.LbmError) as e:
            L.lbm_set_rho(ctx, r)  # checked on the device before the state is touched
        assert e.value.status == L.LBM_EINVAL
        assert np.array_equal(L.lbm_get_f(ctx), f0)
    L.lbm_destroy(ctx)


@pytest.mark.parametrize("precision,kernel", [(64, REF), (32, FUSED)])
def test_instability_is_reported(precision, kernel):
    p = Pair(32, 16, precision=precision, kernel=kernel, check_every=1)
    rho = np.full((16, 32), p.rho_l)
    p.gpu.set_rho(rho)
    f = p.gpu.f()
    f[:, 7, 9] = np.nan
    p.gpu.set_f(f)
    with pytest.raises(L.LbmError) as e:
        p.gpu.step(3)
    assert e.value.status == L.LBM_EUNSTABLE
    with pytest.raises(L.LbmError):
        p.gpu.step(1)  # sticky
    p.close()


def test_torch_owned_state_and_stream():
    torch = pytest.importorskip("torch")
    s = torch.cuda.Stream()
    w = I.single_droplet(90.0)
    a = droplet_pair(w, precision=32, kernel=FUSED, torch_state=True, stream=s)
    b = droplet_pair(w, precision=32, kernel=FUSED)
    a.gpu.step(30)
    b.gpu.step(30)
    assert np.array_equal(a.gpu.f(), b.gpu.f())
    a.close()
    b.close()


def test_contexts_with_different_fused_rings_coexist(monkeypatch):
    """The fused kernel's launch attributes are per kernel: a context planned
    with a deep TMA ring still launches after a shallower one is created."""
    w = I.single_droplet(90.0)
    monkeypatch.setenv("LBM_FUSED_STAGES", "8")
    a = droplet_pair(w, precision=32, kernel=FUSED)
    monkeypatch.setenv("LBM_FUSED_STAGES", "3")
    b = droplet_pair(w, precision=32, kernel=FUSED)
    assert a.gpu.info.tile_stages == 8 and b.gpu.info.tile_stages == 3
    a.gpu.step(5)
    b.gpu.step(5)
    assert np.array_equal(a.gpu.f(), b.gpu.f())
    a.close()
    b.close()


@pytest.mark.parametrize("nx,ny", [(260, 37), (400, 200), (2048, 300)])
def test_fused_partition_does_not_change_the_result(monkeypatch, nx, ny):
    """Which CTA sweeps which rows changes nothing, bit for bit: 1, 2 and the
    default number of CTAs per SM cut the rows into different ranges (at
    400 x 200 the default gives every CTA one row)."""
    w = I.throughput(nx=nx, ny=ny)
    out = []
    for ctas in ("1", "2", None):
        if ctas is None:
            monkeypatch.delenv("LBM_FUSED_CTAS_PER_SM", raising=False)
        else:
            monkeypatch.setenv("LBM_FUSED_CTAS_PER_SM", ctas)
        p = droplet_pair(w, precision=32, kernel=FUSED, check_every=1)
        p.gpu.step(6)
        assert p.gpu.status() == 0
        out.append((p.gpu.info.tile_blocks, p.gpu.f()))
        p.close()
    if nx >= 400:  # 260 x 37 has 70 rows: one per CTA at every setting
        assert len({b for b, _ in out}) == 3
    assert all(np.array_equal(out[0][1], f) for _, f in out[1:])


@pytest.mark.parametrize("kernel", [FUSED, REF])
def test_graph_replay_equals_direct_launches(kernel):
    """lbm_step with graphs of 16 steps (on a non-default stream) gives the
    same bits and counts the same launches as one launch sequence per step."""
    import torch

    stream = torch.cuda.Stream()
    w = I.single_droplet(60.0)
    runs = []
    for gs in (16, 0):
        p = Pair(w.nx, w.ny, t_over_tc=w.t_over_tc, tau=w.tau, theta=w.theta, rates=w.rates, eos=w.eos,
                 precision=32, kernel=kernel, stream=stream)
        p.gpu.close()
        p.params.graph_steps = gs
        g = L.Lbm(w.nx, w.ny, p.geos, p.T, p.tau, theta=p.theta, params=p.params, stream=stream, torch_state=False)
        g.set_rho(I.droplet_field(w.nx, w.ny, w.droplets, p.rho_v, p.rho_l, w.width))
        l0 = g.launches()
        g.step(37)
        g.step(50)
        runs.append((g.f(), g.launches() - l0, g.info.steps_done))
        g.close()
        p.orc.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    assert runs[0][1:] == runs[1][1:]


def test_graph_replay_reports_instability():
    import torch

    stream = torch.cuda.Stream()
    p = Pair(40, 20, precision=32, kernel=FUSED, check_every=32, stream=stream)
    f = I.random_distributions(I.droplet_field(40, 20, [(20.0, 6.0, 0)], p.rho_v, p.rho_l), 3)
    f[:, 7, 11] = np.nan
    p.gpu.set_f(f)
    with pytest.raises(L.LbmError) as e:
        p.gpu.step(64)  # one graph of 64 steps, then the check at step 64
    assert e.value.status == L.LBM_EUNSTABLE
    p.close()
