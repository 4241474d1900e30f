"""Discrete adjoint (lbm_adjoint_record / lbm_adjoint_backward) through the C
ABI against torch autograd of the oracle's differentiable restatement of the
step (oracle/autodiff.py), on small grids with every model variant; FP32
against FP64; the torch.autograd.Function wrapper; and the wall-angle
inversion case (256 x 128, 2000 steps) against the FP64 oracle's central
finite differences stored in tests/golden/c5_oracle_fd.txt."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import autodiff as AD  # noqa: E402
from paper_1501_05430_gb300 import adjoint as ADJ  # noqa: E402
from paper_1501_05430_gb300 import inputs as I  # noqa: E402
from paper_1501_05430_gb300 import lbm as L  # noqa: E402

from helpers import Case, resolve_rates  # noqa: E402

pytestmark = pytest.mark.gpu

PW10 = (0.25, -0.02, 0.3, 1.1216073327407194, 9.540106186999981)
VARIANTS = {
    "geometric": dict(),
    "eq19_only": dict(n_iter=0),
    "eight_iterations": dict(n_iter=8),
    "martys_chen": dict(wetting=1, G_w=-0.2),
    "periodic_box": dict(walls=False),
    "piecewise": dict(eos="pw", pw=PW10),
    "mrt_rates": dict(rates=dict(s_e=0.8, s_eps=0.9, s_j=1.0, s_q=1.1), kappa=0.9, A=-0.3, tau=0.9),
}


def _case(nx, ny, seed, precision=64, **kw):
    rng = np.random.default_rng(seed)
    walls = kw.get("walls", True)
    theta = np.full((ny, nx), np.pi / 2)
    if walls:
        theta[0] = rng.uniform(np.deg2rad(30), np.deg2rad(150), nx)
        theta[-1] = rng.uniform(np.deg2rad(30), np.deg2rad(150), nx)
    c = Case(nx, ny, theta=theta, precision=precision, kernel=L.LBM_KERNEL_REFERENCE, **kw)
    drops = [(nx * 0.3, ny * 0.35, 0), (nx * 0.7, ny * 0.3, 1)] if walls else [(nx * 0.4, ny * 0.3, ny * 0.5)]
    rho = I.droplet_field(nx, ny, drops, c.rho_v, c.rho_l)
    c.f0 = I.random_distributions(rho, seed, walls=walls)
    c.kw = kw
    return c


def _model(c, th_bot, th_top, T):
    kw = c.kw
    r = resolve_rates(kw.get("tau", 1.0), kw.get("rates"))
    s = (r["s_rho"], r["s_e"], r["s_eps"], r["s_j"], r["s_q"], r["s_j"], r["s_q"], r["s_nu"], r["s_nu"])
    e = c.oeos
    eos = ("cs", e.a, e.b, e.R) if kw.get("eos", "cs") == "cs" else ("pw", e.theta_v, e.theta_m, e.theta_l,
                                                                    e.rho1, e.rho2)
    return AD.Model(c.nx, c.ny, eos, T, th_bot, th_top, s, A=kw.get("A", -0.6), kappa=kw.get("kappa", 0.5),
                    G_w=kw.get("G_w", 0.0), n_iter=kw.get("n_iter", 4), wetting=kw.get("wetting", 0),
                    walls=kw.get("walls", True), rho_max=c.rho_max)


def _reference_gradients(c, wts, steps):
    tb = torch.tensor(c.theta[0], requires_grad=True)
    tt = torch.tensor(c.theta[-1], requires_grad=True)
    T = torch.tensor(c.T, dtype=torch.float64, requires_grad=True)
    f0 = torch.tensor(c.f0, requires_grad=True)
    m = _model(c, tb, tt, T)
    loss = (m.run(f0, steps).sum(0) * torch.tensor(wts)).sum()
    loss.backward()

    def g(t):  # parameters the variant does not use get no gradient at all
        return torch.zeros_like(t) if t.grad is None else t.grad

    return np.stack([g(tb).numpy(), g(tt).numpy()]), g(T).item(), f0.grad.numpy()


def _lib_gradients(c, wts, steps, every, precision=64, kernel=None):
    p = L.lbm_params()
    for name, _ in p._fields_:
        setattr(p, name, getattr(c.params, name))
    p.precision = precision
    if kernel is not None:
        p.kernel = kernel
    with L.Lbm(c.nx, c.ny, c.geos, c.T, c.tau, theta=c.theta, walls=c.walls, params=p, torch_state=False) as s:
        s.set_f(c.f0)
        L.lbm_adjoint_record(s.ctx, steps, every)
        dth, dT, df0 = L.lbm_adjoint_backward(s.ctx, wts, want_df0=True)
    return dth, dT, df0


def _close(a, b, tol):
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(np.asarray(a) - np.asarray(b)).max() <= tol * scale


@pytest.mark.parametrize("name", list(VARIANTS))
def test_fp64_adjoint_equals_autograd_of_the_oracle(name):
    """L = sum w rho after 12 steps (checkpoints every 5: segments 5, 5, 2)."""
    c = _case(16, 10, seed=3, **VARIANTS[name])
    wts = np.random.default_rng(4).uniform(-1, 1, (c.ny, c.nx))
    dth_r, dT_r, df0_r = _reference_gradients(c, wts, 12)
    dth, dT, df0 = _lib_gradients(c, wts, 12, 5)
    assert _close(df0, df0_r, 1e-10)
    if c.walls:
        assert _close(dth, dth_r, 1e-9)
    else:
        assert not dth.any()
    assert dT == pytest.approx(dT_r, rel=1e-9, abs=1e-12)
    c.orc.close()


def test_checkpoint_interval_does_not_change_the_gradient():
    c = _case(20, 9, seed=7)
    wts = np.random.default_rng(8).uniform(-1, 1, (c.ny, c.nx))
    ref = _lib_gradients(c, wts, 17, 17)
    for every in (1, 4, 6):
        got = _lib_gradients(c, wts, 17, every)
        assert np.array_equal(got[0], ref[0]) and got[1] == ref[1] and np.array_equal(got[2], ref[2])
    c.orc.close()


@pytest.mark.parametrize("kernel", [L.LBM_KERNEL_REFERENCE, L.LBM_KERNEL_FUSED])
def test_fp32_adjoint_close_to_fp64(kernel):
    """FP32 gradients within 1e-3 of FP64, with the forward recorded and
    replayed by the canonical FP32 kernels or by the fused kernel."""
    c = _case(32, 14, seed=5)
    wts = np.random.default_rng(6).uniform(-1, 1, (c.ny, c.nx))
    d64 = _lib_gradients(c, wts, 40, 10, 64)
    d32 = _lib_gradients(c, wts, 40, 10, 32, kernel=kernel)
    assert _close(d32[0], d64[0], 1e-3)
    assert d32[1] == pytest.approx(d64[1], rel=1e-3)
    c.orc.close()


def test_autograd_function_matches_direct_backward():
    c = _case(24, 12, seed=9)
    wts = np.random.default_rng(10).uniform(-1, 1, (c.ny, c.nx))
    tb = torch.tensor(c.theta[0], requires_grad=True)
    T = torch.tensor(c.T, dtype=torch.float64, requires_grad=True)
    rho = ADJ.final_density(tb, T, nx=c.nx, ny=c.ny, eos=c.geos, tau=c.tau, params=c.params, f0=c.f0, steps=9,
                            checkpoint_every=4, theta_top=c.theta[-1])
    (rho * torch.tensor(wts)).sum().backward()
    dth, dT, _ = _lib_gradients(c, wts, 9, 4)
    assert np.array_equal(tb.grad.numpy(), dth[0])
    assert T.grad.item() == dT
    c.orc.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_record_advances_like_lbm_step(precision):
    """The recorded forward runs the context's own step kernel: the canonical
    kernels in FP64, the fused kernel in FP32 -- the same bits as lbm_step."""
    c = _case(16, 10, seed=2)
    p = L.lbm_params()
    for name, _ in p._fields_:
        setattr(p, name, getattr(c.params, name))
    p.precision = precision
    p.kernel = L.LBM_KERNEL_AUTO
    with L.Lbm(c.nx, c.ny, c.geos, c.T, c.tau, theta=c.theta, params=p, torch_state=False) as a, \
            L.Lbm(c.nx, c.ny, c.geos, c.T, c.tau, theta=c.theta, params=p, torch_state=False) as b:
        assert a.info.kernel_in_use == (L.LBM_KERNEL_FUSED if precision == 32 else L.LBM_KERNEL_REFERENCE)
        a.set_f(c.f0)
        b.set_f(c.f0)
        L.lbm_adjoint_record(a.ctx, 11, 3)
        b.step(11)
        assert np.array_equal(a.f(), b.f())
        assert a.info.steps_done == 11
    c.orc.close()


# ---- wall-angle inversion case against the oracle's finite differences ------

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c5_oracle_fd.txt")


def _golden():
    """(meta, h_target, rows); a row is (name, index, fd, err, fd_coarse): the
    central difference at the middle rung of a step ladder, its noise estimate
    (largest change to the neighbouring rungs) and the one at the coarsest."""
    meta, rows, h_t = {}, [], None
    lines = open(GOLDEN).read().splitlines()
    for k, line in enumerate(lines):
        if line.startswith("# T ="):
            parts = line[2:].replace("=", " ").split()
            meta = {parts[i]: float(parts[i + 1]) for i in range(0, len(parts), 2)}
        elif line.startswith("# W_target ="):
            meta["W_target"] = float(line.split("=")[1])
        elif line.startswith("# h_target"):
            h_t = np.array([float(v) for v in lines[k + 1][2:].split()])
        elif not line.startswith("#") and line.strip():
            name, idx, fd, err, coarse = line.split()
            rows.append((name, int(idx), float(fd), float(err), float(coarse)))
    return meta, h_t, rows


# Tolerances.  FP64: 1e-3 relative on every row (measured: <= 7e-6).  FP32:
# the gradient is the canonical step's transpose evaluated along the FP32
# trajectory, whose densities differ from the FP64 ones by ~1e-4 relative per
# 1000 steps, so on a wall angle where the loss is smooth it moves by a few
# 1e-4 (measured: 1e-4 .. 5.4e-4).  Next to a ghost-clamp kink the FP32
# trajectory switches the clamp at slightly different parameter values, and
# the derivative moves by up to the slope change across the kinks, which the
# step ladder measures as |fd(1e-4) - fd| / |fd| (theta_169: 5.5e-3; its FP32
# gradient is 1.5e-3 .. 2.2e-3 off).  A wall angle is therefore held to
# 1e-3 + that kink term.  dL/dT sums the EOS sensitivity of every node in every
# step, so its FP32 rounding accumulates over 32768 nodes x 2000 steps
# (measured 7e-4 .. 1.2e-3): held to 3e-3.
def _tol(precision, name, fd, coarse):
    if precision == 64:
        return 1e-3
    if name == "T":
        return 3e-3
    return 1e-3 + abs(coarse - fd) / abs(fd)


@pytest.mark.skipif(not os.path.exists(GOLDEN), reason="golden finite differences not generated")
@pytest.mark.parametrize("precision,kernel", [(64, L.LBM_KERNEL_REFERENCE), (32, L.LBM_KERNEL_REFERENCE),
                                              (32, L.LBM_KERNEL_FUSED)])
def test_inversion_gradient_matches_oracle_finite_differences(precision, kernel):
    """Each sampled derivative (15 wall angles next to the contact lines and T)
    against the FP64 oracle's central difference, relative to its own size:
    |adjoint - fd| <= tol |fd| + 2 err (err: the difference's noise estimate)."""
    meta, h_t, rows = _golden()
    ac = I.adjoint_case()
    nx, ny = ac["nx"], ac["ny"]
    eos = L.carnahan_starling(1.0, 4.0, 1.0)
    T = meta["T"]
    rv, rl = meta["rho_v"], meta["rho_l"]
    theta = np.full((ny, nx), np.pi / 2)
    theta[0] = ac["theta"]
    p = L.lbm_params_default(precision=precision, kernel=kernel, check_every=0)
    with L.Lbm(nx, ny, eos, T, ac["tau"], theta=theta, params=p, torch_state=False) as s:
        s.set_rho(I.droplet_field(nx, ny, [ac["droplet"]], rv, rl, ac["width"]))
        L.lbm_adjoint_record(s.ctx, ac["steps"], ac["checkpoint_every"])
        loss, g = I.profile_loss_grad(s.rho(), h_t, meta["W_target"], rv, rl)
        if precision == 64:
            assert loss == pytest.approx(meta["loss"], rel=1e-10)
        dth, dT, _ = L.lbm_adjoint_backward(s.ctx, g)
    for name, idx, fd, err, coarse in rows:
        ad = dT if name == "T" else dth[0, idx]
        tol = _tol(precision, name, fd, coarse)
        assert abs(ad - fd) <= tol * abs(fd) + 2.0 * err, (name, idx, ad, fd, err, tol)


@pytest.mark.parametrize("precision", [64, 32])
def test_graph_replayed_adjoint_equals_direct_launches(precision):
    """On a non-default stream the recorded forward and the reverse sweep of
    every full segment replay captured graphs; same gradients, bit for bit
    (FP32: forward and replays by the fused kernel)."""
    import torch

    c = _case(20, 11, seed=12)
    wts = np.random.default_rng(13).uniform(-1, 1, (c.ny, c.nx))
    p = L.lbm_params()
    for name, _ in p._fields_:
        setattr(p, name, getattr(c.params, name))
    p.precision = precision
    p.kernel = L.LBM_KERNEL_AUTO
    out = []
    for stream in (None, torch.cuda.Stream()):
        with L.Lbm(c.nx, c.ny, c.geos, c.T, c.tau, theta=c.theta, params=p, stream=stream,
                   torch_state=False) as s:
            s.set_f(c.f0)
            L.lbm_adjoint_record(s.ctx, 27, 8)  # segments 8, 8, 8, 3
            out.append((s.f(),) + L.lbm_adjoint_backward(s.ctx, wts, want_df0=True))
            again = L.lbm_adjoint_backward(s.ctx, wts, want_df0=True)  # graphs reused
            assert np.array_equal(again[0], out[-1][1]) and again[1] == out[-1][2]
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    c.orc.close()
