"""Pins of oracle/autodiff.py, the differentiable restatement of the step that
serves as the reference for the adjoint kernels:

* its forward equals the C oracle's step to rounding on every model variant;
* its autograd derivatives w.r.t. the wall angles and T equal central finite
  differences of the C oracle's loss."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1501_05430_gb300 import inputs as I

torch = pytest.importorskip("torch")
from oracle import autodiff as AD  # noqa: E402

PW10 = (0.25, -0.02, 0.3, 1.1216073327407194, 9.540106186999981)
VARIANTS = {
    "geometric": dict(),
    "eq19_only": dict(n_iter=0),
    "martys_chen": dict(wetting=1, G_w=-0.2),
    "periodic_box": dict(walls=False),
    "piecewise": dict(eos="pw"),
    "mrt": dict(rates=(0.0, 0.8, 0.9, 1.0, 1.1, 1.0, 1.1, 1 / 0.9, 1 / 0.9), kappa=0.9, A=-0.3),
}


def _setup(nx, ny, seed, eos="cs", t_over_tc=0.8, rates=None, walls=True, **kw):
    rng = np.random.default_rng(seed)
    if eos == "cs":
        oeos = O.carnahan_starling(1.0, 4.0, 1.0)
        T = t_over_tc * O.cs_critical(oeos)[0]
        adeos = ("cs", 1.0, 4.0, 1.0)
    else:
        oeos = O.piecewise(*PW10)
        T = 0.0
        adeos = ("pw",) + PW10
    rv, rl = O.coexistence(oeos, T)
    rm = O.rho_max(oeos, T, rl)
    theta = np.full((ny, nx), np.pi / 2)
    theta[0] = rng.uniform(np.deg2rad(30), np.deg2rad(150), nx)
    theta[-1] = rng.uniform(np.deg2rad(30), np.deg2rad(150), nx)
    rates = rates or (0.0,) + (1.0,) * 8
    drops = [(nx * 0.3, ny * 0.35, 0), (nx * 0.7, ny * 0.3, 1)] if walls else [(nx * 0.4, ny * 0.3, ny * 0.5)]
    rho = I.droplet_field(nx, ny, drops, rv, rl)
    f0 = I.random_distributions(rho, seed, walls=walls)
    A, kappa, G_w = kw.get("A", -0.6), kw.get("kappa", 0.5), kw.get("G_w", 0.0)
    n_iter, wetting = kw.get("n_iter", 4), kw.get("wetting", 0)

    def oracle_sim(theta_=theta, T_=T):
        r = dict(s_rho=rates[0], s_e=rates[1], s_eps=rates[2], s_j=rates[3], s_q=rates[4], s_nu=rates[7])
        s = O.Sim(nx, ny, oeos, T_, walls=walls, A=A, kappa=kappa, G_w=G_w, n_iter=n_iter, wetting=wetting,
                  theta=theta_, rates=r, rho_max_=rm)
        s.set_f(f0)
        return s

    def model(th_bot, th_top, T_):
        return AD.Model(nx, ny, adeos, T_, th_bot, th_top, rates, A=A, kappa=kappa, G_w=G_w, n_iter=n_iter,
                        wetting=wetting, walls=walls, rho_max=rm)

    return dict(f0=f0, theta=theta, T=T, oracle_sim=oracle_sim, model=model, rm=rm)


@pytest.mark.parametrize("name", list(VARIANTS))
def test_forward_equals_c_oracle(name):
    kw = dict(VARIANTS[name])
    nx, ny = 14, 9
    S = _setup(nx, ny, seed=11, **kw)
    sim = S["oracle_sim"]()
    m = S["model"](torch.tensor(S["theta"][0]), torch.tensor(S["theta"][-1]), S["T"])
    f = torch.tensor(S["f0"])
    for _ in range(4):
        assert sim.step(1) == 0
        f = m.step(f)
        fo = sim.get_f()
        assert np.abs(f.numpy() - fo).max() <= 1e-12 * np.abs(fo).max()
    sim.close()


def _loss_weights(nx, ny, seed):
    return np.random.default_rng(seed).uniform(-1, 1, (ny, nx))


def test_autograd_equals_finite_differences_of_the_c_oracle():
    """L = sum w rho(final) after 8 steps, geometric walls with random angles:
    dL/dtheta at sampled wall nodes of both walls and dL/dT against central
    differences of the C oracle (h = 1e-6)."""
    nx, ny, steps = 16, 10, 8
    S = _setup(nx, ny, seed=4)
    wts = _loss_weights(nx, ny, 5)
    wts[0] = wts[-1] = 0.0

    def c_loss(theta, T):
        s = S["oracle_sim"](theta, T)
        assert s.step(steps) == 0
        v = float((s.rho() * wts).sum())
        s.close()
        return v

    tb = torch.tensor(S["theta"][0], requires_grad=True)
    tt = torch.tensor(S["theta"][-1], requires_grad=True)
    T = torch.tensor(S["T"], dtype=torch.float64, requires_grad=True)
    m = S["model"](tb, tt, T)
    f = m.run(torch.tensor(S["f0"]), steps)
    L = (f.sum(0) * torch.tensor(wts)).sum()
    L.backward()
    h = 1e-6
    for wall, idx in ((0, 3), (0, 9), (1, 5), (1, 12)):
        th_p, th_m = S["theta"].copy(), S["theta"].copy()
        row = 0 if wall == 0 else ny - 1
        th_p[row, idx] += h
        th_m[row, idx] -= h
        fd = (c_loss(th_p, S["T"]) - c_loss(th_m, S["T"])) / (2 * h)
        ad = (tb if wall == 0 else tt).grad[idx].item()
        assert ad == pytest.approx(fd, rel=1e-5, abs=1e-9), (wall, idx)
    hT = 1e-7
    fdT = (c_loss(S["theta"], S["T"] + hT) - c_loss(S["theta"], S["T"] - hT)) / (2 * hT)
    assert T.grad.item() == pytest.approx(fdT, rel=1e-5)


def test_kinks_pass_zero_gradient():
    """theta = 90 deg everywhere and a uniform film: the Eq. 21 root's argument
    and |a| vanish; the gradient is finite (the subgradient convention)."""
    nx, ny = 8, 7
    tb = torch.full((nx,), math.pi / 2, dtype=torch.float64, requires_grad=True)
    T = torch.tensor(0.8 * O.cs_critical(O.carnahan_starling())[0], dtype=torch.float64, requires_grad=True)
    m = AD.Model(nx, ny, ("cs", 1.0, 4.0, 1.0), T, tb, tb.detach().clone(), (0.0,) + (1.0,) * 8)
    rho = torch.full((ny, nx), 0.2, dtype=torch.float64)
    f = torch.tensor(I.LATTICE_SHAPE)[:, None, None] * rho[None]
    f = f * m.fluid
    out = m.run(f, 3)
    out.sum().backward()
    assert torch.isfinite(tb.grad).all() and torch.isfinite(T.grad)
