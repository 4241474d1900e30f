"""Pins for the oracle's interaction force (Eq. 9, Eq. 14) and Eq. 17 tensor.

Checks: exact zeros for uniform fields, second-order convergence of the
lattice sums to their continuum limits (F -> -grad U for any A, which is what
fixes c = 1 in Eq. 10; Q -> the isotropic second-derivative form), momentum
balance in a periodic box, and a hand-evaluated Martys-Chen wall force.
"""
import numpy as np
import pytest

import oracle as O

CS = O.carnahan_starling()
TC, _ = O.cs_critical(CS)


def _sim(n, ny=None, walls=False, **kw):
    ny = ny or n
    return O.Sim(n, ny, CS, kw.pop("T", 0.9 * TC), walls=walls, **kw)


def _dpdrho(T, r, h=1e-6):
    p = lambda x: O.pressure(CS, T, x)
    return (-p(r + 2 * h) + 8 * p(r + h) - 8 * p(r - h) + p(r - 2 * h)) / (12 * h)


def _smooth_rho(n, r0=0.04, d=0.01):
    y, x = np.mgrid[0:n, 0:n].astype(float)
    return r0 + d * np.sin(2 * np.pi * x / n + 0.3) * np.cos(2 * np.pi * y / n - 0.7)


def test_uniform_fields_give_exact_zero():
    for walls in (False, True):
        s = _sim(12, 10, walls=walls, theta=np.deg2rad(37.0))
        rho = np.full((10, 12), 0.2)
        s.set_rho(rho)
        fl = s.fields()
        fluid = slice(1, -1) if walls else slice(None)
        for k in ("Fx", "Fy", "Qxx", "Qyy", "Qxy"):
            assert np.all(fl[k][fluid] == 0.0), k


@pytest.mark.parametrize("A", [-0.6, 0.0, 1.0])
def test_force_converges_to_minus_grad_U(A):
    """F = -A sum w U e - (1-A) G psi sum w psi e -> -grad U with second order
    (sum_a w_a e_a e_a = I for w = 1/3, 1/12); this is the Eq. 10 reading c = 1."""
    T = 0.9 * TC
    errs = []
    for n in (16, 32, 64):
        s = _sim(n, T=T, A=A, kappa=0.0)
        rho = _smooth_rho(n)
        s.set_rho(rho)
        fl = s.fields()
        y, x = np.mgrid[0:n, 0:n].astype(float)
        k = 2 * np.pi / n
        drx = 0.01 * k * np.cos(k * x + 0.3) * np.cos(k * y - 0.7)
        dry = -0.01 * k * np.sin(k * x + 0.3) * np.sin(k * y - 0.7)
        dU = np.vectorize(lambda r: _dpdrho(T, r) - 1.0 / 3.0)(rho)
        gx, gy = dU * drx, dU * dry
        scale = max(np.abs(gx).max(), np.abs(gy).max())
        errs.append(max(np.abs(fl["Fx"] + gx).max(), np.abs(fl["Fy"] + gy).max()) / scale)
    assert errs[-1] < 5e-3
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7


def _spectral_d2(f):
    n = f.shape[0]
    k = np.fft.fftfreq(n) * 2 * np.pi
    F = np.fft.fft2(f)
    ky, kx = np.meshgrid(k, k, indexing="ij")
    dxx = np.real(np.fft.ifft2(-(kx**2) * F))
    dyy = np.real(np.fft.ifft2(-(ky**2) * F))
    dxy = np.real(np.fft.ifft2(-(kx * ky) * F))
    return dxx, dyy, dxy


@pytest.mark.parametrize("A", [-0.6, 1.0])
def test_Q_tensor_converges_to_continuum_form(A):
    """sum_a w_a (phi(x+e_a) - phi(x)) e_ai e_aj -> (delta_ij lap phi + 2 d_i d_j phi)/6,
    so Eq. 17 (with the G/2 prefactor) tends to
    kappa G/2 [(1-A) psi (d_ij lap psi + 2 d_ij psi)/6 + A/2 (d_ij lap psi^2 + 2 d_ij psi^2)/6]."""
    kappa, G = 0.7, -1.0
    errs = []
    for n in (16, 32, 64):
        s = _sim(n, A=A, kappa=kappa)
        s.set_rho(_smooth_rho(n))
        fl = s.fields()
        psi = fl["psi"]
        pxx, pyy, pxy = _spectral_d2(psi)
        qxx, qyy, qxy = _spectral_d2(psi * psi)
        lp, lq = pxx + pyy, qxx + qyy

        def cont(dp_ij, dq_ij, delta):
            return kappa * G / 2 * ((1 - A) * psi * (delta * lp + 2 * dp_ij) / 6 + A / 2 * (delta * lq + 2 * dq_ij) / 6)

        ref = {"Qxx": cont(pxx, qxx, 1), "Qyy": cont(pyy, qyy, 1), "Qxy": cont(pxy, qxy, 0)}
        scale = max(np.abs(v).max() for v in ref.values())
        errs.append(max(np.abs(fl[k] - ref[k]).max() for k in ref) / scale)
    assert errs[-1] < 5e-3
    assert 3.3 < errs[0] / errs[1] < 4.7 and 3.3 < errs[1] / errs[2] < 4.7


def test_periodic_box_total_force_vanishes():
    rng = np.random.default_rng(7)
    n = 24
    s = _sim(n, T=0.7 * TC)
    rv, rl = O.coexistence(CS, 0.7 * TC)
    s.set_rho(rng.uniform(rv, rl, (n, n)))
    fl = s.fields()
    for k in ("Fx", "Fy"):
        assert abs(fl[k].sum()) < 1e-14 * np.abs(fl[k]).sum()


@pytest.mark.parametrize("Gw", [-1.43, 0.5])
def test_martys_chen_wall_force_hand_value(Gw):
    """Uniform fluid between solid rows, Martys-Chen variant.  At the boundary
    row the three solid neighbours below give sum_a w_a S e_a = (0, -1/2);
    they carry psi = U = 0, so the fluid part keeps only the upper half of
    each sum:  F_y = -A U/2 - (1-A) G psi^2/2 + G_w psi/2, F_x = 0."""
    A, G, T, r = -0.6, -1.0, 0.8 * TC, 0.25
    s = O.Sim(10, 8, CS, T, walls=True, A=A, G_w=Gw, wetting=O.MARTYS_CHEN)
    s.set_rho(np.full((8, 10), r))
    fl = s.fields()
    psi, U = O.psi_U(CS, T, r)
    expect = -A * U / 2 - (1 - A) * G * psi * psi / 2 + Gw * psi / 2
    assert np.allclose(fl["Fy"][1], expect, rtol=1e-13)
    assert np.allclose(fl["Fy"][-2], -expect, rtol=1e-13)
    assert np.all(fl["Fx"][1:-1] == 0.0)
    assert np.all(fl["Fy"][2:-2] == 0.0)
    # a negative G_w pulls fluid toward the wall (more wetting, Fig. 1 ordering)
    s0 = O.Sim(10, 8, CS, T, walls=True, A=A, G_w=0.0, wetting=O.MARTYS_CHEN)
    s0.set_rho(np.full((8, 10), r))
    dF = fl["Fy"][1, 0] - s0.fields()["Fy"][1, 0]
    assert np.sign(dF) == np.sign(Gw)
