"""Pins for the oracle's node collision (Eqs. 1-6, 15-16) and equilibrium.

The reference forms used here are textbook statements built independently of
the oracle: the D2Q9 moment basis generated from its defining polynomials of
e (not from a typed integer table), the second-order equilibrium
w_a rho [1 + 3 e.v + 9/2 (e.v)^2 - 3/2 v^2], and Guo's forcing term
w_a [3 (e_a - v) + 9 (e_a . v) e_a] . F.
"""
import math

import numpy as np
import pytest

import oracle as O

E = np.array([[0, 0], [1, 0], [0, 1], [-1, 0], [0, -1], [1, 1], [-1, 1], [-1, -1], [1, -1]], float)
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def moment_basis():
    """Rows: rho, e, eps, jx, qx, jy, qy, pxx, pxy as polynomials of e."""
    ex, ey = E[:, 0], E[:, 1]
    e2 = ex**2 + ey**2
    rows = [np.ones(9), -4 + 3 * e2, 4 - 10.5 * e2 + 4.5 * e2**2, ex, (-5 + 3 * e2) * ex, ey,
            (-5 + 3 * e2) * ey, ex**2 - ey**2, ex * ey]
    return np.array(rows)


def feq_textbook(rho, v):
    ev = E @ v
    return W * rho * (1 + 3 * ev + 4.5 * ev**2 - 1.5 * (v @ v))


def guo_textbook(v, F):
    ev = E @ v
    return W * ((3 * (E - v)) @ F + 9 * ev * (E @ F))


def test_moment_basis_orthogonal():
    M = moment_basis()
    G = M @ M.T
    assert np.allclose(G, np.diag(np.diag(G)))
    assert np.allclose(np.diag(G), [9, 36, 36, 6, 12, 6, 12, 4, 4])


def test_feq_matches_textbook():
    rng = np.random.default_rng(1)
    for _ in range(50):
        rho = rng.uniform(1e-3, 2.0)
        v = rng.uniform(-0.2, 0.2, 2)
        assert np.allclose(O.feq(rho, *v), feq_textbook(rho, v), rtol=1e-14, atol=1e-16)


def _random_f(rng):
    rho = rng.uniform(0.01, 1.0)
    v = rng.uniform(-0.1, 0.1, 2)
    return feq_textbook(rho, v) * (1 + 0.05 * rng.uniform(-1, 1, 9))


def test_bgk_special_case_is_textbook_bgk_guo():
    """All rates equal: m* = m - s(m - m_eq) + (1 - s/2) S is BGK with Guo forcing."""
    rng = np.random.default_rng(2)
    for _ in range(100):
        f = _random_f(rng)
        F = rng.uniform(-1e-2, 1e-2, 2)
        s = rng.uniform(0.5, 1.9)
        rho = f.sum()
        v = (E.T @ f + 0.5 * F) / rho
        ref = f - s * (f - feq_textbook(rho, v)) + (1 - 0.5 * s) * guo_textbook(v, F)
        out = O.collide(f, rho, F[0], F[1], 0.0, 0.0, 0.0, [s] * 9)
        assert np.allclose(out, ref, rtol=1e-12, atol=1e-15)


def test_mrt_general_rates_matrix_form():
    """Independent rates: f* = f - M^-1 L (M f - M f_eq) + M^-1 (I - L/2) M F_guo."""
    rng = np.random.default_rng(3)
    M = moment_basis()
    Minv = np.linalg.inv(M)
    for _ in range(100):
        f = _random_f(rng)
        F = rng.uniform(-1e-2, 1e-2, 2)
        sj, sq, snu = rng.uniform(0.5, 1.9, 3)
        s = np.array([0.0, rng.uniform(0.5, 1.9), rng.uniform(0.5, 1.9), sj, sq, sj, sq, snu, snu])
        rho = f.sum()
        v = (E.T @ f + 0.5 * F) / rho
        L = np.diag(s)
        ref = f - Minv @ L @ (M @ f - M @ feq_textbook(rho, v)) + Minv @ (np.eye(9) - 0.5 * L) @ M @ guo_textbook(v, F)
        out = O.collide(f, rho, F[0], F[1], 0.0, 0.0, 0.0, s)
        assert np.allclose(out, ref, rtol=1e-12, atol=1e-15)


def test_collision_conserves_mass_and_adds_force():
    rng = np.random.default_rng(4)
    for _ in range(50):
        f = _random_f(rng)
        F = rng.uniform(-1e-2, 1e-2, 2)
        Q = rng.uniform(-1e-3, 1e-3, 3)
        s = [0.0] + list(rng.uniform(0.5, 1.9, 8))
        s[5], s[6], s[8] = s[3], s[4], s[7]
        out = O.collide(f, f.sum(), F[0], F[1], *Q, s)
        assert out.sum() == pytest.approx(f.sum(), rel=1e-14)
        assert np.allclose(E.T @ out, E.T @ f + F, rtol=0, atol=1e-15)


def test_rest_state_is_fixed_point():
    for rho in (1.0, 0.3, 7.25e-4):
        f = O.feq(rho, 0.0, 0.0)
        out = O.collide(f, f.sum(), 0.0, 0.0, 0.0, 0.0, 0.0, [0.0] + [1.3] * 8)
        assert np.allclose(out, f, rtol=1e-14, atol=0)


def _source_moments(Q, s):
    """C as seen through the collision: M (f*(Q) - f*(0)) for an arbitrary f."""
    rng = np.random.default_rng(5)
    f = _random_f(rng)
    a = O.collide(f, f.sum(), 1e-3, -2e-3, *Q, s)
    b = O.collide(f, f.sum(), 1e-3, -2e-3, 0.0, 0.0, 0.0, s)
    return moment_basis() @ (a - b)


def test_source_touches_only_e_pxx_pxy():
    """Eq. 16: the source leaves the conserved moments, eps (Q_3 = 0) and the
    energy fluxes alone."""
    C = _source_moments([2e-3, -1e-3, 5e-4], [0.0, 1.1, 1.2, 1.0, 1.3, 1.0, 1.3, 1.4, 1.4])
    assert np.allclose(C[[0, 2, 3, 4, 5, 6]], 0, atol=1e-16)
    assert np.abs(C[[1, 7, 8]]).min() > 1e-5


def test_source_deviatoric_part_is_rotation_covariant():
    """The pxx and pxy entries of C are the two components of one traceless
    symmetric tensor: rotating Q by phi must rotate (C_pxx, 2 C_pxy) by 2 phi.
    This fixes the pxx coefficient to the pxy one (-s_nu), not 1.5 s_nu."""
    s = [0.0, 1.1, 1.2, 1.0, 1.3, 1.0, 1.3, 1.4, 1.4]
    Qm = np.array([[2e-3, 5e-4], [5e-4, -1e-3]])
    for phi in (0.3, math.pi / 6, 1.1):
        R = np.array([[math.cos(phi), -math.sin(phi)], [math.sin(phi), math.cos(phi)]])
        Qr = R @ Qm @ R.T
        c0 = _source_moments([Qm[0, 0], Qm[1, 1], Qm[0, 1]], s)
        c1 = _source_moments([Qr[0, 0], Qr[1, 1], Qr[0, 1]], s)
        R2 = np.array([[math.cos(2 * phi), -math.sin(2 * phi)], [math.sin(2 * phi), math.cos(2 * phi)]])
        assert np.allclose(R2 @ [c0[7], 2 * c0[8]], [c1[7], 2 * c1[8]], atol=1e-15)
        assert c1[1] == pytest.approx(c0[1], rel=1e-12)  # trace part is invariant


def test_half_force_shift_makes_momentum_rate_irrelevant():
    """With v = (j + F/2)/rho the post-collision momentum is j + F whatever s_j is."""
    rng = np.random.default_rng(6)
    f = _random_f(rng)
    F = np.array([3e-3, -1e-3])
    outs = [O.collide(f, f.sum(), *F, 0, 0, 0, [0, 1.1, 1.1, sj, 1.1, sj, 1.1, 1.1, 1.1]) for sj in (0.6, 1.0, 1.7)]
    for o in outs:
        assert np.allclose(E.T @ o, E.T @ f + F, atol=1e-16)
