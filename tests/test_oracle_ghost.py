"""Pins for the oracle's geometric ghost density (Eqs. 19-21).

Eq. 20 (read with its square root) has Eq. 19 as its exact fixed point; the
iteration of Eq. 21 starts from (rho_{i,2} - rho_{i,0}) ~ 2 (rho_{i,2} - rho_{i,1})
and is a contraction with factor |cos theta|.
"""
import math

import numpy as np
import pytest

import oracle as O

BIG = np.finfo(np.float64).max


def _coeffs(theta):
    return math.sin(math.pi / 2 - theta), math.tan(math.pi / 2 - theta)


def _samples(rng, n=200):
    for _ in range(n):
        r = rng.uniform(1e-3, 1.0, 4)
        yield r[0], r[1], r[2], r[3]


def test_ninety_degrees_returns_second_row_exactly():
    rng = np.random.default_rng(10)
    c, cot = _coeffs(math.pi / 2)
    assert c == 0.0
    for rl, rr, r1, r2 in _samples(rng):
        for k in (0, 1, 4, 9):
            assert O.ghost(rl, rr, r1, r2, c, cot, k) == r2


def test_uniform_rows_give_second_row_exactly():
    for th in (15, 45, 120, 165):
        c, cot = _coeffs(math.radians(th))
        for k in (0, 1, 4):
            assert O.ghost(0.3, 0.3, 0.3, 0.3, c, cot, k) == 0.3


@pytest.mark.parametrize("th", [15, 30, 45, 60, 100, 135, 150, 165])
def test_iteration_converges_to_eq19(th):
    """Many Eq. 21 iterations reach the Eq. 19 value rho_2 + cot(theta)|a|."""
    rng = np.random.default_rng(11)
    c, cot = _coeffs(math.radians(th))
    for rl, rr, r1, r2 in _samples(rng, 50):
        g_inf = O.ghost(rl, rr, r1, r2, c, cot, 2000)
        g19 = O.ghost(rl, rr, r1, r2, c, cot, 0)
        assert g_inf == pytest.approx(g19, rel=1e-11, abs=1e-13)


@pytest.mark.parametrize("th", [20, 50, 80])
def test_contraction(th):
    """|g_{k+1} - g*| <= |cos theta| |g_k - g*| (the map d -> -c sqrt(a^2 + d^2)
    has Lipschitz constant |c|)."""
    rng = np.random.default_rng(12)
    c, cot = _coeffs(math.radians(th))
    for rl, rr, r1, r2 in _samples(rng, 50):
        gs = O.ghost(rl, rr, r1, r2, c, cot, 0)
        errs = [abs(O.ghost(rl, rr, r1, r2, c, cot, k) - gs) for k in range(1, 8)]
        for e0, e1 in zip(errs, errs[1:]):
            assert e1 <= abs(c) * e0 + 1e-15


def test_first_iterate_uses_four_times_square():
    """First line of Eq. 21: rho_{i,0,1} = rho_{i,2} + sin(pi/2-theta) sqrt(a^2 + 4 (rho_{i,2}-rho_{i,1})^2)."""
    rng = np.random.default_rng(13)
    for th in (15, 70, 140):
        c, cot = _coeffs(math.radians(th))
        for rl, rr, r1, r2 in _samples(rng, 20):
            ref = r2 + c * math.sqrt((rr - rl) ** 2 + 4 * (r2 - r1) ** 2)
            assert O.ghost(rl, rr, r1, r2, c, cot, 1, BIG) == pytest.approx(max(ref, 0.0), rel=1e-14, abs=1e-16)


def test_supplementary_angles_mirror_the_correction():
    """theta -> pi - theta flips the sign of every iterate's correction."""
    rng = np.random.default_rng(14)
    for th in (15, 40, 75):
        c, cot = _coeffs(math.radians(th))
        for rl, rr, r1, r2 in _samples(rng, 30):
            for k in (1, 2, 4):
                up = O.ghost(rl, rr, r1, r2, c, cot, k, BIG) - r2
                dn = O.ghost(rl, rr, r1, r2, -c, -cot, k, BIG) - r2
                if r2 + dn > 0:  # no clamping at zero on this side
                    assert up == pytest.approx(-dn, rel=1e-12, abs=1e-15)


def test_iterates_approach_eq19_monotonically():
    """|d_k| = c sqrt(a^2 + d_{k-1}^2) moves monotonically toward |d*| = |cot theta||a|,
    so for theta < 90 deg the iterates g_k = rho_2 + |d_k| approach the Eq. 19
    value from the side of the first guess 2 (rho_2 - rho_1)."""
    c, cot = _coeffs(math.radians(15))
    # |d_0| = 0.4 < |d*| = cot(15 deg) * 0.3: approach from below
    g = [O.ghost(0.05, 0.35, 0.1, 0.3, c, cot, k) for k in (1, 2, 3, 4)]
    g19 = O.ghost(0.05, 0.35, 0.1, 0.3, c, cot, 0)
    assert g[0] < g[1] < g[2] < g[3] < g19
    # |d_0| = 2.0 > |d*| = cot(15 deg) * 0.1: approach from above
    g = [O.ghost(0.25, 0.35, 0.1, 1.1, c, cot, k) for k in (1, 2, 3, 4)]
    g19 = O.ghost(0.25, 0.35, 0.1, 1.1, c, cot, 0)
    assert g[0] > g[1] > g[2] > g[3] > g19


def test_clamp_to_valid_range():
    c, cot = _coeffs(math.radians(170))
    assert O.ghost(0.0, 1.0, 0.01, 0.02, c, cot, 4, 0.55) == 0.0
    c, cot = _coeffs(math.radians(5))
    assert O.ghost(0.0, 1.0, 0.01, 0.5, c, cot, 4, 0.55) == 0.55


def test_clamped_ghost_carries_zero_potential():
    """A ghost density clamped at rho_max (the root of U = p - rho/3, Eq. 10)
    carries psi = U = 0 exactly in the simulation fields."""
    eos = O.carnahan_starling()
    T = 0.5 * O.cs_critical(eos)[0]
    rv, rl = O.coexistence(eos, T)
    rm = O.rho_max(eos, T, rl)
    nx, ny = 12, 8
    s = O.Sim(nx, ny, eos, T, tau=0.6, theta=math.radians(20.0), rho_max_=rm)
    rho = np.full((ny, nx), rl)
    rho[1, 6:] = rv  # sharp step on the boundary row: large tangential gradient
    s.set_rho(rho)
    fl = s.fields()
    clamped = fl["rho"][0] == rm
    assert clamped.any()
    assert np.all(fl["psi"][0][clamped] == 0.0) and np.all(fl["U"][0][clamped] == 0.0)
