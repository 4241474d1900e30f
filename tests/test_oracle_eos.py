"""Pins for the oracle's equations of state and their set-up solvers.

Everything here is checked against something other than the oracle's own
formulas: the printed Table 1 (Sec. 3.1), literature constants of the
Carnahan-Starling critical point, a symbolic solve of the critical conditions,
and an independent scipy equal-area (Maxwell) construction.
"""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_piecewise_eos.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            ratio, r1, r2, tv, tm, tl = (float(t) for t in line.split())
            rows.append(dict(ratio=ratio, rho1=r1, rho2=r2, tv=tv, tm=tm, tl=tl))
    return rows


@pytest.mark.parametrize("row", _table1(), ids=lambda r: f"ratio{int(r['ratio'])}")
def test_table1_breakpoints(row):
    """Eqs. 12-13 solved for (rho1, rho2) reproduce Table 1 to its printed digits
    (the printed slopes are themselves rounded, hence 1e-3 relative)."""
    r1, r2 = O.piecewise_breakpoints(1.0, row["ratio"], row["tv"], row["tm"], row["tl"])
    assert r1 == pytest.approx(row["rho1"], rel=1e-3)
    assert r2 == pytest.approx(row["rho2"], rel=1e-3)


@pytest.mark.parametrize("row", _table1(), ids=lambda r: f"ratio{int(r['ratio'])}")
def test_table1_equal_area(row):
    """The solved EOS has equal pressures at rho_v, rho_l (Eq. 12) and a zero
    integral of dp/rho (Eq. 13) by quadrature of the Eq. 11 pressure."""
    from scipy.integrate import quad

    r1, r2 = O.piecewise_breakpoints(1.0, row["ratio"], row["tv"], row["tm"], row["tl"])
    eos = O.piecewise(row["tv"], row["tm"], row["tl"], r1, r2)
    pv, pl = O.pressure(eos, 0.0, 1.0), O.pressure(eos, 0.0, row["ratio"])
    assert pl == pytest.approx(pv, rel=1e-10, abs=1e-12)
    # slope of each branch read off the oracle's pressure, then integrate
    # dp/rho branch by branch
    chem = 0.0
    for lo, hi in [(1.0, r1), (r1, r2), (r2, row["ratio"])]:
        a, b = lo + 1e-3 * (hi - lo), hi - 1e-3 * (hi - lo)
        slope = (O.pressure(eos, 0.0, b) - O.pressure(eos, 0.0, a)) / (b - a)
        chem += quad(lambda r: slope / r, lo, hi, epsabs=1e-13)[0]
    assert abs(chem) < 1e-9
    # and the inverse direction recovers (rho_v, rho_l) = (1, ratio)
    rv, rl = O.coexistence(eos)
    assert rv == pytest.approx(1.0, rel=1e-9)
    assert rl == pytest.approx(row["ratio"], rel=1e-9)


def test_table1_printed_values_nearly_satisfy_eqs_12_13():
    """The printed Table 1 rows themselves satisfy Eq. 12 and Eq. 13 to the
    rounding of their digits, which confirms the reading rho_v = 1,
    rho_l = ratio."""
    for row in _table1():
        rv, rl = 1.0, row["ratio"]
        e12 = (row["rho1"] - rv) * row["tv"] + (row["rho2"] - row["rho1"]) * row["tm"] + (rl - row["rho2"]) * row["tl"]
        e13 = (math.log(row["rho1"] / rv) * row["tv"] + math.log(row["rho2"] / row["rho1"]) * row["tm"]
               + math.log(rl / row["rho2"]) * row["tl"])
        assert abs(e12) < 1e-3 and abs(e13) < 1e-3


def test_cs_critical_point_literature():
    """Carnahan-Starling + attraction: T_c = 0.3773 a/(b R), eta_c = 0.1304,
    critical compressibility Z_c = 0.3590 (literature constants)."""
    for a, b, R in [(1.0, 4.0, 1.0), (0.25, 4.0, 1.0), (0.5, 2.0, 0.7)]:
        eos = O.carnahan_starling(a, b, R)
        Tc, rc = O.cs_critical(eos)
        assert Tc * b * R / a == pytest.approx(0.3773, abs=5e-5)
        assert rc * b / 4.0 == pytest.approx(0.1304, abs=5e-5)
        Zc = O.pressure(eos, Tc, rc) / (rc * R * Tc)
        assert Zc == pytest.approx(0.3590, abs=5e-4)


def test_cs_critical_point_symbolic():
    """A symbolic solve of dp/drho = d2p/drho2 = 0 on the EOS agrees to 1e-12."""
    sp = pytest.importorskip("sympy")
    rho, T = sp.symbols("rho T", positive=True)
    a, b, R = sp.Integer(1), sp.Integer(4), sp.Integer(1)
    eta = b * rho / 4
    p = rho * R * T * (1 + eta + eta**2 - eta**3) / (1 - eta) ** 3 - a * rho**2
    sol = sp.nsolve([sp.diff(p, rho), sp.diff(p, rho, 2)], [rho, T], [0.13, 0.094], prec=30)
    Tc, rc = O.cs_critical(O.carnahan_starling())
    assert rc == pytest.approx(float(sol[0]), rel=1e-12)
    assert Tc == pytest.approx(float(sol[1]), rel=1e-12)


@pytest.mark.parametrize("tr", [0.5, 0.6, 0.7, 0.8, 0.9])
def test_cs_maxwell_equal_area(tr):
    """Coexistence densities satisfy p_v = p_l and the equal-area rule
    integral_{v_l}^{v_v} (p(v) - p_s) dv = 0, checked by scipy quadrature."""
    from scipy.integrate import quad

    eos = O.carnahan_starling()
    Tc, _ = O.cs_critical(eos)
    T = tr * Tc
    rv, rl = O.coexistence(eos, T)
    assert rv < rl
    pv, pl = O.pressure(eos, T, rv), O.pressure(eos, T, rl)
    assert pl == pytest.approx(pv, rel=1e-8, abs=1e-14)
    # equal area in specific volume v = 1/rho; substitute v = exp(s) to keep the
    # huge vapour volume well resolved
    def integrand(s):
        v = math.exp(s)
        return (O.pressure(eos, T, 1.0 / v) - pv) * v

    area = quad(integrand, math.log(1.0 / rl), math.log(1.0 / rv), limit=400, epsabs=1e-14, epsrel=1e-12)[0]
    scale = pv * (1.0 / rv - 1.0 / rl)
    assert abs(area) < 1e-7 * max(scale, 1e-30) + 1e-12


def test_cs_coexistence_approaches_critical():
    eos = O.carnahan_starling()
    Tc, rc = O.cs_critical(eos)
    rv, rl = O.coexistence(eos, 0.999 * Tc)
    assert rv < rc < rl
    assert (rl - rv) / rc < 0.2
    with pytest.raises(ValueError):
        O.coexistence(eos, 1.01 * Tc)


@pytest.mark.parametrize("tr", [0.5, 0.7, 0.9])
def test_rho_max_bounds_psi(tr):
    """rho_max is where psi^2 = 2(rho/3 - p) first returns to zero above rho_l."""
    eos = O.carnahan_starling()
    Tc, _ = O.cs_critical(eos)
    T = tr * Tc
    rv, rl = O.coexistence(eos, T)
    rm = O.rho_max(eos, T, rl)
    assert rl < rm < 1.0
    assert abs(O.pressure(eos, T, rm) - rm / 3.0) < 1e-12
    for r in np.linspace(rl, rm, 50)[1:-1]:
        assert O.pressure(eos, T, r) < r / 3.0
    assert O.psi_U(eos, T, rm * 1.001)[0] == 0.0


def test_psi_positive_on_two_phase_range():
    """With G = -1 the pseudo-potential is real on the whole coexistence range
    for both EOS families."""
    eos = O.carnahan_starling()
    Tc, _ = O.cs_critical(eos)
    for tr in (0.5, 0.8):
        rv, rl = O.coexistence(eos, tr * Tc)
        for r in np.geomspace(rv, rl, 64):
            psi, U = O.psi_U(eos, tr * Tc, r)
            assert psi > 0 and U < 0 and psi * psi == pytest.approx(-2 * U, rel=1e-12)
    for row in _table1():
        r1, r2 = O.piecewise_breakpoints(1.0, row["ratio"], row["tv"], row["tm"], row["tl"])
        pw = O.piecewise(row["tv"], row["tm"], row["tl"], r1, r2)
        for r in np.geomspace(1.0, row["ratio"], 64):
            assert O.psi_U(pw, 0.0, r)[0] > 0
