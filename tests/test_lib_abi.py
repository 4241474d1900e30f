"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
entry point that include/lbm.h declares, and its host-side set-up (critical
point, coexistence) agrees with the oracle.  No kernel runs here."""
import os
import re

import numpy as np
import pytest

import oracle as O
from paper_1501_05430_gb300 import build as B
from paper_1501_05430_gb300 import lbm as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", txt)))


def test_library_builds_and_exports_every_declared_symbol():
    path = B.build()
    assert os.path.exists(path)
    lib = L.load()
    decl = _declared()
    assert len(decl) >= 25
    for name in decl:
        assert hasattr(lib, name), name
    assert set(decl) == set(L.exported_symbols())
    out = os.popen(f"nm -D --defined-only {path}").read()
    for name in decl:
        assert re.search(rf"\bT {name}$", out, re.M), name


def test_binding_has_same_names():
    for name in _declared():
        assert callable(getattr(L, name)), name


def test_params_default_is_paper_setup():
    p = L.lbm_params_default()
    assert (p.A, p.kappa, p.n_iter, p.wetting, p.precision) == (-0.6, 0.5, 4, 0, 32)


def test_strerror_names_codes():
    for code in range(0, -8, -1):
        assert L.lbm_strerror(code) != "unknown status"
    assert L.lbm_strerror(-99) == "unknown status"


@pytest.mark.parametrize("abR", [(1.0, 4.0, 1.0), (0.25, 4.0, 1.0), (0.5, 2.0, 0.7)])
def test_critical_point_matches_oracle(abR):
    tc, rc = L.lbm_eos_critical(L.carnahan_starling(*abR))
    otc, orc = O.cs_critical(O.carnahan_starling(*abR))
    assert tc == pytest.approx(otc, rel=1e-13)
    assert rc == pytest.approx(orc, rel=1e-13)


@pytest.mark.parametrize("tr", [0.5, 0.6, 0.7, 0.8, 0.95])
def test_cs_coexistence_matches_oracle(tr):
    tc, _ = O.cs_critical(O.carnahan_starling())
    rv, rl = L.lbm_coexistence(L.carnahan_starling(), tr * tc)
    orv, orl = O.coexistence(O.carnahan_starling(), tr * tc)
    assert rv == pytest.approx(orv, rel=1e-9)
    assert rl == pytest.approx(orl, rel=1e-12)


@pytest.mark.parametrize("ratio,tv,tm,tl", [(10, 0.25, -0.02, 0.3), (100, 0.1633, -0.02, 0.33333),
                                            (1000, 0.2, -0.01, 0.33333)])
def test_piecewise_coexistence_matches_oracle(ratio, tv, tm, tl):
    r1, r2 = O.piecewise_breakpoints(1.0, ratio, tv, tm, tl)
    rv, rl = L.lbm_coexistence(L.piecewise(tv, tm, tl, r1, r2))
    assert rv == pytest.approx(1.0, rel=1e-9)
    assert rl == pytest.approx(ratio, rel=1e-9)


@pytest.mark.parametrize("a", [1.0, 0.25])
@pytest.mark.parametrize("tr", [0.5, 0.6, 0.7, 0.8])
def test_library_density_bounds_match_oracle_cs(a, tr):
    """The bounds lbm_create derives by itself (no override in lbm_params):
    rho_max, the smallest root of p(rho) = rho/3 above rho_l (Eq. 10: psi^2 >= 0
    below it; the ghost-density clamp and the instability bound), and rho_mid,
    the contour of the angle measurement, equal the oracle's bisection root and
    coexistence midpoint."""
    oeos = O.carnahan_starling(a, 4.0, 1.0)
    T = tr * O.cs_critical(oeos)[0]
    orv, orl = O.coexistence(oeos, T)
    rv, rl, rmax, rmid = L.lbm_eos_bounds(L.carnahan_starling(a, 4.0, 1.0), T)
    assert rmax == pytest.approx(O.rho_max(oeos, T, orl), rel=1e-12)
    assert rmid == pytest.approx(0.5 * (orv + orl), rel=1e-12)
    assert rl < rmax < 1.0  # 4/b is the packing limit of Carnahan-Starling
    assert (rv, rl) == L.lbm_coexistence(L.carnahan_starling(a, 4.0, 1.0), T)


@pytest.mark.parametrize("ratio,tv,tm,tl", [(10, 0.25, -0.02, 0.3), (100, 0.1633, -0.02, 0.33333),
                                            (1000, 0.2, -0.01, 0.33333), (100, 0.1633, -0.02, 0.4)])
def test_library_density_bounds_match_oracle_piecewise(ratio, tv, tm, tl):
    """Eq. 11 rows of Table 1 (liquid slope below 1/3: psi^2 never returns to 0,
    so there is no upper bound) and one liquid slope above 1/3 (a finite root)."""
    r1, r2 = O.piecewise_breakpoints(1.0, ratio, tv, tm, tl)
    oeos = O.piecewise(tv, tm, tl, r1, r2)
    orv, orl = O.coexistence(oeos)
    rv, rl, rmax, rmid = L.lbm_eos_bounds(L.piecewise(tv, tm, tl, r1, r2))
    assert rmax == pytest.approx(O.rho_max(oeos, 0.0, orl), rel=1e-12)
    assert (rmax == np.finfo(np.float64).max) == (tl <= 1.0 / 3.0)
    assert rmid == pytest.approx(0.5 * (orv + orl), rel=1e-12)


def test_invalid_eos_rejected():
    with pytest.raises(L.LbmError) as e:
        L.lbm_coexistence(L.carnahan_starling(), 1.0)  # above T_c
    assert e.value.status == L.LBM_EINVAL
    with pytest.raises(L.LbmError) as e:
        L.lbm_eos_critical(L.piecewise(0.25, -0.02, 0.3, 1.1, 9.5))
    assert e.value.status == L.LBM_EUNSUPPORTED


def test_fp64_units_compiled_without_fma_contraction():
    """The canonical-order units must be built with -fmad=false."""
    assert "-fmad=false" in B.UNITS["lbm_ref.cu"]
    assert "-fmad=false" in B.UNITS["lbm_measure.cu"]


def test_required_state_bytes():
    """Two copies of the 9 nx ny distributions in the given precision; 0 for
    sizes or precisions the library does not take."""
    assert L.lbm_required_state_bytes(4096, 2048, 32) == 2 * 9 * 4096 * 2048 * 4
    assert L.lbm_required_state_bytes(100, 60, 64) == 2 * 9 * 100 * 60 * 8
    assert L.lbm_required_state_bytes(0, 60, 32) == 0
    assert L.lbm_required_state_bytes(100, 60, 16) == 0


def test_batch_config_default_leaves_every_choice_to_the_library():
    """All shape fields 0 (the library's defaults apply) and no held instance."""
    c = L.lbm_batch_config_default()
    assert c.threads == 0 and c.ctas_per_sm == 0 and c.stages == 0 and list(c.band_rows) == [0, 0, 0, 0]
    assert c.steps_per_launch == 0 and c.graph_launches == 0 and c.wait_seconds == 0.0
    assert c.hold_instance == -1
    c2 = L.lbm_batch_config_default(stages=5, band_rows=[8, 16, 32, 64])
    assert c2.stages == 5 and list(c2.band_rows) == [8, 16, 32, 64]
