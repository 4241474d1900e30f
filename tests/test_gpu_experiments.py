"""The paper's stationary-droplet experiments (Secs. 3.1-3.2, 4.2) as presets
of paper_1501_05430_gb300.experiments, each run as one batched sweep:

* parity: preset instances (Table 1 EOS, both wetting rules) against the FP64
  oracle over the first steps;
* the paper's qualitative findings that the presets reproduce: the geometric
  rule leaves the density normal to the wall flat (Fig. 8) and is stable over
  15-150 deg at density ratios 100 and 1000 (Figs. 6-7); the Martys-Chen force
  distorts the near-wall density (Figs. 1, 3), sets smaller angles for stronger
  attraction (Fig. 1), is unstable at ratio 1000 (Sec. 3.1), and its angle
  moves more with kappa than the geometric rule's (Figs. 4, 9)."""
import os

import numpy as np
import pytest

from paper_1501_05430_gb300 import experiments as E
from paper_1501_05430_gb300 import inputs as I
from paper_1501_05430_gb300 import lbm as L

from helpers import Case

pytestmark = pytest.mark.gpu

STEPS = 30000


def _pw(ratio):
    r1, r2, tv, tm, tl = I.TABLE1[ratio]
    return (tv, tm, tl, r1, r2)


@pytest.fixture(scope="module")
def results():
    cache = {}

    def get(name, init="semicircle"):
        if (name, init) not in cache:
            cache[(name, init)] = E.run(name, STEPS, init=init)
        return cache[(name, init)]

    return get


def test_preset_instances_match_the_oracle():
    """Three preset cases in one batch against the oracle after 200 steps."""
    specs = [(10, dict(wetting=1, G_w=-2.1)), (100, dict(theta=np.deg2rad(45.0))),
             (1000, dict(theta=np.deg2rad(90.0)))]
    cases = []
    for ratio, kw in specs:
        th = kw.pop("theta", np.pi / 2)
        theta = I.theta_field(E.NX, E.NY, th, np.pi / 2)
        c = Case(E.NX, E.NY, eos="pw", pw=_pw(ratio), tau=1.0, theta=theta, precision=32, **kw)
        c.rho0 = I.droplet_field(E.NX, E.NY, [(E.NX / 2.0, E.R0, 0)], c.rho_v, c.rho_l, 10.0)
        c.orc.set_rho(c.rho0)
        cases.append(c)
    with L.LbmBatch([c.desc() for c in cases]) as b:
        for c, inst in zip(cases, b.instances):
            inst.set_rho(c.rho0)
        b.step(200)
        for c, inst in zip(cases, b.instances):
            assert c.orc.step(200) == 0
            ro, rg = c.orc.rho()[1:-1], inst.rho()[1:-1]
            assert np.abs(rg - ro).max() <= 2e-5 * np.abs(ro).max()
            c.orc.close()


def test_geometric_rule_keeps_the_density_flat_normal_to_the_wall(results):
    """Fig. 8 (E9): liquid under the droplet and vapour away from it keep their
    bulk density down to the boundary row."""
    for r in results("E9"):
        assert r["status"] == "stable" and r["contact"] == "cap"
        for prof in (np.array(r["liquid_profile"]), np.array(r["vapour_profile"])):
            assert np.abs(prof[:8] - prof[12]).max() <= 2e-3 * prof[12], r["case"]


def test_martys_chen_distorts_the_near_wall_density(results):
    """Figs. 1 and 3 (E4): at G_w = -2.43 (ratio 10) the liquid is depleted and
    the vapour condensed next to the wall."""
    r = [x for x in results("E4") if x["G_w"] == -2.43][0]
    liq, vap = np.array(r["liquid_profile"]), np.array(r["vapour_profile"])
    assert liq[0] < 0.85 * liq[12]
    assert vap[0] > 2.0 * vap[12]


E7E8_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "e7e8_oracle_angles.txt")


def _e7e8_oracle():
    """{(preset, theta_set): angle} of the FP64 oracle's preset runs (cap start,
    four iterations, 30,000 steps), from make_e7e8_oracle_angles.py."""
    out, cols = {}, None
    for line in open(E7E8_GOLDEN):
        if line.startswith("# tag"):
            cols = line[2:].split()
        elif line.strip() and not line.startswith("#"):
            r = dict(zip(cols, line.split()))
            if r["tag"] == "preset":
                out[(r["preset"], float(r["theta"]))] = float(r["angle"])
    return out


@pytest.mark.parametrize("name", ["E7", "E8"])
def test_geometric_rule_is_stable_over_15_to_150_degrees(results, name):
    """Figs. 6-7: every set angle in {15, ..., 150} runs stably at ratio 100
    and 1000 and keeps a contact line; the measured angle rises with the set
    one, is within 3 deg of it up to 90 deg, and at every angle -- the obtuse
    ones included, where the four-iterate ghost rule and the droplet's
    resolution put it 5-25 deg above the set value -- within 0.5 deg of the
    FP64 oracle's angle for the same run."""
    res = results(name, init="cap")
    ref = _e7e8_oracle()
    th = []
    for r in res:
        assert r["status"] == "stable" and r["contact"] == "cap", r
        th.append(r["theta"])
        if r["theta_set"] <= 90.0:
            assert abs(r["theta"] - r["theta_set"]) <= 3.0, r
        assert abs(r["theta"] - ref[(name, r["theta_set"])]) <= 0.5, (r, ref[(name, r["theta_set"])])
    assert np.all(np.diff(th) > 0)


def test_martys_chen_is_unstable_at_ratio_1000(results):
    """Sec. 3.1 (E3): no attaching wall strength is stable at ratio 1000."""
    assert all(r["status"] == "unstable" for r in results("E3"))


def test_martys_chen_angle_falls_with_stronger_attraction(results):
    """Fig. 1 (E1, ratio 10): from droplets lifted off the wall (weak
    attraction) through caps to a film (strongest); the measured angle (on the
    boundary row, or above the depleted layer) falls monotonically."""
    res = results("E1")
    assert all(r["status"] == "stable" for r in res)
    assert res[0]["contact"] == "detached" and res[-1]["contact"] == "film"
    th = [r.get("theta", r.get("theta_above_layer")) for r in res[1:-1]]
    assert all(t is not None for t in th)
    assert np.all(np.diff(th) < 0)


def test_kappa_moves_the_martys_chen_angle_more_than_the_geometric_one(results):
    """Figs. 4 and 9 (E5, E10): over kappa in {0.5, 0.9, 0.98} the geometric
    angles at 45/90/135 deg move by a few degrees; the Martys-Chen angle at
    G_w = -2.1 moves by more."""
    geo = results("E10")
    spread_geo = max(np.ptp([r["theta"] for r in geo if r["theta_set"] == t]) for t in (45.0, 90.0, 135.0))
    mc = [r for r in results("E5") if r["G_w"] == -2.1]
    spread_mc = np.ptp([r["theta"] for r in mc])
    assert spread_geo <= 6.0
    assert spread_mc > spread_geo


def test_eq19_alone_and_four_iterations_agree_at_15_degrees(results):
    """Fig. 5 (E6) under the reading that Eq. 20 carries a square root: its
    fixed point is Eq. 19, so four iterations and Eq. 19 alone set nearly the
    same angle (both within 1 deg of each other and of 15 deg from the
    equilibrium-cap start); the paper reports 30 deg without iteration."""
    res = results("E6", init="cap")
    th = {r["n_iter"]: r["theta"] for r in res}
    assert abs(th[0] - th[4]) <= 1.0
    assert abs(th[4] - 15.0) <= 1.0


def test_martys_chen_calibration_hits_90_degrees_at_ratio_10():
    """G_w(theta) calibration (batched k-section at 5000 steps): 90 deg at
    ratio 10 lies between the E1 strengths -1.43 (107 deg) and -1.77 (84 deg),
    and re-running the calibrated G_w gives the angle within 2 deg."""
    (r,) = E.calibrate_gw([90.0], ratio=10, rounds=4)
    assert r["reached"], r
    assert -1.9 < r["G_w"] < -1.3, r
    (again,) = E.run("check", 5000, cases=[E.Case("check", 10, L.LBM_WET_MARTYS_CHEN, G_w=r["G_w"],
                                                  meta=dict(G_w=r["G_w"]))])
    assert abs(E._angle_of(again) - 90.0) <= 2.0, again
