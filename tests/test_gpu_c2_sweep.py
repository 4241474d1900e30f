"""The 400 x 200 single-droplet sweep (20000 steps, FP32) against the FP64
oracle's results stored in tests/golden/c2_oracle_angles.txt (written by
make_c2_oracle_angles.py, which calls only the oracle).

For every stored case -- geometric wetting (Eqs. 19-21, four iterations) at
theta_set in {30, 60, 90, 120, 150} deg and Martys-Chen wetting (Eq. 14) on a
grid of G_w -- the FP32 run must end in the same state class (stable /
unstable; contact line present, droplet detached from the wall, or film), and
where the oracle measured an apparent angle the FP32 angle must be within
0.5 deg of it.  Both FP32 paths run the sweep: the single-domain fused kernel
one case at a time, and the batched kernel with all cases in one batch."""
import os

import numpy as np
import pytest

from paper_1501_05430_gb300 import inputs as I
from paper_1501_05430_gb300 import lbm as L

from helpers import Case

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "c2_oracle_angles.txt")
ANGLE_TOL_DEG = 0.5
SPEED_RTOL = 0.05


def _golden():
    rows = []
    cols = None
    for line in open(GOLDEN):
        if line.startswith("# method"):
            cols = line[2:].split()
            continue
        if line.startswith("#") or not line.strip():
            continue
        rows.append(dict(zip(cols, line.split())))
    return rows


def _case(row):
    geo = row["method"] == "geometric"
    w = I.single_droplet(float(row["theta_set"]) if geo else 90.0)
    c = Case(w.nx, w.ny, t_over_tc=w.t_over_tc, tau=w.tau, theta=w.theta, rates=w.rates, eos=w.eos, A=w.A,
             kappa=w.kappa, precision=32, kernel=L.LBM_KERNEL_FUSED, wetting=0 if geo else 1,
             G_w=float(row["G_w"]))
    c.orc.close()
    c.rho0 = I.droplet_field(w.nx, w.ny, w.droplets, c.rho_v, c.rho_l, w.width)
    c.steps = int(row["steps"])
    return c


def _classify(sim, c):
    """(status, contact, theta_deg, max_u) of a finished run, as the oracle script classifies it."""
    st = sim.status()
    if st != 0:
        return "unstable", "-", float("nan"), float("nan")
    umax = sim.max_speed()
    try:
        th = np.degrees(sim.contact_angle(0, 0, c.nx)[0])
        return "stable", "cap", th, umax
    except L.LbmError as e:
        assert e.status == L.LBM_ENOCONTACT
        rho = sim.rho()
        return "stable", "detached" if rho[1].max() < c.rho_mid else "film", float("nan"), umax


def _check(row, got):
    st, contact, th, umax = got
    assert st == row["status"], (row, got)
    assert contact == row["contact"], (row, got)
    if contact == "cap":
        assert abs(th - float(row["theta"])) <= ANGLE_TOL_DEG, (row, got)
    if st == "stable":
        assert abs(umax - float(row["max_u"])) <= SPEED_RTOL * float(row["max_u"]), (row, got)


@pytest.mark.parametrize("row", _golden(), ids=lambda r: f"{r['method']}-{r['theta_set']}-{r['G_w']}")
def test_fused_step_matches_oracle_sweep(row):
    c = _case(row)
    with L.Lbm(c.nx, c.ny, c.geos, c.T, c.tau, theta=c.theta, params=c.params, torch_state=False) as s:
        assert s.info.kernel_in_use == L.LBM_KERNEL_FUSED
        s.set_rho(c.rho0)
        try:
            s.step(c.steps)
        except L.LbmError as e:
            assert e.status == L.LBM_EUNSTABLE
        _check(row, _classify(s, c))


def test_batched_sweep_matches_oracle_sweep():
    rows = _golden()
    cases = [_case(r) for r in rows]
    steps = {c.steps for c in cases}
    assert len(steps) == 1
    with L.LbmBatch([c.desc() for c in cases]) as b:
        for c, inst in zip(cases, b.instances):
            inst.set_rho(c.rho0)
        b.step(steps.pop())
        for r, c, inst in zip(rows, cases, b.instances):
            _check(r, _classify(inst, c))
