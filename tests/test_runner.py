"""Workload -> library arguments (paper_1501_05430_gb300/runner.py), on CPU
through the library's host-side functions: the EOS and temperature, the
parameters (A, kappa, MRT rates) and the initial field that the benchmark and
the experiments hand to lbm_create / lbm_batch_create."""
import numpy as np
import pytest

import oracle as O
from paper_1501_05430_gb300 import inputs as I
from paper_1501_05430_gb300 import lbm as L
from paper_1501_05430_gb300 import runner as RN


def test_throughput_workload_arguments():
    w = I.throughput(nx=512, ny=256)
    eos, T = RN.lib_eos(w)
    assert eos.kind == 1 and T == 0.0
    assert (eos.rho1, eos.rho2, eos.theta_v, eos.theta_m, eos.theta_l) == (1.325, 971.1017, 0.2, -0.01, 0.33333)
    p = RN.lib_params(w)
    # the paper's relaxation: every rate left at 1/tau (0 = derived), tau = 1
    assert (p.s_e, p.s_eps, p.s_j, p.s_q) == (0.0, 0.0, 0.0, 0.0) and w.tau == 1.0
    assert p.A == -0.6 and p.kappa == 0.5 and p.precision == 32 and p.n_iter == 4


def test_single_droplet_arguments_and_coexistence():
    w = I.single_droplet(60.0)
    eos, T = RN.lib_eos(w)
    assert eos.kind == 0 and (eos.a, eos.b, eos.R) == (0.25, 4.0, 1.0)
    oeos = O.carnahan_starling(0.25, 4.0, 1.0)
    assert T == pytest.approx(0.6 * O.cs_critical(oeos)[0], rel=1e-12)
    p = RN.lib_params(w)
    assert (p.s_e, p.s_eps, p.s_j, p.s_q) == (0.8, 0.8, 1.0, 1.1)
    # the initial field sits at the coexistence densities of the oracle's own solver
    rv, rl = O.coexistence(oeos, T)
    rho = RN.initial_rho(w)
    assert rho.min() == pytest.approx(rv, rel=1e-9) and rho.max() == pytest.approx(rl, rel=1e-6)
    assert RN.rho_mid(w) == pytest.approx(0.5 * (rv + rl), rel=1e-9)


def test_batch_instance_descriptions():
    for w in I.batched(count=8):
        d = RN.instance_desc(w)
        assert (d["nx"], d["ny"], d["tau"]) == (w.nx, w.ny, w.tau) and d["theta"] is w.theta
        assert d["params"].precision == 32
        Tc, _ = L.lbm_eos_critical(d["eos"])
        assert d["T"] == pytest.approx(w.t_over_tc * Tc, rel=1e-12)
        assert np.isclose(d["eos"].a, 0.25)
