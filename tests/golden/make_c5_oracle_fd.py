"""Write c5_oracle_fd.txt: FP64 central finite differences of the wall-angle
inversion loss of inputs.adjoint_case, computed with the C oracle only, for 15
seeded bottom-wall angles (h = 1e-4) and the EOS temperature T (h = 1e-8).

T takes the small step because the loss is only piecewise smooth in T: along
this trajectory a bottom-wall ghost density is clamped at 0 in most steps
(Eqs. 19-21 return a negative density on a hydrophobic node next to the contact
line), and the clamp switches on and off as T moves, so a central difference
over 2e-4 in T straddles kinks (it reads 0.6% above the derivative; with
h = 1e-5 .. 1e-6 it wanders by 5%).  At h = 1e-8 no clamp changes state and
the roundoff is ~1e-10 relative.

The target profile (h*, W*) is the oracle's final density at the second seeded
angle field; it is stored too, so that any implementation can evaluate the
same loss.  Runs are independent and execute in parallel worker processes.

  python tests/golden/make_c5_oracle_fd.py [--jobs 8]
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "c5_oracle_fd.txt")
H = 1e-4
H_T = 1e-8
N_THETA = 15
SAMPLE_SEED = 9


def _setup():
    sys.path.insert(0, ROOT)
    import numpy as np

    import oracle as O
    from paper_1501_05430_gb300 import inputs as I

    c = I.adjoint_case()
    eos = O.carnahan_starling(1.0, 4.0, 1.0)
    T = c["t_over_tc"] * O.cs_critical(eos)[0]
    rv, rl = O.coexistence(eos, T)
    rm = O.rho_max(eos, T, rl)
    rho0 = I.droplet_field(c["nx"], c["ny"], [c["droplet"]], rv, rl, c["width"])
    return np, O, I, c, eos, T, rv, rl, rm, rho0


def final_rho(args):
    theta_bottom, T_run = args
    np, O, I, c, eos, T, rv, rl, rm, rho0 = _setup()
    th = np.full((c["ny"], c["nx"]), np.pi / 2)
    th[0] = theta_bottom
    s = O.Sim(c["nx"], c["ny"], eos, T_run, tau=c["tau"], theta=th, rho_max_=rm)
    s.set_rho(rho0)
    st = s.step(c["steps"])
    rho = s.rho()
    s.close()
    if st != 0:
        raise RuntimeError("oracle run unstable")
    return rho


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=min(8, os.cpu_count() or 1))
    args = ap.parse_args()
    np, O, I, c, eos, T, rv, rl, rm, rho0 = _setup()
    idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(c["nx"], N_THETA, replace=False))
    runs = [(c["theta_target"], T), (c["theta"], T)]
    for i in idx:
        for sgn in (1.0, -1.0):
            th = c["theta"].copy()
            th[i] += sgn * H
            runs.append((th, T))
    runs += [(c["theta"], T + H_T), (c["theta"], T - H_T)]
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        rhos = pool.map(final_rho, runs)
    h_t, W_t = I.profile(rhos[0], rv, rl)

    def loss(rho):
        return I.profile_loss_grad(rho, h_t, W_t, rv, rl)[0]

    L0 = loss(rhos[1])
    rows = []
    for k, i in enumerate(idx):
        rows.append(("theta", int(i), (loss(rhos[2 + 2 * k]) - loss(rhos[3 + 2 * k])) / (2 * H)))
    rows.append(("T", -1, (loss(rhos[-2]) - loss(rhos[-1])) / (2 * H_T)))
    with open(OUT, "w") as fh:
        fh.write("# Central finite differences (theta: h = 1e-4, T: h = 1e-8) of the inversion loss of\n"
                 "# inputs.adjoint_case"
                 " (256 x 128, CS a = 1, b = 4, R = 1, T/Tc = 0.7, tau = 1, R0 = 40, 2000 steps), FP64 C oracle.\n"
                 f"# T = {T!r}  rho_v = {rv!r}  rho_l = {rl!r}  loss = {L0!r}\n"
                 f"# W_target = {W_t!r}\n"
                 "# h_target (256 values):\n")
        fh.write("# " + " ".join(repr(float(v)) for v in h_t) + "\n")
        fh.write("# Written by tests/golden/make_c5_oracle_fd.py (oracle only).\n")
        fh.write("# param index dL/dparam\n")
        for name, i, g in rows:
            fh.write(f"{name} {i} {g!r}\n")
    print(open(OUT).read()[-2000:])


if __name__ == "__main__":
    main()
