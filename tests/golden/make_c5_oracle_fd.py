"""Write c5_oracle_fd.txt: FP64 central finite differences of the wall-angle
inversion loss of inputs.adjoint_case, computed with the C oracle only, for 15
bottom-wall angles (h = 1e-4) and the EOS temperature T (h = 1e-8), each with a
noise estimate from a second step size.

Which angles.  The gradient in a wall angle is large only where Eqs. 19-21 act,
next to the two contact lines (in the bulk, a = 0 and the ghost density equals
rho(i, 2) whatever theta is), and it falls to 1e-6 .. 1e-3 elsewhere, where a
finite difference is mostly rounding noise.  The candidates are therefore the
wall nodes within 12 of the initial contact lines (x = 88 and 168); each is
differenced with h and h/2, and the noise estimate of a row is
    err = |fd(h) - fd(h/2)|
(truncation error falls by 4 and rounding noise doubles from h to h/2, so err
bounds both to within a small factor).  A candidate is eligible when
err <= 1e-5 |fd(h)|, i.e. a 1e-3 relative check of that row is meaningful; 15
of the eligible ones are drawn with a fixed seed.

T takes the small step because the loss is only piecewise smooth in T: along
this trajectory a bottom-wall ghost density is clamped at 0 in most steps
(Eqs. 19-21 return a negative density on a hydrophobic node next to the contact
line), and the clamp switches on and off as T moves, so a central difference
over 2e-4 in T straddles kinks (it reads 0.6% above the derivative; with
h = 1e-5 .. 1e-6 it wanders by 5%).  At h = 1e-8 no clamp changes state; its
second step is 5e-9.

The target profile (h*, W*) is the oracle's final density at the second seeded
angle field; it is stored too, so that any implementation can evaluate the
same loss.  Runs are independent and execute in parallel worker processes
(about 200 oracle runs of 25 s each).

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
WINDOW = 12          # candidates: wall nodes within this distance of an initial contact line
ELIGIBLE_NOISE = 1e-5  # eligible when err <= this x |fd|


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


def candidates(c):
    xc, r0, _ = c["droplet"]
    lines = (int(round(xc - r0)), int(round(xc + r0)))
    return sorted({x for x0 in lines for x in range(x0 - WINDOW, x0 + WINDOW + 1)})


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=min(8, os.cpu_count() or 1))
    args = ap.parse_args()
    np, O, I, c, eos, T, rv, rl, rm, rho0 = _setup()
    cand = candidates(c)
    runs = [(c["theta_target"], T), (c["theta"], T)]
    steps = (H, H / 2)
    for i in cand:
        for h in steps:
            for sgn in (1.0, -1.0):
                th = c["theta"].copy()
                th[i] += sgn * h
                runs.append((th, T))
    for h in (H_T, H_T / 2):
        runs += [(c["theta"], T + h), (c["theta"], T - h)]
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        rhos = pool.map(final_rho, runs)
    h_t, W_t = I.profile(rhos[0], rv, rl)

    def loss(rho):
        return I.profile_loss_grad(rho, h_t, W_t, rv, rl)[0]

    L0 = loss(rhos[1])
    k = 2
    theta_rows = []
    for i in cand:
        fd = []
        for h in steps:
            fd.append((loss(rhos[k]) - loss(rhos[k + 1])) / (2 * h))
            k += 2
        theta_rows.append((i, fd[0], fd[1], abs(fd[0] - fd[1])))
    fdT = []
    for h in (H_T, H_T / 2):
        fdT.append((loss(rhos[k]) - loss(rhos[k + 1])) / (2 * h))
        k += 2
    eligible = [r for r in theta_rows if r[3] <= ELIGIBLE_NOISE * abs(r[1])]
    if len(eligible) < N_THETA:
        raise RuntimeError(f"only {len(eligible)} eligible angles")
    pick = np.random.default_rng(SAMPLE_SEED).choice(len(eligible), N_THETA, replace=False)
    rows = [("theta",) + eligible[j] for j in sorted(pick)]
    rows.append(("T", -1, fdT[0], fdT[1], abs(fdT[0] - fdT[1])))
    with open(OUT, "w") as fh:
        fh.write("# Central finite differences of the inversion loss of inputs.adjoint_case"
                 " (256 x 128, CS a = 1, b = 4, R = 1, T/Tc = 0.7, tau = 1, R0 = 40, 2000 steps), FP64 C oracle.\n"
                 f"# theta: h = {H!r} and h/2; T: h = {H_T!r} and h/2.  err = |fd(h) - fd(h/2)| (noise estimate).\n"
                 f"# {len(eligible)} of {len(cand)} candidate angles (within {WINDOW} of the initial contact lines) had"
                 f" err <= {ELIGIBLE_NOISE!r} |fd|; {N_THETA} drawn with seed {SAMPLE_SEED}.\n"
                 f"# T = {T!r}  rho_v = {rv!r}  rho_l = {rl!r}  loss = {L0!r}\n"
                 f"# W_target = {W_t!r}\n"
                 "# h_target (256 values):\n")
        fh.write("# " + " ".join(repr(float(v)) for v in h_t) + "\n")
        fh.write("# Written by tests/golden/make_c5_oracle_fd.py (oracle only).\n")
        fh.write("# candidates: index fd(h) fd(h/2)\n")
        for i, f1, f2, _ in theta_rows:
            fh.write(f"# cand {i} {f1!r} {f2!r}\n")
        fh.write("# param index dL/dparam(h) dL/dparam(h/2) err\n")
        for name, i, f1, f2, err in rows:
            fh.write(f"{name} {i} {f1!r} {f2!r} {err!r}\n")
    print(open(OUT).read()[-3000:])


if __name__ == "__main__":
    main()
