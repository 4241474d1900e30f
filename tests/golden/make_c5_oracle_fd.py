"""Write c5_oracle_fd.txt: FP64 central finite differences of the wall-angle
inversion loss of inputs.adjoint_case, computed with the C oracle only, for 15
bottom-wall angles and the EOS temperature T, each over a ladder of step sizes
with a noise estimate.

Which angles.  The gradient in a wall angle is large only where Eqs. 19-21 act,
next to the two contact lines (in the bulk, a = 0 and the ghost density equals
rho(i, 2) whatever theta is), and it falls to 1e-6 .. 1e-3 elsewhere, where a
finite difference is mostly rounding noise.  The candidates are the wall nodes
within 12 of the initial contact lines (x = 88 and 168).

Which step.  The loss is only piecewise smooth: along the trajectory some
boundary-row ghost densities sit at the lower clamp 0 of Eqs. 19-21 in some
steps, and which ones switches as a parameter moves, so L has kinks whose
spacing in theta can be below 1e-4.  A central difference over a step wider
than that spacing averages slopes across kinks: at theta_167 it reads 4058.35
with h = 1e-4 and 4058.39 with h = 5e-5, but 4151.01 (1e-5), 4152.274 (1e-6),
4152.2856 (1e-7), 4152.2863 (1e-8) -- the derivative is 4152.29.  Each
parameter is therefore differenced over a ladder of steps (theta: 1e-4, the
configuration's step, then 1e-5, 1e-6, 1e-7; T: 1e-7, 1e-8, 1e-9) and the
stored derivative is the middle rung's (theta: h = 1e-6; T: h = 1e-8), with
the noise estimate
    err = max(|fd(mid) - fd(coarser)|, |fd(mid) - fd(finer)|)
which bounds truncation and kink averaging from one side and rounding from the
other.  A candidate angle is eligible when err <= 1e-4 |fd|, i.e. a 1e-3
relative check of it is meaningful; 15 of the eligible ones are drawn with a
fixed seed.  fd at h = 1e-4 is stored too, for reference.

The target profile (h*, W*) is the oracle's final density at the second seeded
angle field; it is stored too, so that any implementation can evaluate the
same loss.  Runs are independent and execute in parallel worker processes
(about 400 oracle runs of 25 s each).

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
H_THETA = (1e-4, 1e-5, 1e-6, 1e-7)  # ladder; the stored derivative is at 1e-6
MID_THETA = 2
H_T = (1e-7, 1e-8, 1e-9)             # ladder; the stored derivative is at 1e-8
MID_T = 1
N_THETA = 15
SAMPLE_SEED = 9
WINDOW = 12            # candidates: wall nodes within this distance of an initial contact line
ELIGIBLE_NOISE = 1e-4  # eligible when err <= this x |fd|


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


def ladder(fds, mid):
    """(fd at the middle rung, its noise estimate)."""
    err = max(abs(fds[mid] - fds[k]) for k in (mid - 1, mid + 1) if 0 <= k < len(fds))
    return fds[mid], err


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--jobs", type=int, default=min(8, os.cpu_count() or 1))
    args = ap.parse_args()
    np, O, I, c, eos, T, rv, rl, rm, rho0 = _setup()
    cand = candidates(c)
    runs = [(c["theta_target"], T), (c["theta"], T)]
    for i in cand:
        for h in H_THETA:
            for sgn in (1.0, -1.0):
                th = c["theta"].copy()
                th[i] += sgn * h
                runs.append((th, T))
    for h in H_T:
        runs += [(c["theta"], T + h), (c["theta"], T - h)]
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        rhos = pool.map(final_rho, runs, chunksize=1)
    h_t, W_t = I.profile(rhos[0], rv, rl)

    def loss(rho):
        return I.profile_loss_grad(rho, h_t, W_t, rv, rl)[0]

    L0 = loss(rhos[1])
    k = 2
    theta_rows = []
    for i in cand:
        fds = []
        for h in H_THETA:
            fds.append((loss(rhos[k]) - loss(rhos[k + 1])) / (2 * h))
            k += 2
        fd, err = ladder(fds, MID_THETA)
        theta_rows.append((i, fd, err, fds))
    fdT = []
    for h in H_T:
        fdT.append((loss(rhos[k]) - loss(rhos[k + 1])) / (2 * h))
        k += 2
    fT, errT = ladder(fdT, MID_T)
    eligible = [r for r in theta_rows if r[2] <= ELIGIBLE_NOISE * abs(r[1])]
    if len(eligible) < N_THETA:
        raise RuntimeError(f"only {len(eligible)} eligible angles")
    pick = np.random.default_rng(SAMPLE_SEED).choice(len(eligible), N_THETA, replace=False)
    rows = [("theta", r[0], r[1], r[2], r[3][0]) for r in (eligible[j] for j in sorted(pick))]
    rows.append(("T", -1, fT, errT, fdT[0]))
    with open(OUT, "w") as fh:
        fh.write("# Central finite differences of the inversion loss of inputs.adjoint_case"
                 " (256 x 128, CS a = 1, b = 4, R = 1, T/Tc = 0.7, tau = 1, R0 = 40, 2000 steps), FP64 C oracle.\n"
                 f"# Step ladders: theta {H_THETA}, derivative at {H_THETA[MID_THETA]!r}; T {H_T}, derivative at"
                 f" {H_T[MID_T]!r}.  err = max |fd(mid) - fd(neighbour rung)| (noise estimate).\n"
                 f"# {len(eligible)} of {len(cand)} candidate angles (within {WINDOW} of the initial contact lines) had"
                 f" err <= {ELIGIBLE_NOISE!r} |fd|; {N_THETA} drawn with seed {SAMPLE_SEED}.\n"
                 f"# T = {T!r}  rho_v = {rv!r}  rho_l = {rl!r}  loss = {L0!r}\n"
                 f"# W_target = {W_t!r}\n"
                 "# h_target (256 values):\n")
        fh.write("# " + " ".join(repr(float(v)) for v in h_t) + "\n")
        fh.write("# Written by tests/golden/make_c5_oracle_fd.py (oracle only).\n")
        fh.write("# candidates: index fd at each theta rung\n")
        for i, _, _, fds in theta_rows:
            fh.write(f"# cand {i} " + " ".join(repr(v) for v in fds) + "\n")
        fh.write("# T rungs: " + " ".join(repr(v) for v in fdT) + "\n")
        fh.write("# param index dL/dparam err fd_at_coarsest_rung\n")
        for name, i, fd, err, coarse in rows:
            fh.write(f"{name} {i} {fd!r} {err!r} {coarse!r}\n")
    print(open(OUT).read()[-3000:])


if __name__ == "__main__":
    main()
