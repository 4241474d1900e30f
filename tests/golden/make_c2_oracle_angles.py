"""Write c2_oracle_angles.txt: the FP64 oracle's apparent contact angle and
maximum speed for the 400 x 200 single-droplet sweep (inputs.single_droplet),
geometric wetting (Eqs. 19-21, four iterations) at theta_set in {30, 60, 90,
120, 150} deg and Martys-Chen wetting (Eq. 14) on a fixed grid of G_w values.
For the geometric runs also the share of boundary-row ghost densities at the
lower clamp 0 of Eqs. 19-21 (mean of samples every 1000 steps over the last
10,000 steps), overall and within 10 nodes of a contact line.

Calls only the oracle (and the seeded input generators).  Every run is
independent; they run in parallel worker processes.

  python tests/golden/make_c2_oracle_angles.py [--steps 20000] [--jobs 8]
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
OUT = os.path.join(HERE, "c2_oracle_angles.txt")
THETAS = (30.0, 60.0, 90.0, 120.0, 150.0)
G_WS = (0.0, -0.1, -0.16, -0.17, -0.25)


def run(job):
    sys.path.insert(0, ROOT)
    import numpy as np

    import oracle as O
    from paper_1501_05430_gb300 import inputs as I

    method, theta_deg, g_w, steps = job
    w = I.single_droplet(theta_deg if method == "geometric" else 90.0)
    e = w.eos
    oeos = O.carnahan_starling(e["a"], e["b"], e["R"])
    T = w.t_over_tc * O.cs_critical(oeos)[0]
    rv, rl = O.coexistence(oeos, T)
    rm = O.rho_max(oeos, T, rl)
    inv = 1.0 / w.tau
    r = dict(s_rho=0.0, s_e=inv, s_eps=inv, s_j=inv, s_q=inv, s_nu=inv)
    r.update({k: v for k, v in w.rates.items() if v})
    sim = O.Sim(w.nx, w.ny, oeos, T, tau=w.tau, theta=w.theta, rates=r, rho_max_=rm, A=w.A, kappa=w.kappa,
                G_w=g_w, wetting=O.GEOMETRIC if method == "geometric" else O.MARTYS_CHEN)
    sim.set_rho(I.droplet_field(w.nx, w.ny, w.droplets, rv, rl, w.width))
    m0 = sim.mass()
    rho_mid = 0.5 * (rv + rl)
    half, t0 = steps // 2, time.perf_counter()
    th_half = float("nan")
    zero_all, zero_cl = [], []
    st = 0
    for k in range(steps // 1000):
        st = sim.step(1000)
        if st != 0:
            break
        done = (k + 1) * 1000
        if done == half:
            try:
                th_half = np.degrees(sim.contact_angle(0, 0, w.nx, rho_mid)[0])
            except ValueError:
                pass
        if method == "geometric" and done > steps - 10000:
            fr = sim.fields()["rho"]
            g = fr[0]
            zero_all.append(float((g == 0.0).mean()))
            b = fr[1] >= rho_mid
            near = np.zeros(w.nx, dtype=bool)
            for c in np.nonzero(b != np.roll(b, 1))[0]:
                near[np.arange(c - 10, c + 11) % w.nx] = True
            zero_cl.append(float((g[near] == 0.0).mean()) if near.any() else float("nan"))
    if st == 0 and steps % 1000:
        st = sim.step(steps % 1000)
    row = dict(method=method, theta_set=theta_deg if method == "geometric" else float("nan"), G_w=g_w,
               steps=steps, status="stable" if st == 0 else "unstable", contact="-", theta_half=th_half,
               theta=float("nan"), H=float("nan"), L=float("nan"), max_u=float("nan"), mass_drift=float("nan"),
               ghost0_all=float(np.mean(zero_all)) if zero_all else float("nan"),
               ghost0_contact=float(np.nanmean(zero_cl)) if zero_cl and not np.all(np.isnan(zero_cl)) else float("nan"),
               seconds=0.0)
    if st == 0:
        rho, ux, uy = sim.macro()
        try:
            th, H, L, _ = sim.contact_angle(0, 0, w.nx, rho_mid)
            row.update(theta=np.degrees(th), H=H, L=L, contact="cap")
        except ValueError:
            # no rho_mid crossing on the boundary row: the droplet left the wall
            # (180 deg) or spread into a film (0 deg)
            row["contact"] = "detached" if rho[1].max() < rho_mid else "film"
        row["max_u"] = float(np.sqrt(ux[1:-1] ** 2 + uy[1:-1] ** 2).max())
        row["mass_drift"] = abs(sim.mass() - m0) / m0
    row["seconds"] = time.perf_counter() - t0
    sim.close()
    return row


COLS = ("method", "theta_set", "G_w", "steps", "status", "contact", "theta_half", "theta", "H", "L", "max_u", "mass_drift",
        "ghost0_all", "ghost0_contact")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--jobs", type=int, default=min(10, os.cpu_count() or 1))
    args = ap.parse_args()
    jobs = [("geometric", t, 0.0, args.steps) for t in THETAS] + [("martys_chen", 90.0, g, args.steps) for g in G_WS]
    with mp.get_context("spawn").Pool(args.jobs) as pool:
        rows = pool.map(run, jobs)
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle, single droplet 400 x 200: Carnahan-Starling a = 0.25, b = 4, R = 1, T/Tc = 0.6,\n"
                 "# tau = 0.8 with MRT rates s_e = s_eps = 0.8, s_j = 1, s_q = 1.1, A = -0.9, kappa = 0.5, the\n"
                 "# droplet started as the circular cap at theta_set (90 deg for Martys-Chen) with the area of\n"
                 "# the semicircle of radius 60 centred at (200, 1), tanh width 3.  Angles in degrees from the\n"
                 "# rho_mid contour (circular cap, bottom wall, columns 0..399); theta_half after steps/2.\n"
                 "# ghost0_all / ghost0_contact: share of boundary-row ghost densities at the lower clamp 0\n"
                 "# (geometric runs; mean over the last 10,000 steps; all nodes / within 10 of a contact line).\n"
                 "# geometric: Eqs. 19-21 with four iterations at theta_set; martys_chen: Eq. 14 at G_w.\n"
                 "# contact: cap (angle measured), detached (no liquid on the boundary row), film (no vapour\n"
                 "# on it).\n"
                 "# Written by tests/golden/make_c2_oracle_angles.py (oracle only).\n")
        fh.write("# " + " ".join(COLS) + "\n")
        for r in rows:
            fh.write(" ".join(f"{r[c]:.10g}" if isinstance(r[c], float) else str(r[c]) for c in COLS) + "\n")
    for r in rows:
        print(r, flush=True)


if __name__ == "__main__":
    main()
