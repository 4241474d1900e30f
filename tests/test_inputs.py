"""The seeded input recipes (paper_1501_05430_gb300/inputs.py) that feed both
the oracle and the GPU path: each does what its docstring states, the same
way for the same seed, and Table 1 there is the paper's Table 1 (Sec. 3.1) as
the golden fixture prints it."""
import os

import numpy as np
import pytest

from paper_1501_05430_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_piecewise_eos.txt")


def test_table1_is_the_golden_fixture():
    rows = [line.split() for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    assert len(rows) == 3
    for ratio, r1, r2, tv, tm, tl in rows:
        assert I.TABLE1[int(ratio)] == (float(r1), float(r2), float(tv), float(tm), float(tl))
        e = I.table1_eos(int(ratio))
        assert (e["rho1"], e["rho2"], e["theta_v"], e["theta_m"], e["theta_l"]) == \
               (float(r1), float(r2), float(tv), float(tm), float(tl))


def test_droplet_field_is_a_tanh_profile_with_periodic_x():
    nx, ny, rv, rl, R, w = 64, 40, 0.1, 5.0, 10.0, 3.0
    rho = I.droplet_field(nx, ny, [(2.0, R, 0)], rv, rl, w)
    assert rho.min() >= rv and rho.max() <= rl
    # centre on the boundary row y = 1; the profile depends on the periodic distance only
    assert rho[1, 2] == pytest.approx(0.5 * (rl + rv) - 0.5 * (rl - rv) * np.tanh(-2.0 * R / w))
    assert np.allclose(rho[:, 2 - 1], rho[:, 2 + 1]) and np.allclose(rho[:, (2 - 5) % nx], rho[:, 2 + 5])
    mid = 0.5 * (rl + rv)
    assert np.all(np.diff(rho[1, 2:2 + nx // 2]) <= 0)           # falls with the distance
    assert abs(rho[1, int(2 + R)] - mid) < 1e-12 * rl              # the mid density at r = R
    top = I.droplet_field(nx, ny, [(30.0, R, 1)], rv, rl, w)
    assert np.array_equal(top[::-1], I.droplet_field(nx, ny, [(30.0, R, 0)], rv, rl, w))


def test_theta_field_rows():
    th = I.theta_field(8, 6, np.linspace(0.1, 0.8, 8), 0.3)
    assert np.array_equal(th[0], np.linspace(0.1, 0.8, 8)) and np.all(th[-1] == 0.3)
    assert np.all(th[1:-1] == np.pi / 2)


def test_random_distributions_perturb_the_rest_shape():
    rho = I.droplet_field(32, 16, [(16.0, 6.0, 0)], 0.2, 3.0)
    f = I.random_distributions(rho, seed=5, amp=0.05)
    assert f.shape == (9, 16, 32) and np.all(f[:, 0] == 0) and np.all(f[:, -1] == 0)
    ratio = f[:, 1:-1] / (I.LATTICE_SHAPE[:, None, None] * rho[None, 1:-1])
    assert ratio.min() >= 0.95 and ratio.max() <= 1.05 and ratio.std() > 0.01
    assert np.array_equal(f, I.random_distributions(rho, seed=5, amp=0.05))
    assert not np.array_equal(f, I.random_distributions(rho, seed=6, amp=0.05))
    assert I.LATTICE_SHAPE.sum() == pytest.approx(1.0)


@pytest.mark.parametrize("nx,ny", [(4096, 2048), (1024, 512)])
def test_throughput_layout(nx, ny):
    w = I.throughput(nx=nx, ny=ny)
    assert w.name == I.throughput(nx=nx, ny=ny).name and np.array_equal(w.theta, I.throughput(nx=nx, ny=ny).theta)
    assert len(w.droplets) == 24 and sum(d[2] == 0 for d in w.droplets) == 12
    assert w.eos == I.table1_eos(1000) and w.tau == 1.0 and w.rates == {}
    for wall in (0, 1):
        regs = [r for r in w.regions if r[0] == wall]
        # the regions tile the wall, in order
        assert regs[0][1] == 0 and regs[-1][2] == nx
        assert all(a[2] == b[1] for a, b in zip(regs, regs[1:]))
        row = w.theta[0 if wall == 0 else -1]
        sets = [t for r, t in zip(w.regions, w.theta_set) if r[0] == wall]
        drops = [d for d in w.droplets if d[2] == wall]
        for (_, a, b), t, (xc, R, _) in zip(regs, sets, drops):
            assert 30.0 <= t <= 150.0
            assert np.allclose(row[a:b], np.deg2rad(t))       # one angle per region
            assert a <= xc < b and 0 < R <= 120.0
            assert I._cap_base(R, t) <= (b - a) + 1.0         # the relaxed cap fits its slot
    assert np.all(w.theta[1:-1] == np.pi / 2)
    if nx == 4096:
        assert "1.0000, 1.0000" in w.notes and all(40.0 <= d[1] <= 120.0 for d in w.droplets)


@pytest.mark.parametrize("wall", [0, 1])
def test_cap_droplet_keeps_the_semicircle_area_and_meets_the_wall_at_theta(wall):
    ny = 120
    for deg in (20.0, 45.0, 90.0, 135.0, 160.0):
        xc, R, yc = I.cap_droplet(50.0, 30.0, deg, wall, ny)
        t = np.deg2rad(deg)
        assert R * R * (t - np.sin(t) * np.cos(t)) == pytest.approx(0.5 * np.pi * 30.0 ** 2, rel=1e-12)
        base = 1.0 if wall == 0 else ny - 2.0
        # the circle crosses the boundary row with half-width R sin(theta), and its
        # centre sits below (acute) or above (obtuse) the row for the bottom wall
        h = abs(base - yc)
        assert np.sqrt(R * R - h * h) == pytest.approx(R * np.sin(t), rel=1e-9)
        if deg != 90.0:
            assert ((yc < base) == (deg < 90.0)) if wall == 0 else ((yc > base) == (deg < 90.0))
    assert I.cap_droplet(50.0, 30.0, 90.0, 0, ny) == pytest.approx((50.0, 30.0, 1.0))


def test_throughput_cs_shares_the_layout():
    a, b = I.throughput(), I.throughput_cs()
    assert np.array_equal(a.theta, b.theta) and a.regions == b.regions and a.theta_set == b.theta_set
    assert b.eos == I.cs_eos(a=0.25) and b.t_over_tc == 0.5 and b.tau == 0.6 and b.A == I.CS_A
    assert b.rates == I.LOW_T_RATES and not _unit(b)
    for (xc, r0, wall), (xc2, R, yc), th in zip(a.droplets, b.droplets, a.theta_set):
        assert (xc2, R, yc) == I.cap_droplet(xc, r0, th, wall, b.ny)


def _unit(w):
    return w.tau == 1.0 and all(v in (0.0, 1.0) for v in w.rates.values())


def test_cap_base_keeps_the_semicircle_area():
    r0 = 50.0
    for deg in (30.0, 60.0, 90.0, 120.0, 150.0):
        t = np.deg2rad(deg)
        base = I._cap_base(r0, deg)
        R = base / (2.0 * np.sin(t)) if deg <= 90.0 else base / 2.0
        area = R * R * (t - np.sin(t) * np.cos(t))
        assert area == pytest.approx(0.5 * np.pi * r0 * r0, rel=1e-12)
    assert I._cap_base(r0, 90.0) == pytest.approx(2.0 * r0)


def test_batched_recipe():
    insts = I.batched()
    assert len(insts) == 256
    again = I.batched()
    for a, b in zip(insts, again):
        assert (a.nx, a.ny, a.t_over_tc, a.tau, a.theta_set) == (b.nx, b.ny, b.t_over_tc, b.tau, b.theta_set)
    sizes = {(w.nx, w.ny) for w in insts}
    assert sizes == {(128, 64), (256, 128), (384, 192), (512, 256)}
    for w in insts:
        assert 20.0 <= w.theta_set[0] <= 160.0 and np.allclose(w.theta[0], np.deg2rad(w.theta_set[0]))
        assert w.t_over_tc in (0.5, 0.6, 0.7, 0.8) and 0.6 <= w.tau <= 1.0
        # the cap at the instance's angle with the area of the semicircle of radius nx/4
        xc, R, yc = w.droplets[0]
        t = np.deg2rad(w.theta_set[0])
        assert len(w.droplets) == 1 and xc == w.nx / 2.0
        assert R * R * (t - np.sin(t) * np.cos(t)) == pytest.approx(0.5 * np.pi * (w.nx / 4.0) ** 2, rel=1e-12)
        assert yc == pytest.approx(1.0 - R * np.cos(t), rel=1e-12)
        assert (w.rates == I.LOW_T_RATES) == (w.t_over_tc < 0.7)
        assert w.eos == I.cs_eos(a=0.25) and w.A == I.CS_A == -0.9


def test_adjoint_case():
    c = I.adjoint_case()
    assert (c["nx"], c["ny"], c["steps"], c["checkpoint_every"]) == (256, 128, 2000, 100)
    for k in ("theta", "theta_target"):
        assert c[k].shape == (256,) and np.deg2rad(45.0) <= c[k].min() and c[k].max() <= np.deg2rad(135.0)
    assert not np.array_equal(c["theta"], c["theta_target"])
    assert np.array_equal(c["theta"], I.adjoint_case()["theta"])


def test_profile_loss_gradient_is_the_derivative():
    rng = np.random.default_rng(3)
    rv, rl = 0.1, 4.0
    rho = rng.uniform(rv, rl, (10, 12))
    h_t, W_t = rng.uniform(0, 5, 12), 3.0
    L0, g = I.profile_loss_grad(rho, h_t, W_t, rv, rl)
    h, W = I.profile(rho, rv, rl)
    assert L0 == pytest.approx(((h - h_t) ** 2).sum() + (W - W_t) ** 2)
    eps = 1e-6
    for (y, x) in [(0, 3), (1, 5), (4, 0), (8, 11), (9, 2)]:
        d = np.zeros_like(rho)
        d[y, x] = eps
        lp = I.profile_loss_grad(rho + d, h_t, W_t, rv, rl)[0]
        lm = I.profile_loss_grad(rho - d, h_t, W_t, rv, rl)[0]
        fd = (lp - lm) / (2 * eps)
        assert g[y, x] == pytest.approx(fd, rel=1e-6, abs=1e-9)
