"""Batched persistent sweep (lbm_batch_*), through the C ABI.

* every instance of a mixed batch (sizes, EOS, temperatures, rates, wetting
  rule, angle fields) against the FP64 oracle run alone;
* results independent of the launch shape (threads, stages, band height,
  steps per launch, CUDA graph) and equal to a lone context's FP32 step;
* an unstable instance is flagged and frozen while the others go on;
* a barrier wait that nothing releases ends in LBM_ETIMEOUT within its bound,
  and the device stays usable;
* the autotuner leaves the state untouched.
"""
import time

import numpy as np
import pytest

from paper_1501_05430_gb300 import inputs as I
from paper_1501_05430_gb300 import lbm as L

from helpers import Case

pytestmark = pytest.mark.gpu

PW10 = (0.25, -0.02, 0.3, 1.1216073327407194, 9.540106186999981)
SPECS = [
    (128, 24, dict(theta="random")),
    (100, 20, dict(theta="random", n_iter=0)),
    (260, 18, dict(wetting=1, G_w=-0.2)),
    (36, 12, dict(eos="pw", pw=PW10, theta="random")),
    (512, 16, dict(rates=dict(s_e=0.8, s_eps=0.9, s_j=1.0, s_q=1.1), kappa=0.9, A=-0.3, theta="random")),
    (132, 24, dict(t_over_tc=0.55, tau=0.7, rates=dict(s_e=0.8, s_eps=0.8, s_j=1.0, s_q=1.1), theta="random")),
    (64, 9, dict(theta="random", n_iter=8, tau=0.7)),
    (384, 14, dict(theta="random", t_over_tc=0.7, tau=0.9)),
    (4, 5, dict(theta="random")),            # the smallest instance: one lane pair per row, 16 ring slots
    (12, 6, dict(wetting=1, G_w=-0.1)),
]


def _cases(specs=SPECS, seed=3):
    rng = np.random.default_rng(seed)
    out = []
    for k, (nx, ny, kw) in enumerate(specs):
        kw = dict(kw)
        if kw.get("theta") == "random":
            kw["theta"] = rng.uniform(np.deg2rad(20), np.deg2rad(160), (ny, nx))
        c = Case(nx, ny, precision=32, **kw)
        rho = I.droplet_field(nx, ny, [(nx * 0.3, ny * 0.35, 0), (nx * 0.75, ny * 0.3, 1)], c.rho_v, c.rho_l)
        c.f0 = I.random_distributions(rho, seed + k)
        c.orc.set_f(c.f0)
        out.append(c)
    return out


def _batch(cases, stream=None, **cfg):
    b = L.LbmBatch([c.desc() for c in cases], L.lbm_batch_config_default(**cfg), stream=stream)
    for c, inst in zip(cases, b.instances):
        inst.set_f(c.f0)
    return b


def _close(cases):
    for c in cases:
        c.orc.close()


@pytest.mark.parametrize("threads", [256, 128])
def test_every_instance_matches_the_oracle(threads):
    """Mixed batch, several items per instance (cross-CTA barriers), an odd
    number of steps per launch: every instance's f against the oracle.  With
    128 threads the instances up to 256 wide run in a launch of their own."""
    cases = _cases()
    with _batch(cases, band_rows=[4, 4, 4, 4], steps_per_launch=5, threads=threads) as b:
        assert b.plan()["items"] > len(cases)
        b.step(12)
        st, inst = b.status()
        assert st == 0 and (inst == 0).all()
        for c, g in zip(cases, b.instances):
            assert c.orc.step(12) == 0
            fo, fg = c.orc.get_f(), g.f()
            assert np.abs(fg - fo).max() < 2e-5 * np.abs(fo).max(), (c.nx, c.ny)
    _close(cases)


SHAPES = [
    dict(),
    dict(stages=3, band_rows=[1, 1, 1, 1], steps_per_launch=1),
    dict(stages=6, band_rows=[64, 64, 64, 64], steps_per_launch=3),
    dict(stages=5, band_rows=[2, 7, 3, 5], steps_per_launch=16, ctas_per_sm=1),
    dict(threads=256, steps_per_launch=4, stages=4),
    dict(steps_per_launch=2, graph_launches=3),
    dict(threads=128),
    dict(threads=128, stages=3, band_rows=[2, 7, 3, 5], steps_per_launch=5, graph_launches=2),
    dict(threads=128, stages=5, band_rows=[1, 64, 4, 16], steps_per_launch=1, ctas_per_sm=1),
]


def test_results_do_not_depend_on_the_launch_shape():
    import torch

    cases = _cases()
    ref = None
    stream = torch.cuda.Stream()
    for cfg in SHAPES:
        with _batch(cases, stream=stream, **cfg) as b:
            b.step(10)
            b.step(7)
            assert b.status()[0] == 0
            fs = [g.f() for g in b.instances]
        if ref is None:
            ref = fs
        else:
            for a, r in zip(fs, ref):
                assert np.array_equal(a, r), cfg
    _close(cases)


SPECS_CS = [
    (512, 20, dict(theta="random", rates=dict(s_e=0.8, s_eps=0.8, s_j=1.0, s_q=1.1), t_over_tc=0.6)),
    (512, 12, dict(theta="random", tau=0.8)),
    (384, 16, dict(theta="random", t_over_tc=0.7, tau=0.9)),
    (128, 24, dict(theta="random")),
    (256, 10, dict(theta="random", tau=0.7)),
]


@pytest.mark.parametrize("threads", [256, 128])
def test_specialised_kernels_match_the_generic_one(threads):
    """A launch whose instances all share the Carnahan-Starling EOS and
    geometric wetting runs the kernel with both fixed at compile time (and its
    512-wide instances a sweep with the width fixed too).  The same instances
    next to one Martys-Chen instance run the generic kernel; instances do not
    interact, so every shared instance must come out with the same bits."""
    cases = _cases(SPECS_CS, seed=11)
    extra = _cases([(36, 12, dict(wetting=1, G_w=-0.1))], seed=12)
    with _batch(cases, band_rows=[4, 8, 8, 8], steps_per_launch=4, threads=threads) as a, \
            _batch(cases + extra, band_rows=[4, 8, 8, 8], steps_per_launch=4, threads=threads) as b:
        a.step(9)
        b.step(9)
        assert a.status()[0] == 0 and b.status()[0] == 0
        for ga, gb in zip(a.instances, b.instances):
            assert np.array_equal(ga.f(), gb.f())
        # and the specialised run against the oracle
        for c, g in zip(cases, a.instances):
            assert c.orc.step(9) == 0
            fo, fg = c.orc.get_f(), g.f()
            assert np.abs(fg - fo).max() < 2e-5 * np.abs(fo).max(), (c.nx, c.ny)
    _close(cases + extra)


def test_graph_replays_are_counted_and_match_direct_launches():
    import torch

    cases = _cases()[:3]
    stream = torch.cuda.Stream()
    with _batch(cases, stream=stream, steps_per_launch=2, graph_launches=4) as g, \
            _batch(cases, stream=stream, steps_per_launch=2) as d:
        g.step(19)  # two graph replays (8 steps each) + 3 direct steps
        d.step(19)
        assert g.launches() == d.launches() == 10
        for a, b_ in zip(g.instances, d.instances):
            assert np.array_equal(a.f(), b_.f())
    # split shape: the 128- and 100-wide instances in 128-thread CTAs, the
    # 260-wide one in 256-thread CTAs: two kernels per launch of the batch
    with _batch(cases, stream=stream, steps_per_launch=2, graph_launches=4, threads=128) as g, \
            _batch(cases, stream=stream, steps_per_launch=2, threads=128) as d:
        g.step(19)
        d.step(19)
        assert g.launches() == d.launches() == 20
        plan = g.plan()
        assert plan["items"] == sum(-(-(c.ny - 2) // 32) for c in cases)
        for a, b_ in zip(g.instances, d.instances):
            assert np.array_equal(a.f(), b_.f())
    _close(cases)


def test_batch_equals_lone_fused_context():
    """The 400 x 200 single-droplet workload inside a batch against the same
    case run alone by lbm_step's fused kernel: the same per-node operations
    (packed two-node form in both), so the same bits."""
    w = I.single_droplet(60.0)
    c = Case(w.nx, w.ny, t_over_tc=w.t_over_tc, tau=w.tau, theta=w.theta, rates=w.rates, eos=w.eos,
             precision=32, kernel=L.LBM_KERNEL_FUSED)
    rho = I.droplet_field(w.nx, w.ny, w.droplets, c.rho_v, c.rho_l, w.width)
    others = _cases()[:2]
    with L.LbmBatch([c.desc()] + [o.desc() for o in others]) as b, \
            L.Lbm(w.nx, w.ny, c.geos, c.T, c.tau, theta=c.theta, params=c.params, torch_state=False) as lone:
        assert lone.info.kernel_in_use == L.LBM_KERNEL_FUSED
        b[0].set_rho(rho)
        lone.set_rho(rho)
        for o, inst in zip(others, b.instances[1:]):
            inst.set_f(o.f0)
        b.step(500)
        lone.step(500)
        rb, rl = b[0].rho(), lone.rho()
        assert np.array_equal(rb, rl)
    _close(others)
    c.orc.close()


def test_unstable_instance_is_frozen_and_others_go_on():
    cases = _cases()[:4]
    bad = cases[1].f0.copy()
    bad[:, 5, 7] = np.nan
    with _batch(cases, band_rows=[4, 4, 4, 4], steps_per_launch=3) as b, _batch(cases) as ok:
        b[1].set_f(bad)
        b.step(9)
        ok.step(9)
        st, inst = b.status()
        assert st == 0
        assert inst[1] == L.LBM_EUNSTABLE and inst[0] == inst[2] == inst[3] == 0
        assert b[1].status() == L.LBM_EUNSTABLE
        for k in (0, 2, 3):
            assert np.array_equal(b[k].f(), ok[k].f())
        # computed work: every fluid node of every step for the stable
        # instances; the frozen one stops inside its first step (the NaN is
        # found there; items of that step that start after the flag skip too)
        upd = b.node_updates()
        for k in (0, 2, 3):
            assert upd[k] == cases[k].nx * (cases[k].ny - 2) * 9
        assert 0 < upd[1] <= cases[1].nx * (cases[1].ny - 2)
        assert upd[1] % cases[1].nx == 0
    _close(cases)


def test_unreleased_barrier_times_out_and_device_stays_usable():
    """Instance 1's first work item never arrives at its barrier; the waits
    on it run out after 0.2 s and the step returns LBM_ETIMEOUT."""
    cases = _cases()[:3]
    b = _batch(cases, band_rows=[4, 4, 4, 4], steps_per_launch=4, wait_seconds=0.2, hold_instance=1)
    t0 = time.perf_counter()
    st = L.load().lbm_batch_step(b.b, 8)
    dt = time.perf_counter() - t0
    assert st == L.LBM_ETIMEOUT
    assert dt < 10.0
    st, inst = b.status()
    assert st == L.LBM_ETIMEOUT and inst[1] == L.LBM_ETIMEOUT
    assert L.load().lbm_batch_step(b.b, 1) == L.LBM_ETIMEOUT  # failed for good
    b.close()
    # a fresh batch on the same device runs and matches the oracle
    with _batch(cases) as b2:
        b2.step(3)
        for c, g in zip(cases, b2.instances):
            assert c.orc.step(3) == 0
            fo = c.orc.get_f()
            assert np.abs(g.f() - fo).max() < 2e-5 * np.abs(fo).max()
    _close(cases)


def test_autotune_keeps_the_state_and_installs_a_valid_shape():
    cases = _cases()
    with _batch(cases) as b, _batch(cases) as ref:
        b.step(3)
        ref.step(3)
        before = [g.f() for g in b.instances]
        best = b.autotune(trial_steps=4)
        assert best.threads in (128, 256) and best.steps_per_launch >= 1
        after = [g.f() for g in b.instances]
        for x, y in zip(before, after):
            assert np.array_equal(x, y)
        assert b.status()[0] == 0
        b.step(5)
        ref.step(5)
        for x, y in zip(b.instances, ref.instances):
            assert np.array_equal(x.f(), y.f())
        # the trials' steps are not counted as the caller's work
        want = np.array([c.nx * (c.ny - 2) * 8 for c in cases], dtype=np.uint64)
        assert np.array_equal(b.node_updates(), want)
        assert np.array_equal(ref.node_updates(), want)
    _close(cases)


def test_instance_contexts_support_the_full_api():
    cases = _cases()[:2]
    with _batch(cases) as b:
        b.step(4)
        img = b[0].save()
        m = b[0].mass()
        assert abs(m - cases[0].orc.mass()) / m < 1e-5
        b.step(3)
        b[0].load(img)
        b.step(3)
        b2f = b[0].f()
        b[0].load(img)
        b[0].step(3)  # the instance alone, through lbm_step
        assert np.abs(b[0].f() - b2f).max() <= 1e-6 * np.abs(b2f).max()
    _close(cases)


def test_invalid_batches_rejected():
    c = _cases()[:1][0]
    d = c.desc()
    for bad in (dict(nx=130), dict(ny=4)):
        dd = dict(d, **bad)
        dd["theta"] = None
        with pytest.raises(L.LbmError):
            L.LbmBatch([dd])
    with pytest.raises(L.LbmError):
        L.LbmBatch([d], L.lbm_batch_config_default(threads=96))
    with pytest.raises(L.LbmError):
        L.LbmBatch([d], L.lbm_batch_config_default(stages=9))
    c.orc.close()
