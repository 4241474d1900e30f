"""Host <-> device density transfers through the C ABI (GPU).

lbm_set_rho reads pinned host memory in place and stages pageable memory
through a device copy; both routes must give the same bits, and lbm_get_rho
must fill pinned and pageable destinations alike.  For FP32 states the
density readback is the left-to-right double sum of the nine populations,
which the kernel evaluates with integer arithmetic whenever that sum is exact;
the inputs below cover both that route and the double-addition fallback (wide
exponent spans, subnormal, infinite and NaN populations) and the boundary
between them.
"""
import numpy as np
import pytest

from paper_1501_05430_gb300 import lbm as L

pytestmark = pytest.mark.gpu


def _pinned(shape):
    import torch

    return torch.empty(shape, dtype=torch.float64, pin_memory=True).numpy()


def _ctx(nx, ny, precision=32):
    eos = L.carnahan_starling()
    T = 0.8 * L.lbm_eos_critical(eos)[0]
    return L.lbm_create(nx, ny, eos, T, 1.0, params=L.lbm_params_default(precision=precision))


def _adversarial_f(nx, ny, seed):
    """Populations [9][ny][nx] mixing ordinary densities with nodes whose
    double sum is inexact, cancels, or meets special values."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(0.01, 2.0, (9, ny, nx))
    nodes = [(y, x) for y in range(1, ny - 1) for x in range(nx)]
    pick = rng.permutation(len(nodes))
    k = 0

    def take(m):
        nonlocal k
        out = [nodes[i] for i in pick[k:k + m]]
        k += m
        return out

    for (y, x) in take(40):  # magnitudes over 60 decades, random signs
        f[:, y, x] = rng.choice([-1.0, 1.0], 9) * 10.0 ** rng.uniform(-30, 30, 9)
    for (y, x) in take(40):  # exact cancellation within a narrow span
        v = rng.uniform(0.5, 1.5, 4)
        f[:, y, x] = [0.0, v[0], -v[0], v[1], -v[1], v[2], -v[2], v[3], -v[3]]
    for (y, x) in take(10):  # signed zeros
        f[:, y, x] = rng.choice([-0.0, 0.0], 9)
    full = (2.0 ** 24 - 1) / 2.0 ** 23  # all 24 significand bits set
    for i, (y, x) in enumerate(take(40)):  # spans of 24..27 binades around the limit
        span = 24 + i % 4
        f[:, y, x] = full * rng.choice([-1.0, 1.0], 9)
        f[rng.integers(1, 9), y, x] = full * 2.0 ** (-span)
    specials = [1e-40, -1e-41, np.inf, -np.inf, np.nan, 1e-39]
    for (y, x), v in zip(take(6), specials):  # a subnormal, an infinity, a NaN among ordinary terms
        f[rng.integers(0, 9), y, x] = v
    return f


def _double_sum(f32, walls=True):
    r = np.zeros(f32.shape[1:])
    for a in range(9):
        r = r + f32[a].astype(np.float64)
    if walls:
        r[0] = r[-1] = 0.0
    return r


def _same_bits(a, b):
    a, b = np.asarray(a), np.asarray(b)
    both_nan = np.isnan(a) & np.isnan(b)
    return bool(np.all(both_nan | (a.view(np.int64) == b.view(np.int64))))


@pytest.mark.parametrize("nx", [64, 30])  # 16-byte vector path and the scalar path
def test_fp32_density_readback_is_the_double_sum(nx):
    ny = 12
    ctx = _ctx(nx, ny)
    f = _adversarial_f(nx, ny, seed=nx)
    L.lbm_set_f(ctx, f)
    want = _double_sum(f.astype(np.float32))
    got_pageable = L.lbm_get_rho(ctx)
    got_pinned = L.lbm_get_rho(ctx, _pinned((ny, nx)))
    L.lbm_destroy(ctx)
    assert _same_bits(got_pageable, want)
    assert _same_bits(got_pinned, want)


@pytest.mark.parametrize("nx,precision", [(64, 32), (30, 32), (32, 64)])
def test_set_rho_from_pinned_memory_matches_pageable(nx, precision):
    ny = 16
    rng = np.random.default_rng(3)
    rho = rng.uniform(0.05, 8.0, (ny, nx))
    pinned = _pinned((ny, nx))
    pinned[:] = rho
    a, b = _ctx(nx, ny, precision), _ctx(nx, ny, precision)
    L.lbm_set_rho(a, rho)
    L.lbm_set_rho(b, pinned)
    fa, fb = L.lbm_get_f(a), L.lbm_get_f(b)
    ra = L.lbm_get_rho(a, _pinned((ny, nx)))
    assert _same_bits(fa, fb)
    # a rejected pinned input leaves the state untouched
    for bad in (-1.0, 0.0, np.nan, np.inf, -0.0):
        pinned[:] = rho
        pinned[5, 7] = bad
        with pytest.raises(L.LbmError) as e:
            L.lbm_set_rho(b, pinned)
        assert e.value.status == L.LBM_EINVAL
        assert _same_bits(L.lbm_get_f(b), fa)
    # ... and the state then advances exactly like the one set from pageable memory
    L.lbm_step(a, 4)
    L.lbm_step(b, 4)
    assert _same_bits(L.lbm_get_f(a), L.lbm_get_f(b))
    # wall rows are ignored by the check, whatever they hold
    pinned[:] = rho
    pinned[0, :] = -1.0
    pinned[-1, :] = np.nan
    L.lbm_set_rho(b, pinned)
    assert _same_bits(L.lbm_get_rho(b), ra)
    L.lbm_destroy(a)
    L.lbm_destroy(b)


@pytest.mark.parametrize("nx,ny,precision", [(1024, 1030, 32), (1030, 1024, 32), (1028, 1026, 64)])
def test_large_field_readback_in_chunks(nx, ny, precision):
    # fields of 2^20 nodes and more come back in row chunks whose copies overlap
    # the density kernel; ragged last chunks, the scalar path (nx % 4 != 0) and
    # FP64 included
    ctx = _ctx(nx, ny, precision)
    rng = np.random.default_rng(nx + ny)
    L.lbm_set_rho(ctx, rng.uniform(0.05, 8.0, (ny, nx)))
    f = L.lbm_get_f(ctx)
    want = _double_sum(f)
    for out in (None, _pinned((ny, nx))):
        assert _same_bits(L.lbm_get_rho(ctx, out), want)
    L.lbm_destroy(ctx)
