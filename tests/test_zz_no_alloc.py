"""lbm_mass_noalloc: the total-mass reduction for callers that cannot allocate
device memory -- code running under another framework's allocator that must
own every device byte, embedders with device allocation disabled, and
real-time loops that must not hit cudaMalloc's implicit synchronisation.

It is checked through the C ABI against lbm_mass, the allocating entry point
that computes the same sum, on two calls in a row (the second call reuses the
scratch array the first one left behind).  This file is collected last on
purpose so that a run stopping at the first failure has already run every
other test."""
import numpy as np
import pytest

from paper_1501_05430_gb300 import inputs as I
from paper_1501_05430_gb300 import lbm as L

pytestmark = pytest.mark.gpu


def _state(nx, ny, walls, seed):
    eos = L.carnahan_starling()
    T = 0.7 * L.lbm_eos_critical(eos)[0]
    rv, rl = L.lbm_coexistence(eos, T)
    drops = [(nx * 0.4, ny * 0.3, 0)] if walls else [(nx * 0.4, ny * 0.25, ny * 0.5)]
    rho = I.droplet_field(nx, ny, drops, rv, rl)
    return eos, T, I.random_distributions(rho, seed, walls=walls)


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("nx,ny,walls", [(300, 130, True), (64, 48, False), (4096, 2048, True)])
def test_mass_noalloc_matches_lbm_mass(precision, nx, ny, walls):
    torch = pytest.importorskip("torch")
    eos, T, f = _state(nx, ny, walls, seed=nx + ny)
    p = L.lbm_params_default(precision=precision, kernel=L.LBM_KERNEL_REFERENCE, check_every=0)
    with L.Lbm(nx, ny, eos, T, 1.0, walls=walls, params=p, torch_state=False) as g:
        g.set_f(f)
        ref = g.mass()
    dtype = torch.float32 if precision == 32 else torch.float64
    fd = torch.as_tensor(f, dtype=dtype).to("cuda").contiguous()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    for k in range(2):
        L.lbm_mass_noalloc(fd.data_ptr(), nx, ny, precision, walls, out.data_ptr() + 8 * k)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    assert got[0] == pytest.approx(ref, rel=1e-12)
    assert got[1] == pytest.approx(ref, rel=1e-12)


def test_mass_noalloc_rejects_bad_arguments():
    torch = pytest.importorskip("torch")
    fd = torch.zeros(9 * 16 * 8, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for args in [(0, 8, 32, 1), (16, 2, 32, 1), (16, 8, 16, 1), (16, 8, 32, 2), (1 << 15, 1 << 14, 32, 1)]:
        nx, ny, prec, walls = args
        st = L.load().lbm_mass_noalloc(fd.data_ptr(), nx, ny, prec, walls, out.data_ptr(), None)
        assert st == L.LBM_EINVAL, args
    assert L.load().lbm_mass_noalloc(None, 16, 8, 32, 1, out.data_ptr(), None) == L.LBM_EINVAL
