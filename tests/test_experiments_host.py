"""Host-side pieces of the experiment presets (no GPU): the preset table and
the circular-cap measurement above a depleted wall layer."""
import numpy as np
import pytest

from paper_1501_05430_gb300 import experiments as E
from paper_1501_05430_gb300 import inputs as I


def test_presets_follow_the_paper():
    P = E.presets()
    assert [c.G_w for c in P["E1"]] == [-0.766, -1.1, -1.43, -1.77, -2.1, -2.43, -2.766]
    assert [c.G_w for c in P["E2"]] == [-2.666, -3.333, -4.0]
    assert [c.theta_deg for c in P["E7"]] == [15.0, 30.0, 45.0, 90.0, 135.0, 150.0]
    assert {c.ratio for c in P["E8"]} == {1000}
    assert [(c.n_iter, c.theta_deg) for c in P["E6"]] == [(0, 15.0), (4, 15.0)]
    assert sorted({c.kappa for c in P["E10"]}) == [0.5, 0.9, 0.98]
    assert all(c.wetting == 1 for k in ("E1", "E2", "E3", "E4", "E5") for c in P[k])
    # psi_l of Table 1's liquid: psi^2 = 2 (rho_l/3 - p(rho_l))
    assert E._psi_l(100) == pytest.approx(8.145, abs=1e-3)


@pytest.mark.parametrize("theta", [40.0, 90.0, 130.0, 160.0])
@pytest.mark.parametrize("base", [1, 2, 4])
def test_cap_above_layer_recovers_synthetic_caps(theta, base):
    nx, ny, R = 300, 100, 35.0
    t = np.deg2rad(theta)
    rho = I.droplet_field(nx, ny, [(140.6, R, base - R * np.cos(t))], 1.0, 10.0, 3.0)
    rho[1:base] = 1.0  # depleted rows under the droplet
    th, H, L, b = E.cap_above_layer(rho, 5.5)
    assert b == base
    assert th == pytest.approx(theta, abs=0.3)


def test_cap_above_layer_wraps_across_the_periodic_edge():
    nx, ny, R = 120, 60, 20.0
    rho = I.droplet_field(nx, ny, [(2.3, R, 1.0)], 1.0, 10.0, 3.0)
    th, H, L, b = E.cap_above_layer(rho, 5.5)
    assert th == pytest.approx(90.0, abs=0.3)


def test_cap_above_layer_without_liquid_near_the_wall():
    rho = np.ones((60, 120))
    assert E.cap_above_layer(rho, 5.5) is None
