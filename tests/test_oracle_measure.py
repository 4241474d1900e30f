"""Pins for the oracle's apparent contact-angle measurement.

A circular cap cut by the base row with a known angle theta has chord
L = 2 R sin(theta) and height H = R (1 - cos(theta)), so tan(theta/2) = 2H/L
for every theta.  Density fields are built from that geometry with a tanh
profile whose mid-density contour is exactly the circle.
"""
import math

import numpy as np
import pytest

import oracle as O


def cap_field(nx, ny, xc, R, theta, rv, rl, W=3.0, wall=0):
    """Circle of radius R through the base row at angle theta (radians)."""
    base = 1.0 if wall == 0 else ny - 2.0
    yc = base - R * math.cos(theta) if wall == 0 else base + R * math.cos(theta)
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    r = np.hypot(x - xc, y - yc)
    rho = 0.5 * (rl + rv) - 0.5 * (rl - rv) * np.tanh(2 * (r - R) / W)
    rho[0] = rho[-1] = 0.0  # wall rows carry no fluid
    return rho


@pytest.mark.parametrize("theta_deg", [30, 60, 90, 120, 150])
@pytest.mark.parametrize("wall", [0, 1])
def test_circular_cap_angle(theta_deg, wall):
    th = math.radians(theta_deg)
    R = 40.0
    rho = cap_field(240, 200, 119.6, R, th, 0.01, 0.4, wall=wall)
    got, H, L, xc = O.contact_angle_field(rho, wall, 20, 220, 0.205)
    assert abs(math.degrees(got) - theta_deg) < 0.6
    assert L == pytest.approx(2 * R * math.sin(th), abs=0.3)
    assert H == pytest.approx(R * (1 - math.cos(th)), abs=0.3)
    assert xc in (119, 120)


def test_centre_column_tie_goes_to_lowest_x():
    rho = cap_field(100, 60, 50.5, 15.0, math.pi / 2, 0.01, 0.4)
    _, _, _, xc = O.contact_angle_field(rho, 0, 0, 100, 0.205)
    assert xc == 50


def test_no_contact_raises():
    rho = np.full((40, 60), 0.01)
    with pytest.raises(ValueError):
        O.contact_angle_field(rho, 0, 0, 60, 0.205)
    rho = cap_field(60, 40, 30.0, 28.0, math.pi / 2, 0.01, 0.4)  # touches the region edge
    with pytest.raises(ValueError):
        O.contact_angle_field(rho, 0, 5, 55, 0.205)
