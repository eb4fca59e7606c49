"""Pins of the droplet-shape oracle (readings of Sec. III.A, Fig. 2) against geometry.

Expected values come from the geometry of the synthetic droplets (spherical
and ellipsoidal caps, whose contact angle satisfies tan(theta/2) = height /
footprint radius), from linear profiles whose zero is known, and from uniform
or layered velocity fields, not from the oracle's own formulas.
"""
import numpy as np
import pytest

from oracle import shape as sh

NX, NY, NZ = 96, 80, 40


def cap_fields(cx, cy, zc, a, b, c, width=1.5, u=(0.0, 0.0, 0.0)):
    """Moments of an ellipsoidal liquid cap (semi-axes a, b, c; centre below the wall)."""
    z, y, x = np.meshgrid(np.arange(NZ), np.arange(NY), np.arange(NX), indexing="ij")
    q = np.sqrt(((x - cx) / a) ** 2 + ((y - cy) / b) ** 2 + ((z - zc) / c) ** 2)
    C = np.tanh(-(q - 1.0) * min(a, b, c) / width)
    rhoR, rhoB = (1.0 + C) / 2.0, (1.0 - C) / 2.0
    j = np.stack([np.full(C.shape, u[d]) * (rhoR + rhoB) for d in range(3)], axis=-1)
    return rhoR, rhoB, j


def test_spherical_cap_height_radius_and_contact_angle():
    R, zc = 22.0, -8.0
    r = sh.shape(*cap_fields(47.0, 39.0, zc, R, R, R))
    height = zc + R + 0.5          # liquid from the wall z = -1/2 to the apex
    r0 = np.sqrt(R * R - zc * zc)  # footprint radius in the first fluid layer z = 0
    assert r["xc"] == pytest.approx(47.0, abs=1e-9) and r["yc"] == pytest.approx(39.0, abs=1e-9)
    assert r["height"] == pytest.approx(height, abs=0.02)
    assert r["r_x"] == pytest.approx(r0, abs=0.02) and r["r_y"] == pytest.approx(r0, abs=0.02)
    theta = np.degrees(2 * np.arctan(height / r0))
    assert r["theta_x"] == pytest.approx(theta, abs=0.1) and r["theta_y"] == pytest.approx(theta, abs=0.1)
    # a hemisphere-like cap is near 90 degrees, a flat one well below
    assert 50 < r["theta_x"] < 100


def test_elongated_cap_has_different_axial_and_transverse_angles():
    a, b, c, zc = 36.0, 14.0, 12.0, -3.0
    r = sh.shape(*cap_fields(47.5, 39.5, zc, a, b, c))
    height = zc + c + 0.5
    rx0 = a * np.sqrt(1 - (zc / c) ** 2)
    ry0 = b * np.sqrt(1 - (zc / c) ** 2)
    assert r["height"] == pytest.approx(height, abs=0.05)
    assert r["r_x"] == pytest.approx(rx0, abs=0.1)
    assert r["r_y"] == pytest.approx(ry0, abs=0.1)
    assert r["theta_y"] > r["theta_x"] + 10  # the narrow direction is steeper
    assert r["theta_x"] == pytest.approx(np.degrees(2 * np.arctan(height / rx0)), abs=0.2)


def test_volume_of_a_cap_matches_the_solid_of_revolution():
    R, zc = 18.0, -6.0
    # a thin interface: the diffuse layer adds O((width/R)^2) to the volume
    r = sh.shape(*cap_fields(47.0, 39.0, zc, R, R, R, width=0.6))
    # spherical cap above the wall z = -1/2: height hc, volume pi hc^2 (3R - hc) / 3
    hc = zc + R + 0.5
    assert r["volume"] == pytest.approx(np.pi * hc * hc * (3 * R - hc) / 3.0, rel=5e-3)


def test_crossings_interpolate_linearly():
    p = np.array([-2.0, -1.0, 0.5, 1.5, 2.0, 1.0, -0.25, -3.0])
    left, right = sh.crossing_run(p, 3)
    assert left == pytest.approx(1 + 1.0 / 1.5)
    assert right == pytest.approx(5 + 1.0 / 1.25)
    assert sh.crossing_run(p, 0) == (0.0, 0.0)


def test_velocity_means_over_the_liquid_columns():
    rhoR, rhoB, j = cap_fields(47.0, 39.0, -8.0, 22.0, 22.0, 22.0, u=(0.01, -0.02, 0.0))
    r = sh.shape(rhoR, rhoB, j)
    assert r["v_x"] == pytest.approx(0.01, rel=1e-12) and r["v_y"] == pytest.approx(-0.02, rel=1e-12)
    # a layered flow u_x = 1e-3 z in the liquid: the column mean is 1e-3 times the mean liquid z
    z = np.arange(NZ)[:, None, None] * np.ones((1, NY, NX))
    j2 = j.copy()
    j2[..., 0] = 1e-3 * z * (rhoR + rhoB)
    r2 = sh.shape(rhoR, rhoB, j2)
    C = (rhoR - rhoB) / (rhoR + rhoB)
    xq, yq = int(np.floor(r2["xc"] + r2["r_x"] / 2 + 0.5)), int(np.floor(r2["yc"] + 0.5))
    liq = np.nonzero(C[:, yq, xq] > 0)[0]
    assert r2["v_x"] == pytest.approx(1e-3 * liq.mean(), rel=1e-12)
