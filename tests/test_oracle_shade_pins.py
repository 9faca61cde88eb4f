"""Pins of the shading oracle (Lambertian irradiance of the lit fractions).

  * flat terrain: the surface is the sphere of radius R + h0, so the normal is
    the radial direction and E = sum_l I_l s_l max(0, n . L_l) with n from the
    inverse tile mapping (checked at every texel, both projections);
  * a plane tilted by slope a along grid x through the tile centre: the normal
    there is unit(-a, 0, 1) (the tangent vectors are x + a z and y);
  * E is linear in each light's intensity and lit fraction and lights add.
"""
import math

import numpy as np
import pytest

import oracle

R = 1737.4e3


def _L(e, a):
    return np.array([math.cos(e) * math.sin(a), math.cos(e) * math.cos(a), math.sin(e)])


def _radial(nx, ny, g, proj):
    v, u = np.meshgrid(np.arange(ny, dtype=float), np.arange(nx, dtype=float), indexing="ij")
    X, Y = (u - (nx - 1) / 2) * g, (v - (ny - 1) / 2) * g
    if proj == "gnomonic":
        d = np.stack([X, Y, np.full_like(X, R)], -1)
        return (d / np.linalg.norm(d, axis=-1, keepdims=True)).reshape(-1, 3)
    r2 = X * X + Y * Y
    return (np.stack([4 * R * X, 4 * R * Y, 4 * R * R - r2], -1) /
            (4 * R * R + r2)[..., None]).reshape(-1, 3)


@pytest.mark.parametrize("proj", ["gnomonic", "polar_stereo"])
def test_flat_terrain_radial_normal(proj):
    nx, ny, g = 41, 33, 900.0
    h = np.full((ny, nx), 250.0, np.float32)
    rng = np.random.default_rng(3)
    s1 = rng.uniform(0, 1, nx * ny)
    lights = [(math.radians(3.0), math.radians(40.0), 1.0, s1),
              (math.radians(-0.5), math.radians(200.0), 0.01, np.ones(nx * ny))]
    E = oracle.shade(h, g, R, lights, proj=proj)
    n = _radial(nx, ny, g, proj)
    exp = sum(I * s * np.maximum(0.0, n @ _L(e, a)) for e, a, I, s in lights)
    assert np.abs(E - exp).max() < 1e-9


@pytest.mark.parametrize("proj", ["gnomonic", "polar_stereo"])
@pytest.mark.parametrize("slope", [0.0, 0.3, -1.2])
def test_tilted_plane_at_the_centre(proj, slope):
    n, g = 31, 20.0
    c = (n - 1) // 2
    X = (np.arange(n) - c) * g
    h = np.tile((slope * X).astype(np.float32), (n, 1))
    N = np.array([-slope, 0.0, 1.0]) / math.hypot(slope, 1.0)
    for e, a in ((0.4, 0.0), (0.2, math.pi / 2), (0.9, 4.0), (0.05, 1.3)):
        L = _L(e, a)
        s = np.ones(n * n)
        E = oracle.shade(h, g, R, [(e, a, 1.0, s)], proj=proj)
        assert abs(E[c * n + c] - max(0.0, N @ L)) < 1e-8
        Eu = oracle.shade(h, g, R, [(e, a, 1.0, np.ones(1))], proj=proj,
                          uv=np.array([[c, c]], np.float32))
        assert abs(Eu[0] - max(0.0, N @ L)) < 1e-8


def test_linear_in_intensity_and_fraction():
    rng = np.random.default_rng(4)
    h = rng.normal(0, 40, (24, 28)).astype(np.float32)
    n = h.size
    s1, s2 = rng.uniform(0, 1, n), rng.uniform(0, 1, n)
    l1 = (0.3, 1.0, 1.7, s1)
    l2 = (0.1, 3.0, 0.4, s2)
    E1 = oracle.shade(h, 30.0, R, [l1])
    E2 = oracle.shade(h, 30.0, R, [l2])
    E12 = oracle.shade(h, 30.0, R, [l1, l2])
    assert np.abs(E12 - (E1 + E2)).max() < 1e-12
    E1x = oracle.shade(h, 30.0, R, [(0.3, 1.0, 3.4, s1 * 0.5)])
    assert np.abs(E1x - E1).max() < 1e-12
