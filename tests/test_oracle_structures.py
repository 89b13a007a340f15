"""Pins of the Section 6.3 structures in the oracle (the BCC single gyroid and the FCC diamond of spheres and
spheroids) against exact values of the gyroid function, the symmetries of the two crystals, and volume fractions
computed without the lattice mapping."""
import numpy as np
import pytest

from oracle import geometry as g

BCC = 0.5 * np.array([[-1.0, 1.0, 1.0], [1.0, -1.0, 1.0], [1.0, 1.0, -1.0]])
FCC = 0.5 * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])


def test_gyroid_exact_values():
    """g(0) = 0; g(l/4, 0, l/4) = 1; the maximum 3/2 at (l/8)(1, 1, 1) (each product is sin(pi/4) cos(pi/4) = 1/2)."""
    for l in (1.0, 2.5):
        assert g.gyroid_value(np.zeros(3), l) == 0.0
        assert np.isclose(g.gyroid_value(np.array([0.25, 0.0, 0.25]) * l, l), 1.0, atol=1e-15)
        assert np.isclose(g.gyroid_value(np.ones(3) * l / 8, l), 1.5, atol=1e-15)
    x = np.random.default_rng(0).uniform(-2, 2, (100000, 3))
    assert np.max(g.gyroid_value(x)) <= 1.5 + 1e-12 and np.min(g.gyroid_value(x)) >= -1.5 - 1e-12


def test_gyroid_has_the_bcc_translations():
    """g is invariant under the BCC lattice vectors (each product changes sign twice) but not under half the cube
    along one axis: the structure of Section 6.3 belongs to the BCC lattice, not to a finer one."""
    x = np.random.default_rng(1).uniform(-1, 1, (1000, 3))
    for a in BCC.T:
        assert np.allclose(g.gyroid_value(x + a), g.gyroid_value(x), atol=1e-13)
    assert not np.allclose(g.gyroid_value(x + np.array([0.5, 0.0, 0.0])), g.gyroid_value(x), atol=1e-3)


def test_gyroid_fill_fraction_matches_the_cube():
    """The share of edge DoFs of the BCC primitive cell inside {g > 1.1} equals the volume fraction of the set in the
    conventional cube, estimated by uniform samples of the cube (no lattice mapping)."""
    x = np.random.default_rng(2).uniform(0, 1, (400000, 3))
    frac = np.mean(g.gyroid_value(x) > 1.1)
    eps = g.eps_edges_gyroid(32, BCC)
    assert set(np.unique(eps)) == {1.0, 16.0}
    assert abs(np.mean(eps == 16.0) - frac) < 0.004


def test_diamond_inversion_and_translations():
    """The diamond is symmetric under inversion through a bond midpoint (l/8)(1, 1, 1) and periodic under the FCC
    vectors."""
    x = np.random.default_rng(3).uniform(-1, 1, (20000, 3))
    inside = g.in_diamond(x, FCC)
    assert 0.03 < inside.mean() < 0.3
    assert np.array_equal(inside, g.in_diamond(np.ones(3) / 4 - x, FCC))
    for a in FCC.T:
        assert np.array_equal(inside, g.in_diamond(x + a, FCC))


def test_diamond_bonds_are_tetrahedral():
    """From the site at the origin the bonds run along (1,1,1), (1,-1,-1), (-1,1,-1), (-1,-1,1): a point 0.2 l out
    along a bond lies in its spheroid, the same distance along the opposite directions (no bond there) is outside."""
    for d in g.DIAMOND_BONDS:
        u = d / np.linalg.norm(d)
        assert g.in_diamond((0.2 * u)[None], FCC)[0]
        assert not g.in_diamond((-0.2 * u)[None], FCC)[0]
    assert g.in_diamond((np.ones(3) / 8)[None], FCC)[0]  # a bond midpoint


def test_diamond_spheres_alone_fill_their_volume():
    """With the spheroids shrunk to segments (b = 0) the fill is that of two spheres of radius 0.12 l per primitive
    cell of volume l^3 / 4."""
    eps = g.eps_edges_diamond(48, FCC, b=0.0)
    frac = 2 * 4.0 / 3.0 * np.pi * 0.12 ** 3 / abs(np.linalg.det(FCC))
    assert abs(np.mean(eps == 13.0) - frac) < 0.003


@pytest.mark.parametrize("b", [0.11, 0.2])
def test_diamond_spheroid_geometry(b):
    """Each spheroid has its foci at the two sphere centres and semi-minor axis b l / 2: on the bond's perpendicular
    bisector the boundary lies at distance b l / 2 from the bond axis."""
    m = np.ones(3) / 8
    perp = np.array([1.0, -1.0, 0.0]) / np.sqrt(2.0)
    inside = g.in_diamond((m + (0.5 * b - 1e-9) * perp)[None], FCC, b=b)[0]
    outside = g.in_diamond((m + (0.5 * b + 1e-9) * perp)[None], FCC, b=b)[0]
    assert inside and not outside
