"""Pins of the oracle's M0 construction (Section 4.4) by hand-computed entries, volume fractions and symmetry."""
import numpy as np

import workloads as wl
from oracle import geometry


def test_hand_computed_entries_N6():
    """N = 6, sphere r = 1/4 at the cell centre, eps 13 in air. Entries worked out by hand:
    * x-edge (2,3,3) at (5/12, 1/2, 1/2) lies inside: 1/13;
    * x-edge (1,3,3) at (1/4, 1/2, 1/2) lies on the surface; its 4 cells are all outside: 4/(1+1+1+1) = 1;
    * x-edge (2,4,4) at (5/12, 2/3, 2/3) lies on the surface (distance^2 = 1/144 + 2/36 = 1/16); one of its cells,
      (2,3,3) centred at (5/12, 7/12, 7/12), is inside: 4/(13+1+1+1) = 1/4."""
    s = wl.sc_single_sphere()
    m0 = geometry.m0_from_structure(6, s.as_array(), s.eps_bg)
    assert m0[0, 3, 3, 2] == 1 / 13          # index order [axis, z, y, x]
    assert m0[0, 3, 3, 1] == 1.0
    assert m0[0, 4, 4, 2] == 0.25
    assert set(np.unique(m0)) == {1 / 13, 0.25, 1.0}


def test_volume_fraction():
    s = wl.sc_single_sphere()
    m0 = geometry.m0_from_structure(64, s.as_array(), s.eps_bg)
    frac = np.mean(m0 < 0.5)
    assert abs(frac - 4 / 3 * np.pi * 0.25 ** 3) < 0.01 * frac


def test_periodic_images():
    """A sphere at the corner (wrapping across the periodic boundary) is the centred sphere rolled by N/2."""
    N = 16
    a = geometry.m0_from_structure(N, np.array([[0.5, 0.5, 0.5, 0.3, 9.0]]), 1.0)
    b = geometry.m0_from_structure(N, np.array([[0.0, 0.0, 0.0, 0.3, 9.0]]), 1.0)
    assert np.array_equal(np.roll(a, (N // 2, N // 2, N // 2), axis=(1, 2, 3)), b)


def test_later_sphere_takes_precedence():
    sph = np.array([[0.5, 0.5, 0.5, 0.3, 5.0], [0.5, 0.5, 0.5, 0.1, 11.0]])
    m0 = geometry.m0_from_structure(16, sph, 1.0)
    assert np.isclose(m0[0, 8, 8, 8], 1 / 11) and 1 / 5 in np.unique(m0)


def test_diamond_air_spheres_background():
    """Air spheres in eps = 13: the majority of edges carry 1/13, the sphere interiors 1."""
    s = wl.diamond_air_spheres()
    m0 = geometry.m0_from_structure(16, s.as_array(), s.eps_bg)
    vals = set(np.round(np.unique(m0), 12))
    assert {round(1 / 13, 12), 1.0} <= vals
