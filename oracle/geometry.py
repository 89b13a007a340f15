"""M0 from a sphere structure (Section 4.4): inverse permittivity at the edge DoFs, FP64.

Grid convention (forward differences of eq. stencils): node (i,j,k) sits at (i,j,k)h; the x-edge with index (i,j,k)
at ((i+1/2)h, jh, kh), the y-edge at (ih, (j+1/2)h, kh), the z-edge at (ih, jh, (k+1/2)h); cell (i,j,k) at
((i+1/2)h, (j+1/2)h, (k+1/2)h). h = a / N with a = 1.

Readings:
* The entry of M0 is eps^{-1} at the edge midpoint (Section 4.4 and Section 6.2 state eps^{-1}; the case display
  writes eps values, read as the permittivity whose inverse is taken).
* A point is inside a sphere when its distance to some periodic image of the centre is <= r (closed ball).
  Where spheres overlap, the last sphere in the list that contains the point gives its permittivity.
* An edge midpoint whose distance to a sphere surface is below 1e-12 is "on the interface": its entry is
  4 / (sum of eps at the centres of the 4 cells sharing that edge), as in Section 4.4's harmonic rule.

General lattice (Section 2's coordinate change x = A y): the grid above lives in y on the unit cube; a DoF at y sits
at the Cartesian point x = A y. Sphere centres and radii are then Cartesian, and periodicity is under the columns of
A: the distance to a centre is the minimum over the images c + A n. The nearest image is found by reducing the
fractional offset A^{-1}(x - c) to [-1/2, 1/2]^3 and searching the 27 neighbouring translates, which is exact for
cells whose reduced offset lies within one translate of the nearest image (the SC, FCC and BCC primitive cells).
"""
from __future__ import annotations

import numpy as np

INTERFACE_TOL = 1e-12


def _periodic_distance(p, c):
    """Euclidean distance from points p (..., 3) to the nearest periodic image of c in the unit cube."""
    d = p - np.asarray(c)[None, :]
    d = d - np.round(d)
    return np.sqrt(np.sum(d * d, axis=-1))


def _lattice_distance(x, c, A, Ainv):
    """Euclidean distance from Cartesian points x (..., 3) to the nearest image c + A n of the centre c."""
    f = (x - np.asarray(c)[None, :]) @ Ainv.T
    f = f - np.round(f)
    r = np.array([-1.0, 0.0, 1.0])
    shifts = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    best = np.full(f.shape[0], np.inf)
    for s in shifts:
        v = (f + s[None, :]) @ A.T
        best = np.minimum(best, np.sqrt(np.sum(v * v, axis=-1)))
    return best


def eps_at_points(points: np.ndarray, spheres: np.ndarray, eps_bg: float, lattice=None):
    """Permittivity at each point, and a flag telling whether the point lies on some sphere surface. Without a
    lattice the points are fractions of the unit cube; with one they are y coordinates, mapped to x = A y."""
    pts = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    if lattice is not None:
        A = np.asarray(lattice, dtype=np.float64)
        Ainv = np.linalg.inv(A)
        pts = pts @ A.T
    eps = np.full(pts.shape[0], float(eps_bg))
    on_iface = np.zeros(pts.shape[0], dtype=bool)
    for cx, cy, cz, r, e in np.asarray(spheres, dtype=np.float64).reshape(-1, 5):
        if lattice is None:
            dist = _periodic_distance(pts, (cx, cy, cz))
        else:
            dist = _lattice_distance(pts, (cx, cy, cz), A, Ainv)
        eps[dist <= r] = e
        on_iface |= np.abs(dist - r) < INTERFACE_TOL
    return eps, on_iface


def edge_positions(N: int, axis: int) -> np.ndarray:
    """Midpoints of the edges along ``axis`` (0 = x, 1 = y, 2 = z), shape (N, N, N, 3) indexed [z, y, x]."""
    h = 1.0 / N
    i = np.arange(N)
    z, y, x = np.meshgrid(i, i, i, indexing="ij")
    pos = np.stack([x * h, y * h, z * h], axis=-1).astype(np.float64)
    pos[..., axis] += 0.5 * h
    return pos


def eps_edges(N: int, spheres, eps_bg: float, lattice=None) -> np.ndarray:
    """Permittivity at the 3 N^3 edge DoFs, shape (3, N, N, N), with the interface rule applied. With ``lattice``
    the edge midpoints and cell centres are y coordinates mapped to x = A y, and the spheres are Cartesian."""
    h = 1.0 / N
    out = np.empty((3, N, N, N))
    i = np.arange(N)
    zc, yc, xc = np.meshgrid(i, i, i, indexing="ij")
    for axis in range(3):
        pos = edge_positions(N, axis)
        eps, on = eps_at_points(pos, spheres, eps_bg, lattice)
        eps = eps.reshape(N, N, N)
        on = on.reshape(N, N, N)
        for z, y, x in zip(*np.nonzero(on)):
            # the 4 cells around this edge: offsets -1/0 in the two axes transverse to it
            others = [a for a in range(3) if a != axis]
            total = 0.0
            for o1 in (-1, 0):
                for o2 in (-1, 0):
                    idx = [x, y, z]
                    idx[others[0]] += o1
                    idx[others[1]] += o2
                    centre = (np.asarray(idx, dtype=np.float64) + 0.5) * h
                    e, _ = eps_at_points(centre[None, :], spheres, eps_bg, lattice)
                    total += e[0]
            # stored as a permittivity, so that the M0 entry 1/eps equals the harmonic-rule value 4 / total
            eps[z, y, x] = total / 4.0
        out[axis] = eps
    return out


def m0_from_structure(N: int, spheres, eps_bg: float, lattice=None) -> np.ndarray:
    """The diagonal of M0, shape (3, N, N, N)."""
    return 1.0 / (eps_edges(N, spheres, eps_bg) if lattice is None else eps_edges(N, spheres, eps_bg, lattice))
