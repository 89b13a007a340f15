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


# ------------------------------------------------------------------------------------ the structures of Section 6.3
def gyroid_value(x: np.ndarray, l: float = 1.0) -> np.ndarray:
    """g(x, y, z) = sin(2 pi x / l) cos(2 pi y / l) + sin(2 pi y / l) cos(2 pi z / l) + sin(2 pi z / l) cos(2 pi x / l)
    at Cartesian points x (..., 3): the single gyroid of Section 6.3 is the set {g > 1.1} in the BCC lattice."""
    X = 2.0 * np.pi * np.asarray(x, dtype=np.float64) / l
    s, c = np.sin(X), np.cos(X)
    return s[..., 0] * c[..., 1] + s[..., 1] * c[..., 2] + s[..., 2] * c[..., 0]


def eps_edges_gyroid(N: int, lattice, l: float = 1.0, threshold: float = 1.1, eps_in: float = 16.0,
                     eps_out: float = 1.0) -> np.ndarray:
    """Permittivity at the 3 N^3 edge DoFs of a cell with lattice matrix A (the BCC primitive cell in Section 6.3):
    eps_in where g(A y) > threshold at the edge midpoint y, eps_out elsewhere. Reading: the paper gives no interface
    rule for a level set; the strict inequality decides every point (g = threshold has measure zero)."""
    A = np.asarray(lattice, dtype=np.float64)
    out = np.empty((3, N, N, N))
    for axis in range(3):
        x = edge_positions(N, axis) @ A.T
        out[axis] = np.where(gyroid_value(x, l) > threshold, eps_in, eps_out)
    return out


DIAMOND_BONDS = 0.25 * np.array([[1.0, 1.0, 1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])


def diamond_objects(l: float = 1.0, r: float = 0.12, b: float = 0.11):
    """The FCC diamond of Section 6.3 in Cartesian coordinates: spheres of radius r l at the two sites (0, 0, 0) and
    (1/4, 1/4, 1/4) l of the primitive cell, and one spheroid per nearest-neighbour bond (four per cell, from the
    site at the origin along DIAMOND_BONDS) with its foci at the two sphere centres and minor axis b l.
    Reading: the minor axis is the full length b l (semi-minor axis b l / 2); the semi-major axis follows from the
    foci, a = sqrt(c^2 + (b l / 2)^2) with c half the bond length. Returns (spheres [(centre, radius)],
    spheroids [(focus1, focus2, a)])."""
    sites = [np.zeros(3), 0.25 * l * np.ones(3)]
    spheres = [(s, r * l) for s in sites]
    spheroids = []
    for d in DIAMOND_BONDS:
        f1, f2 = np.zeros(3), d * l
        c = 0.5 * np.linalg.norm(f2 - f1)
        spheroids.append((f1, f2, float(np.sqrt(c * c + (0.5 * b * l) ** 2))))
    return spheres, spheroids


def _nearest_offset(x, c, A, Ainv):
    """x - (c + A n) for the image of c nearest to each point x (..., 3), searched as in _lattice_distance."""
    f = (x - np.asarray(c)[None, :]) @ Ainv.T
    f = f - np.round(f)
    r = np.array([-1.0, 0.0, 1.0])
    shifts = np.stack(np.meshgrid(r, r, r, indexing="ij"), -1).reshape(-1, 3)
    best = np.full(f.shape[0], np.inf)
    off = np.zeros_like(f)
    for s in shifts:
        v = (f + s[None, :]) @ A.T
        d = np.sum(v * v, axis=-1)
        take = d < best
        best[take] = d[take]
        off[take] = v[take]
    return off


def in_diamond(x: np.ndarray, lattice, l: float = 1.0, r: float = 0.12, b: float = 0.11) -> np.ndarray:
    """Whether Cartesian points x (..., 3) lie in a sphere or a spheroid of the diamond (closed sets), periodic
    under the columns of the lattice matrix (the FCC primitive cell)."""
    A = np.asarray(lattice, dtype=np.float64)
    Ainv = np.linalg.inv(A)
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    spheres, spheroids = diamond_objects(l, r, b)
    inside = np.zeros(x.shape[0], dtype=bool)
    for c, rad in spheres:
        inside |= np.sqrt(np.sum(_nearest_offset(x, c, A, Ainv) ** 2, axis=-1)) <= rad
    for f1, f2, a in spheroids:
        mid = 0.5 * (f1 + f2)
        v = _nearest_offset(x, mid, A, Ainv)  # relative to the nearest image of the bond midpoint
        h = 0.5 * (f2 - f1)
        dsum = np.sqrt(np.sum((v + h) ** 2, axis=-1)) + np.sqrt(np.sum((v - h) ** 2, axis=-1))
        inside |= dsum <= 2.0 * a
    return inside


def eps_edges_diamond(N: int, lattice, l: float = 1.0, r: float = 0.12, b: float = 0.11, eps_in: float = 13.0,
                      eps_out: float = 1.0) -> np.ndarray:
    """Permittivity at the edge DoFs of the FCC primitive cell holding the diamond of Section 6.3 (eps_in inside a
    sphere or spheroid, eps_out elsewhere)."""
    A = np.asarray(lattice, dtype=np.float64)
    out = np.empty((3, N, N, N))
    for axis in range(3):
        x = (edge_positions(N, axis) @ A.T).reshape(-1, 3)
        out[axis] = np.where(in_diamond(x, A, l, r, b), eps_in, eps_out).reshape(N, N, N)
    return out
