"""Seeded, synthetic workload definitions shared by the oracle and the CUDA path.

This module holds structure descriptions (lists of dielectric spheres in the unit cell), Brillouin-zone paths and
the per-workload settings (grid size, band count, tolerance). It contains none of the method's arithmetic: no
discretisation, no permittivity sampling, no operator and no eigensolver. Both the oracle (``oracle/``) and the CUDA
path (``paper_2503_19379_gb300``) take their inputs from here and compute everything else on their own.

Units: lattice constant a = 1, so positions are fractions of the cubic cell and Bloch vectors are in 1/a.
The paper's own structures for its band figures (Section 6.2-6.3) are partly lost with its figure images, so the
workloads below are synthetic stand-ins with the same ingredients: dielectric spheres with permittivity ratio 13
in simple-cubic, FCC and diamond arrangements, and seeded random sphere packings.

A sphere is a tuple ``(cx, cy, cz, r, eps_in)``; points inside any periodic image of a sphere take that sphere's
permittivity (later spheres in the list take precedence), all other points take ``eps_bg``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

PI = math.pi

# Symmetry points, Section 6 (the paper's own SC labels; FCC points in the conventional-cube frame).
SC_POINTS = {"G": (0.0, 0.0, 0.0), "L": (PI, 0.0, 0.0), "M": (PI, PI, 0.0), "N": (PI, PI, PI)}
FCC_POINTS = {"G": (0.0, 0.0, 0.0), "X": (0.0, 2 * PI, 0.0), "W": (PI, 2 * PI, 0.0),
              "K": (1.5 * PI, 1.5 * PI, 0.0), "L": (PI, PI, PI)}


@dataclass(frozen=True)
class Structure:
    """Dielectric spheres in the unit cube (periodic) on a background permittivity."""
    spheres: tuple
    eps_bg: float = 1.0
    name: str = ""

    def as_array(self) -> np.ndarray:
        return np.asarray(self.spheres, dtype=np.float64).reshape(-1, 5)


def sc_single_sphere(r: float = 0.25, eps_in: float = 13.0) -> Structure:
    """Simple cubic lattice: one dielectric sphere centred in the unit cube."""
    return Structure(((0.5, 0.5, 0.5, r, eps_in),), 1.0, "sc-sphere")


FCC_CENTRES = ((0.0, 0.0, 0.0), (0.0, 0.5, 0.5), (0.5, 0.0, 0.5), (0.5, 0.5, 0.0))


def fcc_spheres(r: float = 0.25, eps_in: float = 13.0) -> Structure:
    """FCC conventional cubic cell: four dielectric spheres at the FCC sites, in air."""
    return Structure(tuple((*c, r, eps_in) for c in FCC_CENTRES), 1.0, "fcc-spheres")


def diamond_air_spheres(r: float = 0.3, eps_bg: float = 13.0) -> Structure:
    """Diamond conventional cell: air spheres at the FCC sites and the same shifted by (1/4,1/4,1/4)."""
    centres = list(FCC_CENTRES) + [tuple(x + 0.25 for x in c) for c in FCC_CENTRES]
    return Structure(tuple((*c, r, 1.0) for c in centres), eps_bg, "diamond-air")


def homogeneous(eps: float = 1.0) -> Structure:
    return Structure((), eps, "homogeneous")


def random_structure(seed: int) -> Structure:
    """1-8 spheres, centres U[0,1)^3, radii U[0.1,0.3], permittivity U[4,16] each, in air."""
    rng = np.random.Generator(np.random.PCG64(seed))
    count = int(rng.integers(1, 9))
    sph = []
    for _ in range(count):
        c = rng.random(3)
        r = rng.uniform(0.1, 0.3)
        e = rng.uniform(4.0, 16.0)
        sph.append((float(c[0]), float(c[1]), float(c[2]), float(r), float(e)))
    return Structure(tuple(sph), 1.0, f"random-{seed}")


def kpath(labels, points: dict, npts: int) -> np.ndarray:
    """Piecewise-linear Bloch-vector path through the given symmetry points.

    Every vertex appears once (so a repeated label such as Gamma appears at each visit); the remaining
    ``npts - len(labels)`` interior points are shared among the segments in proportion to segment length
    (largest-remainder rounding). Returns an array of shape (npts, 3).
    """
    verts = [np.asarray(points[s], dtype=np.float64) for s in labels]
    nseg = len(verts) - 1
    if npts < len(verts):
        raise ValueError("npts must be at least the number of vertices")
    lengths = np.array([np.linalg.norm(verts[i + 1] - verts[i]) for i in range(nseg)])
    interior = npts - len(verts)
    share = lengths / lengths.sum() * interior
    alloc = np.floor(share).astype(int)
    rem = interior - alloc.sum()
    order = np.argsort(-(share - alloc), kind="stable")
    alloc[order[:rem]] += 1
    out = [verts[0]]
    for i in range(nseg):
        for j in range(1, alloc[i] + 1):
            t = j / (alloc[i] + 1)
            out.append(verts[i] + t * (verts[i + 1] - verts[i]))
        out.append(verts[i + 1])
    return np.asarray(out)


FCC_PATH = ("G", "X", "W", "K", "G", "L")
SC_PATH = ("G", "L", "M", "G", "N")
# BCC symmetry points of Section 6 (Cartesian, l = 1). The paper lists the points but its band figure, which would
# show their order, is lost; the path below is a reading: the usual BCC circuit through all of them.
BCC_POINTS = {"G": (0.0, 0.0, 0.0), "H": (0.0, 2 * PI, 0.0), "N": (PI, 0.0, PI), "P": (PI, PI, PI),
              "H'": (0.0, 0.0, 2 * PI)}
BCC_PATH = ("G", "H", "N", "G", "P", "H'")


@dataclass
class Workload:
    name: str
    structure: Structure
    N: int
    kpts: np.ndarray
    nbands: int
    tol: float
    precision: str = "c128"
    extra: dict = field(default_factory=dict)


def workload_sc_sphere_16() -> Workload:
    """SC lattice, one eps=13 sphere r=0.25, N=16, k=(pi/2,0,0), 8 bands, tol 1e-10."""
    return Workload("sc-sphere-N16", sc_single_sphere(), 16, np.array([[PI / 2, 0.0, 0.0]]), 8, 1e-10)


def workload_homogeneous_8() -> Workload:
    """Homogeneous eps=1 at N=8, k=(pi/2,0,0): every eigenvalue has a closed form."""
    return Workload("homogeneous-N8", homogeneous(1.0), 8, np.array([[PI / 2, 0.0, 0.0]]), 8, 1e-10)


def workload_fcc_32(precision: str = "c128", npts: int = 40) -> Workload:
    """FCC 4 spheres eps=13 r=0.25, N=32, 10 bands, 40 k-points on Gamma-X-W-K-Gamma-L, tol 1e-6."""
    return Workload("fcc-spheres-N32", fcc_spheres(), 32, kpath(FCC_PATH, FCC_POINTS, npts), 10, 1e-6, precision)


def workload_diamond_64(precision: str = "c128", npts: int = 60) -> Workload:
    """Diamond air spheres r=0.3 in eps=13, N=64, 12 bands, 60 k-points on the FCC path, tol 1e-6."""
    return Workload("diamond-air-N64", diamond_air_spheres(), 64, kpath(FCC_PATH, FCC_POINTS, npts), 12, 1e-6,
                    precision)


def workload_fcc_128(npts: int = 64) -> Workload:
    """FCC spheres eps=13, N=128, 16 bands, 64 k-points, complex64 search space with FP64 Rayleigh-Ritz."""
    return Workload("fcc-spheres-N128", fcc_spheres(), 128, kpath(FCC_PATH, FCC_POINTS, npts), 16, 1e-6, "mixed")



# ------------------------------------------------------------------------------------------ the paper's own cells
# Section 6's translation vectors (lattice constant l = 1) as the columns of A, and the timing setting of its BCC
# and FCC tables: the first 10 eigenvalues at k = (pi, pi, pi) / l. The structures themselves (the single gyroid and
# the diamond of spheres and spheroids) are sampled by each side's own geometry code; a workload only names them.
SC_CELL = np.eye(3)
FCC_CELL = 0.5 * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])
BCC_CELL = 0.5 * np.array([[-1.0, 1.0, 1.0], [1.0, -1.0, 1.0], [1.0, 1.0, -1.0]])


def workload_bcc_gyroid(N: int = 128) -> Workload:
    """BCC single gyroid {g > 1.1}, eps 16 in air, on the BCC primitive cell at N (power of two; the paper's timing
    table uses N = 100, 120, 150), 10 bands at k = (pi, pi, pi), tol 1e-6."""
    s = Structure((), 1.0, "bcc-gyroid")
    return Workload(f"bcc-gyroid-N{N}", s, N, np.array([[PI, PI, PI]]), 10, 1e-6,
                    extra={"lattice": BCC_CELL, "geometry": "gyroid", "threshold": 1.1, "eps_in": 16.0})


def workload_fcc_diamond(N: int = 128) -> Workload:
    """FCC diamond of spheres (r = 0.12) and bond spheroids (minor axis 0.11), eps 13 in air, on the FCC primitive
    cell at N, 10 bands at k = (pi, pi, pi), tol 1e-6."""
    s = Structure((), 1.0, "fcc-diamond")
    return Workload(f"fcc-diamond-N{N}", s, N, np.array([[PI, PI, PI]]), 10, 1e-6,
                    extra={"lattice": FCC_CELL, "geometry": "diamond", "r": 0.12, "b": 0.11, "eps_in": 13.0})
