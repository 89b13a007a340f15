"""Band-gap ratio of Section 6.2 (host post-processing) on hand-made band structures, and the BCC path."""
import numpy as np

import workloads as wl
from paper_2503_19379_gb300 import bands


def test_gap_ratio_by_hand():
    # frequencies: band 1 in [1, 2], band 2 in [3, 4] -> gap 2..3: ratio (3 - 2) / 2.5 = 0.4; band 3 overlaps band 2
    w = np.array([[1.0, 3.0, 3.5], [2.0, 4.0, 4.5], [1.5, 3.2, 3.9]])
    r = bands.gap_ratios(w ** 2)
    assert np.allclose(r, [0.4, 0.0])
    assert bands.largest_gap(w ** 2) == (1, 0.4)


def test_no_gap():
    w = np.array([[1.0, 2.0], [2.5, 3.0]])
    assert bands.largest_gap(w ** 2) == (0, 0.0)


def test_bcc_path_visits_every_point():
    k = wl.kpath(wl.BCC_PATH, wl.BCC_POINTS, 30)
    for p in wl.BCC_POINTS.values():
        assert np.min(np.linalg.norm(k - np.asarray(p), axis=1)) == 0.0
    # H and H' are equivalent in the BCC lattice: they differ by a reciprocal-lattice vector of the primitive cell
    d = np.asarray(wl.BCC_POINTS["H"]) - np.asarray(wl.BCC_POINTS["H'"])
    f = wl.BCC_CELL.T @ d / (2 * np.pi)
    assert np.allclose(f, np.round(f))
