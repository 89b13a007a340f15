"""Pins of the oracle's eigensolvers (LOBPCG, Algorithm 4.1, k = 0 handling) against dense LAPACK."""
import numpy as np

import workloads as wl
from oracle import eigs, geometry, mfd, rng


def sphere_m0(N):
    s = wl.sc_single_sphere()
    return geometry.m0_from_structure(N, s.as_array(), s.eps_bg)


def test_lobpcg_matches_dense():
    N = 6
    h = 1.0 / N
    k = np.array([1.3, 0.4, -0.9])
    m0 = sphere_m0(N)
    g = mfd.penalty_gamma(h, k)
    out = eigs.solve_kpoint(N, k, m0, 6, 1e-11, guard=3)
    assert out["doublings"] == 0
    w, _ = eigs.lowest_dense(mfd.compensated_operator(N, k, h, m0, g), 6)
    assert np.max(np.abs(out["evals"] - w) / w) < 1e-11


def test_gamma_point_deflation_matches_dense():
    """k = 0: the lowest nonzero eigenvalues, the 3 constant fields projected out."""
    N = 6
    h = 1.0 / N
    k = np.zeros(3)
    m0 = sphere_m0(N)
    out = eigs.solve_kpoint(N, k, m0, 6, 1e-11, guard=3)
    w, _ = eigs.lowest_dense(mfd.compensated_operator(N, k, h, m0, 2.0 / h), 6, skip=3)
    assert np.max(np.abs(out["evals"] - w) / w) < 1e-10


def test_recompute_values_of_dense_eigenvectors():
    """lambda_re (Algorithm 4.1) equals lambda on physical eigenvectors and is 0 on compensation ones."""
    N = 6
    h = 1.0 / N
    k = np.array([0.3, 0.1, 0.2])
    m0 = sphere_m0(N)
    g = 1.0  # small penalty: compensation eigenvalues gamma*sigma appear among the lowest
    Op = mfd.compensated_operator(N, k, h, m0, g)
    w, V = eigs.lowest_dense(Op, 8)
    Ah, B = mfd.half_operators(N, k, h)
    lam_re, spurious = eigs.recompute_check(V, w, m0, Ah, 1e-10)
    sig = np.sort(geometry_free_sigma(N, h, k))
    comp = np.isclose(w[:, None], g * sig[None, :8], rtol=1e-9).any(axis=1)
    assert comp.any() and (~comp).any()
    assert np.all(spurious == comp)
    assert np.allclose(lam_re[comp], 0.0, atol=1e-9)
    assert np.allclose(lam_re[~comp], w[~comp], rtol=1e-9)


def geometry_free_sigma(N, h, k):
    from oracle.spectrum import sigma_grid
    return sigma_grid(N, h, k).ravel()


def test_algorithm_4_1_doubles_gamma_until_clean():
    """With a small gamma the compensation eigenvalue gamma |k|^2 enters the lowest bands; Algorithm 4.1 doubles
    gamma until the result equals the nonzero spectrum of A M0 A'."""
    N = 6
    h = 1.0 / N
    k = np.array([0.3, 0.1, 0.2])
    m0 = sphere_m0(N)
    out = eigs.solve_kpoint(N, k, m0, 6, 1e-11, guard=3, gamma=1.0)
    assert out["doublings"] >= 1 and not out["spurious"].any()
    wa = np.linalg.eigvalsh(mfd.curl_part(N, k, h, m0).toarray())
    phys = np.sort(wa[wa > 1e-10 * wa.max()])[:6]
    assert np.max(np.abs(out["evals"] - phys) / phys) < 1e-10


def test_reduce_to_first_zone():
    assert np.array_equal(eigs.reduce_to_first_zone([0.0, 2 * np.pi, 0.0]), np.zeros(3))
    assert np.allclose(eigs.reduce_to_first_zone([1.5 * np.pi, 1.5 * np.pi, 0.0]), [-0.5 * np.pi, -0.5 * np.pi, 0])
    assert np.allclose(eigs.reduce_to_first_zone([np.pi, np.pi, np.pi]), [np.pi, np.pi, np.pi])


def test_rng_splitmix64_reference_outputs():
    """mix64 is splitmix64's output function: seeded with 0, splitmix64 returns mix64(G), mix64(2G), mix64(3G) =
    0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F (published reference sequence)."""
    G = 0x9E3779B97F4A7C15
    got = [int(rng.mix64(np.uint64((i * G) & 0xFFFFFFFFFFFFFFFF))) for i in (1, 2, 3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_rng_complex_normal_moments():
    z = rng.complex_normal(7, 3, 200000)
    assert abs(z.mean()) < 0.01
    assert abs(np.mean(np.abs(z) ** 2) - 2.0) < 0.02
    assert abs(np.mean(z.real * z.imag)) < 0.01
    assert not np.array_equal(rng.complex_normal(7, 4, 8), rng.complex_normal(7, 3, 8))


def test_previous_k_start_cuts_iterations():
    """Starting LOBPCG from the eigenvectors of the previous k-point of a path (the fallback warm start) reaches the
    same eigenvalues in markedly fewer iterations than the random block: FCC spheres at N = 8, four consecutive
    k-points of the 40-point path, 6 bands to 1e-6."""
    import workloads as wl
    from oracle import geometry
    from oracle.rng import initial_block
    N, nb = 8, 6
    st = wl.fcc_spheres()
    m0 = geometry.m0_from_structure(N, st.as_array(), st.eps_bg).ravel()
    path = wl.kpath(wl.FCC_PATH, wl.FCC_POINTS, 40)
    prev = eigs.solve_kpoint(N, path[5], m0, nb, 1e-6, guard=4)["evecs"]
    tot_random = tot_warm = 0
    for i in (6, 7, 8):
        base = eigs.solve_kpoint(N, path[i], m0, nb, 1e-6, guard=4)
        X0 = initial_block(0, 0, 3 * N ** 3, nb + 4)
        X0[:, :nb] = prev
        warm = eigs.solve_kpoint(N, path[i], m0, nb, 1e-6, guard=4, X0=X0)
        assert np.max(np.abs(warm["evals"] - base["evals"]) / base["evals"]) <= 1e-9
        tot_random += base["iters"]
        tot_warm += warm["iters"]
        prev = base["evecs"]
    assert tot_warm <= 0.8 * tot_random
