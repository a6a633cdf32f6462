"""Pins of the oracle's polynomial two-body Jastrow term u (paper Sec. 2.3,
Eq. (8)): the Kato cusp slope it is built to have, its smooth cut-off at L_u,
finite differences, a closed form, nearest-image and spin bookkeeping and
the symmetries of a pair sum."""
import math

import numpy as np
import pytest

import oracle
from paper_2507_02888_gb300 import inputs as I

A_LIKE = [0.31, 0.0, -0.02, 0.004, 1e-3, -2e-4, 3e-5]
A_UNLIKE = [0.55, 0.0, 0.03, -0.006, 5e-4, 1e-4, -1e-5]


def _cell(dim):
    return (I.fcc_lattice(16, 1.2) if dim == 3 else I.hex_lattice(16, 1.2))


def _lu(lat, frac=0.9):
    """frac of half the shortest lattice vector (searching small combinations)."""
    dim = lat.shape[0]
    rng = range(-2, 3)
    best = 1e300
    for m in np.array(np.meshgrid(*([rng] * dim))).reshape(dim, -1).T:
        if np.any(m):
            best = min(best, np.linalg.norm(m @ lat))
    return frac * best / 2


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("like", [True, False])
def test_cusp_slope(dim, like):
    # two particles 1e-7 apart: |grad| = u'(0+) = Gamma (Kato), 3D 1/4 like,
    # 1/2 unlike; 2D 1/3 like, 1 unlike
    lat = _cell(dim)
    L = _lu(lat)
    pos = np.zeros((2, dim))
    pos[1, 0] = 1e-7
    _, g, _ = oracle.jastrow_u(dim, lat, pos + 0.3, 2 if like else 1, L, 3, A_LIKE, A_UNLIKE)
    gamma = {(3, True): 0.25, (3, False): 0.5, (2, True): 1 / 3, (2, False): 1.0}[(dim, like)]
    assert abs(np.linalg.norm(g[0]) - gamma) < 1e-5
    assert g[0][0] < 0 < g[1][0]          # grad_0 = u'(r) (r_0 - r_1)/r points away from 1


@pytest.mark.parametrize("C", [2, 3])
def test_smooth_cutoff(C):
    # u ~ (L - r)^C near L: halving the gap divides J by 2^C and grad by 2^(C-1)
    lat = _cell(3)
    L = _lu(lat)
    vals = []
    for h in (1e-3, 5e-4):
        pos = np.array([[0.1, 0.2, 0.3], [0.1 + L * (1 - h), 0.2, 0.3]])
        j, g, _ = oracle.jastrow_u(3, lat, pos, 1, L, C, A_LIKE, A_UNLIKE)
        vals.append((j, g[0, 0]))
    assert abs(vals[0][0] / vals[1][0] - 2 ** C) < 0.02 * 2 ** C
    assert abs(vals[0][1] / vals[1][1] - 2 ** (C - 1)) < 0.02 * 2 ** (C - 1)
    pos = np.array([[0.1, 0.2, 0.3], [0.1 + L * 1.0001, 0.2, 0.3]])
    j, g, lap = oracle.jastrow_u(3, lat, pos, 1, L, C, A_LIKE, A_UNLIKE)
    assert j == 0.0 and not np.any(g) and not np.any(lap)


@pytest.mark.parametrize("dim", [2, 3])
def test_derivatives_match_finite_differences(dim):
    rng = np.random.default_rng(8)
    lat = _cell(dim)
    L = _lu(lat)
    n = 10
    pos = rng.random((n, dim)) @ lat
    j0, g, lap = oracle.jastrow_u(dim, lat, pos, 4, L, 3, A_LIKE, A_UNLIKE)
    h1, h2 = 1e-6, 1e-4
    for i in (0, 6):
        lp = 0.0
        for k in range(dim):
            p = pos.copy(); p[i, k] += h1
            m = pos.copy(); m[i, k] -= h1
            fd = (oracle.jastrow_u(dim, lat, p, 4, L, 3, A_LIKE, A_UNLIKE)[0] -
                  oracle.jastrow_u(dim, lat, m, 4, L, 3, A_LIKE, A_UNLIKE)[0]) / (2 * h1)
            assert abs(fd - g[i, k]) < 1e-7 * max(1.0, abs(g[i, k]))
            p = pos.copy(); p[i, k] += h2
            m = pos.copy(); m[i, k] -= h2
            lp += (oracle.jastrow_u(dim, lat, p, 4, L, 3, A_LIKE, A_UNLIKE)[0] - 2 * j0 +
                   oracle.jastrow_u(dim, lat, m, 4, L, 3, A_LIKE, A_UNLIKE)[0]) / h2 ** 2
        assert abs(lp - lap[i]) < 1e-5 * max(1.0, abs(lap[i]))


def test_closed_form_with_alpha0_zero():
    # alpha_0 = 0 and no higher terms: u(r) = Gamma r (1 - r/L)^C
    lat = _cell(3)
    L = _lu(lat)
    r = 0.37 * L
    pos = np.array([[0.5, 0.5, 0.5], [0.5, 0.5 + r, 0.5]])
    for like, gamma in ((True, 0.25), (False, 0.5)):
        j, _, _ = oracle.jastrow_u(3, lat, pos, 2 if like else 1, L, 3, [0.0, 0.0], [0.0, 0.0])
        assert abs(j - gamma * r * (1 - r / L) ** 3) < 1e-15


def test_nearest_image_and_symmetries():
    rng = np.random.default_rng(3)
    lat = _cell(3)
    L = _lu(lat, 0.99)
    n = 12
    pos = rng.random((n, 3)) @ lat
    j0, g0, l0 = oracle.jastrow_u(3, lat, pos, 5, L, 2, A_LIKE, A_UNLIKE)
    # lattice moves of single particles, a common translation
    p = pos.copy()
    p[2] += lat[0] - 2 * lat[2]
    p[7] -= lat[1]
    j1, g1, l1 = oracle.jastrow_u(3, lat, p + rng.normal(size=3), 5, L, 2, A_LIKE, A_UNLIKE)
    assert abs(j1 - j0) < 1e-12 * max(1, abs(j0)) and np.allclose(g1, g0, atol=1e-12) and np.allclose(l1, l0)
    # permutations inside each spin species
    perm = np.concatenate([rng.permutation(5), 5 + rng.permutation(7)])
    j2, g2, _ = oracle.jastrow_u(3, lat, pos[perm], 5, L, 2, A_LIKE, A_UNLIKE)
    assert abs(j2 - j0) < 1e-12 * max(1, abs(j0)) and np.allclose(g2, g0[perm], atol=1e-12)
    # flipping every spin leaves like / unlike pairs as they are
    j3, _, _ = oracle.jastrow_u(3, lat, np.concatenate([pos[5:], pos[:5]]), 7, L, 2, A_LIKE, A_UNLIKE)
    assert abs(j3 - j0) < 1e-12 * max(1, abs(j0))
    # all spins alike: only the like set enters
    ja, _, _ = oracle.jastrow_u(3, lat, pos, n, L, 2, A_LIKE, A_UNLIKE)
    jb, _, _ = oracle.jastrow_u(3, lat, pos, 0, L, 2, A_LIKE, [9.0] * len(A_LIKE))
    assert abs(ja - jb) < 1e-13 * max(1, abs(ja))
    # sum of gradients vanishes (pair forces cancel)
    assert np.max(np.abs(g0.sum(axis=0))) < 1e-12


def test_pair_across_the_boundary_uses_the_nearest_image():
    lat = _cell(3)
    L = _lu(lat)
    d = np.array([0.2, -0.5, 0.3]) * L / np.linalg.norm([0.2, -0.5, 0.3]) * 0.8
    a = np.array([0.05, 0.1, 0.02])
    inside = oracle.jastrow_u(3, lat, np.array([a, a + d]), 1, L, 3, A_LIKE, A_UNLIKE)[0]
    across = oracle.jastrow_u(3, lat, np.array([a, a + d + lat[1] - lat[2]]), 1, L, 3, A_LIKE, A_UNLIKE)[0]
    assert inside != 0.0 and abs(inside - across) < 1e-14


def test_refuses_a_cutoff_beyond_half_the_shortest_lattice_vector():
    lat = _cell(3)
    with pytest.raises(oracle.OracleError):
        oracle.jastrow_u(3, lat, np.zeros((2, 3)) + [[0, 0, 0], [1, 0, 0]], 1, _lu(lat, 1.01), 3, A_LIKE, A_UNLIKE)
