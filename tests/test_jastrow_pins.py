"""Pins of the oracle's two-body plane-wave Jastrow term (paper Sec. 2.3,
Eqs. (7) and (9)): shell counts of textbook lattices, derivatives against
finite differences, the structure-factor identity, a closed form, and the
symmetries of a pair sum of periodic functions."""
import math

import numpy as np
import pytest

import oracle
from paper_2507_02888_gb300 import inputs as I


def test_shell_counts_of_textbook_lattices():
    # simple cubic: number of integer vectors with |n|^2 = 1, 2, 3, 4, 5, 6, 8, 9
    _, st = oracle.jastrow_stars(3, np.eye(3) * 2.7, 8)
    assert np.bincount(st).tolist() == [6, 12, 8, 6, 24, 24, 12, 30]
    # the reciprocal lattice of fcc is bcc: shells of 8, 6, 12, 24, 8, 6
    _, st = oracle.jastrow_stars(3, I.fcc_lattice(4, 1.0), 6)
    assert np.bincount(st).tolist() == [8, 6, 12, 24, 8, 6]
    # the reciprocal lattice of a hexagonal (triangular) lattice is hexagonal
    _, st = oracle.jastrow_stars(2, I.hex_lattice(1, 1.0), 5)
    assert np.bincount(st).tolist() == [6, 6, 6, 12, 6]


def _case(dim, n=7, seed=3):
    rng = np.random.default_rng(seed)
    lat = I.fcc_lattice(n, 1.3) if dim == 3 else I.hex_lattice(n, 1.3)
    pos = rng.random((n, dim)) @ lat
    a = np.array([0.31, -0.12, 0.07, 0.02])
    return lat, pos, a


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_and_laplacian_match_finite_differences(dim):
    lat, pos, a = _case(dim)
    j0, g, lap = oracle.jastrow_p(dim, lat, pos, a)
    h1, h2 = 1e-6, 1e-4
    for i in (0, 3):
        lp = 0.0
        for k in range(dim):
            p = pos.copy(); p[i, k] += h1
            m = pos.copy(); m[i, k] -= h1
            fd = (oracle.jastrow_p(dim, lat, p, a)[0] - oracle.jastrow_p(dim, lat, m, a)[0]) / (2 * h1)
            assert abs(fd - g[i, k]) < 1e-7 * max(1.0, abs(g[i, k]))
            p = pos.copy(); p[i, k] += h2
            m = pos.copy(); m[i, k] -= h2
            lp += (oracle.jastrow_p(dim, lat, p, a)[0] - 2 * j0 + oracle.jastrow_p(dim, lat, m, a)[0]) / h2 ** 2
        assert abs(lp - lap[i]) < 1e-5 * max(1.0, abs(lap[i]))


@pytest.mark.parametrize("dim", [2, 3])
def test_structure_factor_identity(dim):
    # sum_{i<j} cos(G.r_ij) = (|sum_i exp(iG.r_i)|^2 - N) / 2, for each G of a shell
    lat, pos, a = _case(dim)
    nv, st = oracle.jastrow_stars(dim, lat, len(a))
    B = 2 * math.pi * np.linalg.inv(lat).T            # rows b_k, a_i . b_j = 2 pi delta_ij
    G = nv @ B
    rho = np.exp(1j * (pos @ G.T)).sum(axis=0)
    n = pos.shape[0]
    j_sf = 0.5 * np.sum(a[st] * 0.5 * (np.abs(rho) ** 2 - n))    # both signs of every G: factor 1/2
    assert abs(oracle.jastrow_p(dim, lat, pos, a)[0] - j_sf) < 1e-12 * max(1.0, abs(j_sf))


def test_closed_form_two_particles_simple_cubic():
    L, a1 = 3.1, 0.4
    d = np.array([0.37, -1.1, 0.9])
    pos = np.array([[0.2, 0.3, 0.1], [0.2, 0.3, 0.1] + d])
    b = 2 * math.pi / L
    expect = a1 * (math.cos(b * d[0]) + math.cos(b * d[1]) + math.cos(b * d[2]))
    j, g, lap = oracle.jastrow_p(3, np.eye(3) * L, pos, [a1])
    assert abs(j - expect) < 1e-14
    # the first particle's gradient: -dp/dd = a1 b (sin(b d_x), sin(b d_y), sin(b d_z))
    assert np.allclose(g[0], a1 * b * np.sin(b * d), atol=1e-14)
    assert abs(lap[0] - (-a1 * b * b * np.sum(np.cos(b * d)))) < 1e-13


@pytest.mark.parametrize("dim", [2, 3])
def test_symmetries(dim):
    lat, pos, a = _case(dim)
    j0, g0, l0 = oracle.jastrow_p(dim, lat, pos, a)
    # translation of every particle, one particle by a lattice vector, relabelling
    j1, g1, l1 = oracle.jastrow_p(dim, lat, pos + 0.37 * lat[0] - 1.1 * lat[-1], a)
    p2 = pos.copy(); p2[2] += lat[0] - 2 * lat[1]
    j2, g2, l2 = oracle.jastrow_p(dim, lat, p2, a)
    perm = np.array([3, 0, 6, 1, 5, 2, 4])
    j3, g3, l3 = oracle.jastrow_p(dim, lat, pos[perm], a)
    for j, g, l in ((j1, g1, l1), (j2, g2, l2)):
        assert abs(j - j0) < 1e-12 and np.allclose(g, g0, atol=1e-11) and np.allclose(l, l0, atol=1e-11)
    assert abs(j3 - j0) < 1e-12 and np.allclose(g3, g0[perm], atol=1e-11) and np.allclose(l3, l0[perm], atol=1e-11)
    # internal forces sum to zero
    assert np.allclose(g0.sum(axis=0), 0.0, atol=1e-11)
