"""Pins of the oracle's 2D energy with charges at heights z != 0 (paper
Sec. 2.2, Eqs. (5)-(6) at z != 0): reduction to the in-plane energy, alpha
independence, the Fourier series of a charged sheet lattice (Poisson's
equation solved directly, no splitting), the charged-sheet limit of far
layers, invariances and the move energy change."""
import math

import numpy as np
import pytest

import oracle
from paper_2507_02888_gb300 import inputs as I


def _bilayer(n=12, d=2.5, seed=4, cell=None):
    rng = np.random.default_rng(seed)
    lat = I.hex_lattice(n, 1.6) if cell is None else cell
    pos = rng.random((n, 2)) @ lat
    z = np.where(np.arange(n) < n // 2, 0.0, d)
    q = np.where(np.arange(n) < n // 2, -1.0, 1.0)
    q[0] = q[n // 2] = -1.0                        # layers of unequal charge: a net field between them
    return lat, pos, z, q


def _cut(alpha):
    return oracle.cutoffs(2, alpha)


def _scale(comp):
    return abs(comp[0]) + abs(comp[2]) + abs(comp[1] + comp[3]) + abs(comp[4])


def test_equal_heights_reduce_to_the_plane():
    lat, pos, _, q = _bilayer()
    alpha = 4.0 / math.sqrt(abs(np.linalg.det(lat)))
    rc, gc = _cut(alpha)
    e0, c0 = oracle.energy(2, lat, pos, q, alpha, rc, gc)
    for h in (0.0, 3.7, -11.0):
        e, c = oracle.energy_z(lat, pos, np.full(len(q), h), q, alpha, rc, gc)
        assert abs(e - e0) <= 1e-12 * _scale(c0)
        assert np.allclose(c, c0, rtol=0, atol=1e-12 * _scale(c0))


@pytest.mark.parametrize("d", [0.4, 2.5, 9.0])
def test_alpha_independence(d):
    lat, pos, z, q = _bilayer(d=d)
    a0 = 4.0 / math.sqrt(abs(np.linalg.det(lat)))
    es = []
    for f in (0.6, 1.0, 1.6):
        rc, gc = _cut(a0 * f)
        es.append(oracle.energy_z(lat, pos, z, q, a0 * f, rc, gc))
    s = _scale(es[1][1])
    assert max(abs(e[0] - es[1][0]) for e in es) <= 1e-10 * s
    # the split moves weight between the pieces, so they differ
    assert abs(es[0][1][0] - es[2][1][0]) > 1e-3 * s


def _sheet_potential(lat, rho, z, g_max):
    """Potential at (rho, z), z != 0, of unit charges on the 2D lattice with no
    background, from the in-plane Fourier series of Poisson's equation:
    (2 pi / A) sum_{G != 0} e^{-G|z|} / G cos(G.rho) - 2 pi |z| / A."""
    A = abs(np.linalg.det(lat))
    B = 2 * math.pi * np.linalg.inv(lat).T
    nmax = [int(math.ceil(g_max * np.linalg.norm(lat[k]) / (2 * math.pi))) for k in range(2)]
    n1, n2 = np.meshgrid(np.arange(-nmax[0], nmax[0] + 1), np.arange(-nmax[1], nmax[1] + 1), indexing="ij")
    n = np.stack([n1.ravel(), n2.ravel()], axis=1)
    n = n[np.any(n != 0, axis=1)]
    G = n @ B
    g = np.linalg.norm(G, axis=1)
    keep = g <= g_max
    G, g = G[keep], g[keep]
    return 2 * math.pi / A * (np.sum(np.exp(-g * abs(z)) / g * np.cos(G @ rho)) - abs(z))


@pytest.mark.parametrize("z", [0.3, 1.7, -4.0])
def test_pair_potential_is_the_sheet_fourier_series(z):
    # two unit charges: E = v_E(r_12) + v_M, one charge alone: E = v_M / 2
    lat = I.hex_lattice(7, 1.4)
    alpha = 3.0 / math.sqrt(abs(np.linalg.det(lat)))
    rc, gc = _cut(alpha)
    rho = np.array([1.3, -0.8])
    e2, _ = oracle.energy_z(lat, np.array([[0.0, 0.0], rho]), np.array([0.0, z]), np.ones(2), alpha, rc, gc)
    e1, _ = oracle.energy_z(lat, np.zeros((1, 2)), np.zeros(1), np.ones(1), alpha, rc, gc)
    v_ewald = e2 - 2 * e1
    v_fourier = _sheet_potential(lat, rho, z, 40.0 / abs(z))
    assert abs(v_ewald - v_fourier) <= 1e-11 * max(1.0, abs(v_fourier))


def test_far_layers_interact_as_charged_sheets():
    # separation >> cell: the layers see each other's mean charge only,
    # E - E_1 - E_2 -> -(2 pi / A) Q_1 Q_2 d
    lat, pos, _, q = _bilayer(n=10)
    A = abs(np.linalg.det(lat))
    L = math.sqrt(A)
    alpha = 4.0 / L
    h = len(q) // 2
    d = 6 * L
    rc, gc = _cut(alpha)
    z = np.where(np.arange(len(q)) < h, 0.0, d)
    e, _ = oracle.energy_z(lat, pos, z, q, alpha, rc, gc)
    e1, _ = oracle.energy(2, lat, pos[:h], q[:h], alpha, rc, gc)
    e2, _ = oracle.energy(2, lat, pos[h:], q[h:], alpha, rc, gc)
    expect = -2 * math.pi / A * q[:h].sum() * q[h:].sum() * d
    assert abs((e - e1 - e2) - expect) <= 1e-10 * abs(expect)


def test_invariances():
    lat, pos, z, q = _bilayer()
    alpha = 4.0 / math.sqrt(abs(np.linalg.det(lat)))
    rc, gc = _cut(alpha)
    e0, c0 = oracle.energy_z(lat, pos, z, q, alpha, rc, gc)
    tol = 1e-12 * _scale(c0)
    rng = np.random.default_rng(1)
    assert abs(oracle.energy_z(lat, pos, z + 5.25, q, alpha, rc, gc)[0] - e0) <= tol      # shift in z
    assert abs(oracle.energy_z(lat, pos, -z, q, alpha, rc, gc)[0] - e0) <= tol            # mirror
    perm = rng.permutation(len(q))
    assert abs(oracle.energy_z(lat, pos[perm], z[perm], q[perm], alpha, rc, gc)[0] - e0) <= tol
    assert abs(oracle.energy_z(lat, pos + rng.normal(size=2), z, q, alpha, rc, gc)[0] - e0) <= tol
    p2 = pos.copy()
    p2[3] += 2 * lat[0] - lat[1]
    assert abs(oracle.energy_z(lat, p2, z, q, alpha, rc, gc)[0] - e0) <= tol


def test_move_delta_matches_energy_difference():
    lat, pos, z, q = _bilayer()
    alpha = 4.0 / math.sqrt(abs(np.linalg.det(lat)))
    rc, gc = _cut(alpha)
    e0, c0 = oracle.energy_z(lat, pos, z, q, alpha, rc, gc)
    rng = np.random.default_rng(7)
    for k in (0, 5, 8):
        rn = pos[k] + rng.normal(scale=0.8, size=2)
        de = oracle.delta_e_z(lat, pos, z, q, k, rn, alpha, rc, gc)
        p2 = pos.copy()
        p2[k] = rn
        e1, _ = oracle.energy_z(lat, p2, z, q, alpha, rc, gc)
        assert abs(de - (e1 - e0)) <= 1e-11 * _scale(c0)


def test_refuses_heights_beyond_the_evaluable_range():
    lat, pos, z, q = _bilayer()
    alpha = 4.0 / math.sqrt(abs(np.linalg.det(lat)))
    rc, gc = _cut(alpha)
    with pytest.raises(oracle.OracleError):
        oracle.energy_z(lat, pos, z * 1e4, q, alpha, rc, gc)
