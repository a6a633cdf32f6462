"""Pins for the FP64 CPU oracle (no GPU).

Each test ties the oracle to something other than itself: literature
Madelung energies, the independence of the total from the splitting
parameter, symmetry invariances, the continuity of v_E(r) - 1/r at r -> 0
(paper Sec. 2.2, Eqs. (3)-(4)), a brute-force identity for the reciprocal
sum, brute-force image sums with a huge image box, and the single-move
energy change against two full energies (Sec. 2.1).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import erfc

import oracle
from paper_2507_02888_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "madelung.json")))


def scale(comp):
    """S = |E_real| + |E_recip| + |E_madR + E_self| + |E_bg| (floor for relative errors)."""
    return abs(comp[0]) + abs(comp[2]) + abs(comp[1] + comp[3]) + abs(comp[4])


def energy(dim, lat, pos, q, alpha, tol=1e-16):
    rc, gc = oracle.cutoffs(dim, alpha, tol)
    return oracle.energy(dim, lat, pos, q, alpha, rc, gc)


# ---------------------------------------------------------------- P1, P2, P8

@pytest.mark.parametrize("rs", [1.0, 2.0, 5.0])
def test_bcc_wigner_primitive(rs):
    g = GOLD["bcc_wigner_3d"]
    lat = I.bcc_primitive_lattice(rs)
    alpha = 2.0 / abs(np.linalg.det(lat)) ** (1 / 3)
    e, _ = energy(3, lat, np.zeros((1, 3)), [-1.0], alpha)
    assert abs(e * rs - g["value_times_rs"]) < g["tol"]
    assert abs(e * rs - (-0.895929)) < 5e-7


@pytest.mark.parametrize("m", [1, 3])
def test_bcc_wigner_conventional_supercell(m):
    # m = 3 is the 54-electron simple-cubic cell of the small 3D workload, alpha = 2.8/L.
    g = GOLD["bcc_wigner_3d"]
    lat, pos = I.bcc_crystal(m, 1.0)
    n = len(pos)
    e, _ = energy(3, lat, pos, -np.ones(n), 2.8 / lat[0, 0])
    assert abs(e / n - g["value_times_rs"]) < g["tol"]


@pytest.mark.parametrize("m", [1, 18, 19])
def test_hex_wigner_2d(m):
    g = GOLD["hex_wigner_2d"]
    rs = 5.0
    lat, pos = I.hex_crystal(m, rs)
    n = len(pos)
    alpha = 4.0 / math.sqrt(abs(np.linalg.det(lat)))
    e, _ = energy(2, lat, pos, -np.ones(n), alpha)
    assert abs(e / n * rs - g["value_times_rs"]) < g["tol"]


def test_rocksalt_madelung():
    g = GOLD["rocksalt"]
    a = 2.0
    lat, pos, q = I.rocksalt_cell(a)
    e, comp = energy(3, lat, pos, q, 2.0)
    r_nn = a / 2
    assert comp[4] == 0.0                         # neutral cell: no background
    assert abs(-e / 4 * r_nn - g["madelung_constant"]) < g["tol"]


# ---------------------------------------------------------------- P3

@pytest.mark.parametrize("case", ["sc", "fcc", "hex", "ions"])
def test_alpha_independence(case):
    rng = np.random.default_rng(11)
    if case == "sc":
        dim, lat, n = 3, I.sc_lattice(20, 1.5), 20
        pos, q = I.uniform_positions(rng, lat, 1, n)[0], -np.ones(n)
    elif case == "fcc":
        dim, lat, n = 3, I.fcc_lattice(24, 2.0), 24
        pos, q = I.uniform_positions(rng, lat, 1, n)[0], -np.ones(n)
    elif case == "hex":
        dim, lat, n = 2, I.hex_lattice(30, 3.0), 30
        pos, q = I.uniform_positions(rng, lat, 1, n)[0], -np.ones(n)
    else:
        lat, ions = I.diamond_ions(1, 6.74)
        dim = 3
        el = I.scattered_positions(rng, ions, 1, 32, 0.8)[0]
        pos = np.concatenate([el, ions])
        q = np.concatenate([-np.ones(32), 4.0 * np.ones(len(ions))])
    alpha0 = 5.0 / abs(np.linalg.det(lat)) ** (1 / dim)
    res = [energy(dim, lat, pos, q, alpha0 * f) for f in (0.6, 1.0, 1.6)]
    s = max(scale(c) for _, c in res)
    for e, c in res[1:]:
        assert abs(e - res[0][0]) < 1e-10 * max(abs(res[0][0]), 1e-2 * s)
    # The split itself must really move: the parts change a lot with alpha.
    assert abs(res[0][1][0] - res[2][1][0]) > 1e-2 * s


# ---------------------------------------------------------------- P4, P9

def _random_system(dim, seed, n=18):
    rng = np.random.default_rng(seed)
    lat = I.fcc_lattice(n, 1.7) if dim == 3 else I.hex_lattice(n, 2.5)
    pos = I.uniform_positions(rng, lat, 1, n)[0]
    q = np.where(np.arange(n) % 3 == 0, 2.0, -1.0)
    alpha = 4.5 / abs(np.linalg.det(lat)) ** (1 / dim)
    return lat, pos, q, alpha


@pytest.mark.parametrize("dim", [2, 3])
def test_invariances(dim):
    lat, pos, q, alpha = _random_system(dim, 5)
    e0, c0 = energy(dim, lat, pos, q, alpha)
    tol = 1e-12 * scale(c0)
    rng = np.random.default_rng(6)
    e_t, _ = energy(dim, lat, pos + rng.normal(size=dim) * 3.0, q, alpha)    # translation
    perm = rng.permutation(len(q))
    e_p, _ = energy(dim, lat, pos[perm], q[perm], alpha)                      # permutation
    shifted = pos.copy()
    shifted[4] += 2 * lat[0] - lat[dim - 1]                                   # lattice vector
    e_l, _ = energy(dim, lat, shifted, q, alpha)
    assert abs(e_t - e0) < tol and abs(e_p - e0) < tol and abs(e_l - e0) < tol


@pytest.mark.parametrize("dim", [2, 3])
def test_unimodular_basis_change(dim):
    lat, pos, q, alpha = _random_system(dim, 7)
    U = np.array([[1, 2, 0], [0, 1, 0], [1, 1, 1]]) if dim == 3 else np.array([[2, 1], [1, 1]])
    assert round(abs(np.linalg.det(U))) == 1
    lat2 = U @ lat
    e0, c0 = energy(dim, lat, pos, q, alpha)
    e1, _ = energy(dim, lat2, pos, q, alpha)
    assert abs(e1 - e0) < 1e-12 * scale(c0)


# ---------------------------------------------------------------- P5

@pytest.mark.parametrize("dim", [2, 3])
def test_delta_e_against_two_energies(dim):
    lat, pos, q, alpha = _random_system(dim, 8)
    rc, gc = oracle.cutoffs(dim, alpha)
    e0, c0 = oracle.energy(dim, lat, pos, q, alpha, rc, gc)
    rng = np.random.default_rng(9)
    for k in (0, 4, 11):
        r_new = pos[k] + rng.normal(size=dim) * 0.7
        de = oracle.delta_e(dim, lat, pos, q, k, r_new, alpha, rc, gc)
        moved = pos.copy()
        moved[k] = r_new
        e1, _ = oracle.energy(dim, lat, moved, q, alpha, rc, gc)
        assert abs(de - (e1 - e0)) < 1e-11 * scale(c0)
        assert abs(de) > 1e-6


@pytest.mark.parametrize("dim", [2, 3])
def test_delta_e_parts_against_two_energies(dim):
    """The real-space and reciprocal parts of a move each equal the change of
    that piece between two full energies (the other pieces do not move)."""
    lat, pos, q, alpha = _random_system(dim, 8)
    rc, gc = oracle.cutoffs(dim, alpha)
    _, c0 = oracle.energy(dim, lat, pos, q, alpha, rc, gc)
    rng = np.random.default_rng(19)
    for k in (1, 6):
        r_new = pos[k] + rng.normal(size=dim) * 0.7
        d_real, d_recip = oracle.delta_e_parts(dim, lat, pos, q, k, r_new, alpha, rc, gc)
        moved = pos.copy()
        moved[k] = r_new
        _, c1 = oracle.energy(dim, lat, moved, q, alpha, rc, gc)
        assert abs(d_real - (c1[0] - c0[0])) < 1e-11 * scale(c0)
        assert abs(d_recip - (c1[2] - c0[2])) < 1e-11 * scale(c0)
        assert np.array_equal(c1[[1, 3, 4]], c0[[1, 3, 4]])
        assert abs(d_real + d_recip - oracle.delta_e(dim, lat, pos, q, k, r_new, alpha, rc, gc)) < 1e-14 * scale(c0)


# ---------------------------------------------------------------- P6

@pytest.mark.parametrize("dim,n", [(3, 2), (3, 4), (2, 3)])
def test_rho_against_pair_double_sum(dim, n):
    lat, pos, q, alpha = _random_system(dim, 10, n=n)
    rc, gc = oracle.cutoffs(dim, alpha)
    _, comp = oracle.energy(dim, lat, pos, q, alpha, rc, gc)
    e_pairs = oracle.recip_pairsum(dim, lat, pos, q, alpha, gc)
    assert abs(comp[2] - e_pairs) < 1e-12 * abs(e_pairs)


def test_rho_at_phase_sign_one_particle():
    """rho(G) = q e^{+iG.r} for one particle: the sign of the phase, which
    conjugate symmetry, the origin value and periodicity leave open."""
    lat = np.array([[5.0, 0.0, 0.0], [1.0, 4.0, 0.0], [0.5, -0.7, 6.0]])
    r = np.array([[0.9, 1.3, -0.4]])
    nv = np.array([[1, 0, 0], [0, 2, -1], [3, -1, 2]])
    B = 2 * np.pi * np.linalg.inv(lat).T                 # rows b_k, a_i . b_k = 2 pi delta_ik
    rho = oracle.rho_at(3, lat, r, np.array([2.5]), nv)
    for g, n in enumerate(nv):
        ph = (n @ B) @ r[0]
        assert abs(rho[g] - 2.5 * complex(math.cos(ph), math.sin(ph))) < 1e-13
    # a quarter period along a_1 turns rho(b_1) by +i
    rq = oracle.rho_at(3, lat, 0.25 * lat[:1], np.array([1.0]), nv[:1])[0]
    assert abs(rq - 1j) < 1e-14


def test_rho_at_conjugate_symmetry_and_origin():
    lat, pos, q, _ = _random_system(3, 12, n=6)
    nv = np.array([[1, 0, 0], [-1, 0, 0], [2, -1, 3], [-2, 1, -3], [0, 0, 0]])
    rho = oracle.rho_at(3, lat, pos, q, nv)
    assert abs(rho[0] - np.conj(rho[1])) < 1e-13 and abs(rho[2] - np.conj(rho[3])) < 1e-13
    assert abs(rho[4] - q.sum()) < 1e-13
    # rho is periodic: moving a particle by a lattice vector leaves it unchanged
    p2 = pos.copy()
    p2[2] += lat[1] - 3 * lat[2]
    assert np.max(np.abs(oracle.rho_at(3, lat, p2, q, nv) - rho)) < 1e-11


# ---------------------------------------------------------------- P7

def test_supercell_consistency_bcc_and_hex():
    lat1, pos1 = I.bcc_crystal(1, 1.3)
    lat2, pos2 = I.bcc_crystal(2, 1.3)
    e1, _ = energy(3, lat1, pos1, -np.ones(len(pos1)), 2.8 / lat1[0, 0])
    e2, _ = energy(3, lat2, pos2, -np.ones(len(pos2)), 2.8 / lat2[0, 0])
    assert abs(e2 - 8 * e1) < 1e-12 * abs(e2)
    h1, p1 = I.hex_crystal(1, 2.0)
    h3, p3 = I.hex_crystal(3, 2.0)
    a1 = 4.0 / math.sqrt(abs(np.linalg.det(h1)))
    a3 = 4.0 / math.sqrt(abs(np.linalg.det(h3)))
    e1, _ = energy(2, h1, p1, [-1.0], a1)
    e3, _ = energy(2, h3, p3, -np.ones(9), a3)
    assert abs(e3 - 9 * e1) < 1e-12 * abs(e3)


# ---------------------------------------------------------------- P10

@pytest.mark.parametrize("dim", [2, 3])
def test_continuity_pair_to_single_charge(dim):
    # E(pair at separation s) - q1 q2 / s -> energy of one charge q1 + q2 as s -> 0
    lat = I.sc_lattice(4, 1.0) if dim == 3 else I.hex_lattice(4, 1.0)
    alpha = 4.0 / abs(np.linalg.det(lat)) ** (1 / dim)
    s = 1e-4
    x0 = 0.3 * lat[0] + 0.2 * lat[1]
    pos = np.array([x0, x0 + s * np.eye(dim)[0]])
    e_pair, _ = energy(dim, lat, pos, [-1.0, -1.0], alpha)
    e_one, _ = energy(dim, lat, x0[None, :], [-2.0], alpha)
    assert abs((e_pair - 1.0 / s) - e_one) < 1e-7


# ---------------------------------------------------------------- enumeration bounds

def _brute_real(dim, lat, pos, q, alpha, rc):
    """Real-space sum over a generous image box (tiny N only).

    The box is twice what the unwrapped displacements could need, so it does
    not rely on the oracle's wrapping or its per-pair bound.
    """
    b = 2 * np.pi * np.linalg.inv(lat).T
    dmax = max(np.linalg.norm(pos[i] - pos[j]) for i in range(len(q)) for j in range(len(q)))
    box = int(2 * math.ceil((rc + dmax) * np.max(np.linalg.norm(b, axis=1)) / (2 * np.pi))) + 2
    rng_m = range(-box, box + 1)
    Rs = [np.array(m) @ lat for m in np.array(np.meshgrid(*([rng_m] * dim))).reshape(dim, -1).T]
    tot = 0.0
    for i in range(len(q)):
        for j in range(i + 1, len(q)):
            for R in Rs:
                r = np.linalg.norm(pos[i] - pos[j] + R)
                if r < rc:
                    tot += q[i] * q[j] * erfc(alpha * r) / r
    return tot


@pytest.mark.parametrize("dim", [2, 3])
def test_image_box_is_sufficient_in_skewed_cell(dim):
    # A strongly skewed cell and particles far outside the home cell.
    lat = np.array([[3.0, 0, 0], [2.7, 1.2, 0], [0.4, 0.9, 2.5]]) if dim == 3 else \
        np.array([[3.0, 0.0], [2.8, 0.9]])
    rng = np.random.default_rng(3)
    pos = rng.normal(size=(3, dim)) * 3.0
    q = np.array([1.0, -2.0, 1.5])
    alpha = 0.9
    rc, gc = oracle.cutoffs(dim, alpha, 1e-8)
    _, comp = oracle.energy(dim, lat, pos, q, alpha, rc, gc)
    ref = _brute_real(dim, lat, pos, q, alpha, rc)
    assert abs(comp[0] - ref) < 1e-12 * max(1.0, abs(ref))


def test_gcount_against_wide_box():
    lat = I.fcc_lattice(16, 1.0)
    gc = 5.0
    b = 2 * np.pi * np.linalg.inv(lat).T
    m = np.arange(-12, 13)
    n = np.array(np.meshgrid(m, m, m)).reshape(3, -1).T
    g = np.linalg.norm(n @ b, axis=1)
    assert oracle.gcount(3, lat, gc) == int(np.sum((g > 0) & (g <= gc)))


def test_cutoffs_meet_tolerance():
    for dim in (2, 3):
        rc, gc = oracle.cutoffs(dim, 0.7, 1e-16)
        assert abs(erfc(0.7 * rc) / 1e-16 - 1) < 1e-6
        w = math.exp(-gc ** 2 / (4 * 0.49)) if dim == 3 else erfc(gc / 1.4)
        assert abs(w / 1e-16 - 1) < 1e-6


def test_coincident_particles_rejected():
    lat = I.sc_lattice(2, 1.0)
    pos = np.array([[0.1, 0.2, 0.3], [0.1, 0.2, 0.3] + lat[0]])
    with pytest.raises(oracle.OracleError):
        energy(3, lat, pos, [-1.0, -1.0], 1.0)
