"""Seeded synthetic inputs shared by the GPU library's tests, the oracle's tests
and the benchmark.

This module only builds cells, particle positions, charges and random move
streams.  It holds none of the Ewald arithmetic, so both the GPU path and the
CPU oracle can take their inputs from it.

Random numbers come from NumPy's ``default_rng`` (PCG64, seeded).  Positions
are returned as Cartesian float64 arrays of shape ``(W, N, dim)``; lattices
as ``(dim, dim)`` arrays whose rows are the lattice vectors (bohr).

The workloads stand in for the paper's test systems (Sec. 5.1: 3D electron
gas with 100 to 1630 electrons; Sec. 8.1: 2D electron gas with 100 to 1642
electrons; Sec. 8.2: a bulk solid).  The paper's runs used trained wave
functions that are not available, so electrons are placed uniformly at random
(electron gases) or Gaussian-scattered around ions (bulk solid).
"""
import math

import numpy as np

SEED_BASE = 20250702


def rng_for(tag):
    """Generator for a workload tag (an int offset from the base seed)."""
    return np.random.default_rng(SEED_BASE + int(tag))


# --------------------------------------------------------------------------
# Cells.  Volume per electron is 4 pi r_s^3 / 3 (3D) or pi r_s^2 (2D).
# --------------------------------------------------------------------------

def sc_lattice(n, rs):
    """Simple-cubic cell holding n electrons at density parameter rs."""
    L = (n * 4.0 * math.pi / 3.0) ** (1.0 / 3.0) * rs
    return np.diag([L, L, L])


def fcc_lattice(n, rs):
    """fcc-shaped (primitive fcc vectors) cell of volume n * 4 pi rs^3 / 3."""
    omega = n * 4.0 * math.pi / 3.0 * rs ** 3
    a = (4.0 * omega) ** (1.0 / 3.0)
    return 0.5 * a * np.array([[0.0, 1.0, 1.0], [1.0, 0.0, 1.0], [1.0, 1.0, 0.0]])


def bcc_primitive_lattice(rs):
    """Primitive bcc cell holding one electron at density rs."""
    omega = 4.0 * math.pi / 3.0 * rs ** 3
    a = (2.0 * omega) ** (1.0 / 3.0)
    return 0.5 * a * np.array([[-1.0, 1.0, 1.0], [1.0, -1.0, 1.0], [1.0, 1.0, -1.0]])


def hex_lattice(n, rs):
    """Hexagonal (60 degree) 2D cell of area n * pi * rs^2."""
    area = n * math.pi * rs ** 2
    a = math.sqrt(2.0 * area / math.sqrt(3.0))
    return np.array([[a, 0.0], [0.5 * a, 0.5 * math.sqrt(3.0) * a]])


def bcc_crystal(m, rs):
    """m x m x m supercell of the conventional bcc cube: (lattice, positions (2 m^3, 3))."""
    omega1 = 4.0 * math.pi / 3.0 * rs ** 3
    a = (2.0 * omega1) ** (1.0 / 3.0)
    pts = []
    for i in range(m):
        for j in range(m):
            for k in range(m):
                pts.append([i, j, k])
                pts.append([i + 0.5, j + 0.5, k + 0.5])
    return np.diag([m * a] * 3), a * np.array(pts, dtype=np.float64)


def hex_crystal(m, rs):
    """m x m supercell of the primitive triangular lattice: (lattice, positions (m^2, 2))."""
    prim = hex_lattice(1, rs)
    pts = [i * prim[0] + j * prim[1] for i in range(m) for j in range(m)]
    return m * prim, np.array(pts, dtype=np.float64)


def rocksalt_cell(a):
    """Conventional rocksalt cube of side a: (lattice, positions (8, 3), charges (8,))."""
    pos, q = [], []
    for i in range(2):
        for j in range(2):
            for k in range(2):
                pos.append([0.5 * a * i, 0.5 * a * j, 0.5 * a * k])
                q.append(1.0 if (i + j + k) % 2 == 0 else -1.0)
    return np.diag([a, a, a]), np.array(pos), np.array(q)


def diamond_ions(m, a):
    """Diamond structure in an m x m x m supercell of the conventional cube of side a."""
    fcc = [(0, 0, 0), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]
    basis = [(0, 0, 0), (0.25, 0.25, 0.25)]
    pts = []
    for i in range(m):
        for j in range(m):
            for k in range(m):
                for f in fcc:
                    for b in basis:
                        pts.append([i + f[0] + b[0], j + f[1] + b[1], k + f[2] + b[2]])
    return np.diag([m * a] * 3), a * np.array(pts, dtype=np.float64)


# --------------------------------------------------------------------------
# Positions and moves.
# --------------------------------------------------------------------------

def frac_to_cart(frac, lattice):
    """Cartesian positions from fractional coordinates (rows of lattice are a_i)."""
    return np.asarray(frac) @ np.asarray(lattice)


def uniform_positions(rng, lattice, n_walkers, n):
    """(W, N, dim) positions i.i.d. uniform in the cell."""
    dim = lattice.shape[0]
    return frac_to_cart(rng.random((n_walkers, n, dim)), lattice)


def scattered_positions(rng, centres, n_walkers, n, sigma):
    """(W, N, 3) positions: each at a uniformly chosen centre plus N(0, sigma^2) per axis."""
    idx = rng.integers(0, centres.shape[0], size=(n_walkers, n))
    return centres[idx] + sigma * rng.standard_normal((n_walkers, n, centres.shape[1]))


def move_stream(rng, n_walkers, n, n_moves, dim, sigma, accept_prob=0.5):
    """Random single-particle moves: (k (M, W) int32, disp (M, W, dim), accept (M, W) uint8).

    The moved particle is uniform in [0, n); the displacement is Gaussian with
    standard deviation sigma per axis; a move is accepted when a uniform
    number falls below accept_prob (there is no wave function to decide it).
    """
    k = rng.integers(0, n, size=(n_moves, n_walkers)).astype(np.int32)
    disp = sigma * rng.standard_normal((n_moves, n_walkers, dim))
    acc = (rng.random((n_moves, n_walkers)) < accept_prob).astype(np.uint8)
    return k, disp, acc


# --------------------------------------------------------------------------
# Named workloads.
# --------------------------------------------------------------------------

def workload(name, n_walkers=None):
    """Return a dict describing a named synthetic workload.

    Keys: dim, lattice, n, q (mobile charges), fixed_pos, fixed_q, alpha,
    n_walkers, pos (W, N, dim), tag, moves (n per walker), sigma; layered 2D
    workloads add z (N,), each mobile particle's height above the plane.

    alpha values other than the sc cell's are chosen so that the number of
    reciprocal vectors inside the 1e-16 cutoff is about 4000 (3D) or about
    1000 (2D), which puts real- and reciprocal-space work near balance.
    """
    if name == "heg3d_sc_n54":            # 3D gas, N=54, r_s=1, sc cell, alpha = 2.8/L
        tag, n, rs = 0, 54, 1.0
        lat = sc_lattice(n, rs)
        W = n_walkers or 16
        alpha = 2.8 / lat[0, 0]
        d = dict(dim=3, lattice=lat, n=n, alpha=alpha, moves=100, sigma=0.3)
        pos = uniform_positions(rng_for(tag), lat, W, n)
        q = -np.ones(n)
        fpos, fq = np.zeros((0, 3)), np.zeros(0)
    elif name == "heg3d_fcc_n1024":       # 3D gas, N=1024, r_s=2, fcc cell, ~4000 G vectors
        tag, n, rs = 1, 1024, 2.0
        lat = fcc_lattice(n, rs)
        W = n_walkers or 4096
        d = dict(dim=3, lattice=lat, n=n, alpha=0.15685, moves=1000, sigma=0.3)
        pos = uniform_positions(rng_for(tag), lat, W, n)
        q = -np.ones(n)
        fpos, fq = np.zeros((0, 3)), np.zeros(0)
    elif name == "heg2d_hex_n338":        # 2D gas, N=338, r_s=5, hexagonal cell, ~1000 G vectors
        tag, n, rs = 2, 338, 5.0
        lat = hex_lattice(n, rs)
        W = n_walkers or 2048
        d = dict(dim=2, lattice=lat, n=n, alpha=0.05858, moves=100, sigma=1.5)
        pos = uniform_positions(rng_for(tag), lat, W, n)
        q = -np.ones(n)
        fpos, fq = np.zeros((0, 2)), np.zeros(0)
    elif name == "diamond_3x3x3":         # 216 ions (+4) and 864 electrons, a = 6.74 bohr
        tag, n = 3, 864
        lat, fpos = diamond_ions(3, 6.74)
        fq = 4.0 * np.ones(fpos.shape[0])
        W = n_walkers or 1024
        d = dict(dim=3, lattice=lat, n=n, alpha=0.25207, moves=100, sigma=0.3)
        pos = scattered_positions(rng_for(tag), fpos, W, n, 0.8)
        q = -np.ones(n)
    elif name == "ehbilayer2d_hex_n338":  # 2D electron-hole bilayer: 169 e (z = 0) + 169 h (z = 5), r_s = 5
        tag, n, rs, sep = 4, 338, 5.0, 5.0
        lat = hex_lattice(n // 2, rs)        # area 169 pi r_s^2: r_s = 5 in each layer
        W = n_walkers or 2048
        # about 1000 G vectors: N_G ~ g_c^2 A / (4 pi), g_c = 2 alpha erfc^-1(1e-16)
        d = dict(dim=2, lattice=lat, n=n, alpha=0.0839, moves=100, sigma=1.5)
        pos = uniform_positions(rng_for(tag), lat, W, n)
        q = np.where(np.arange(n) < n // 2, -1.0, 1.0)
        d["z"] = np.where(np.arange(n) < n // 2, 0.0, sep)
        fpos, fq = np.zeros((0, 2)), np.zeros(0)
    elif name.startswith("heg3d_sc_n"):   # serving-mix sizes: sc cells at r_s = 2
        n = int(name[len("heg3d_sc_n"):])
        tag, rs = 10 + n, 2.0
        lat = sc_lattice(n, rs)
        W = n_walkers or 64
        omega = abs(np.linalg.det(lat))
        # about 4000 G vectors: N_G ~ g_c^3 Omega / (6 pi^2), g_c = 12.1394 alpha
        alpha = (4000.0 * 6.0 * math.pi ** 2 / omega) ** (1.0 / 3.0) / 12.1394
        d = dict(dim=3, lattice=lat, n=n, alpha=alpha, moves=100, sigma=0.3)
        pos = uniform_positions(rng_for(tag), lat, W, n)
        q = -np.ones(n)
        fpos, fq = np.zeros((0, 3)), np.zeros(0)
    else:
        raise KeyError(name)
    d.update(name=name, tag=tag, n_walkers=W, pos=pos, q=q, fixed_pos=fpos, fixed_q=fq)
    return d
