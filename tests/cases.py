"""Small seeded systems shared by the GPU parity tests and the host-only
set-up tests: sizes the oracle finishes in seconds, spanning 3D and 2D
cells, fixed ions, a single particle, unequal charges and clustered
particles."""
import numpy as np

from paper_2507_02888_gb300 import inputs as I


def small_case(name, W):
    rng = np.random.default_rng(1234)
    if name == "sc54":
        return I.workload("heg3d_sc_n54", W)
    if name == "fcc100":
        lat = I.fcc_lattice(100, 1.5)
        d = dict(dim=3, lattice=lat, n=100, alpha=6.0 / abs(np.linalg.det(lat)) ** (1 / 3))
        d["pos"] = I.uniform_positions(rng, lat, W, 100)
        d["q"] = -np.ones(100)
        d["fixed_pos"], d["fixed_q"] = np.zeros((0, 3)), np.zeros(0)
    elif name == "hex70":
        lat = I.hex_lattice(70, 3.0)
        d = dict(dim=2, lattice=lat, n=70, alpha=5.0 / np.sqrt(abs(np.linalg.det(lat))))
        d["pos"] = I.uniform_positions(rng, lat, W, 70)
        d["q"] = -np.ones(70)
        d["fixed_pos"], d["fixed_q"] = np.zeros((0, 2)), np.zeros(0)
    elif name == "diamond1":
        lat, ions = I.diamond_ions(1, 6.74)
        d = dict(dim=3, lattice=lat, n=32, alpha=0.9)
        d["pos"] = I.scattered_positions(rng, ions, W, 32, 0.8)
        d["q"] = -np.ones(32)
        d["fixed_pos"], d["fixed_q"] = ions, 4.0 * np.ones(len(ions))
    elif name == "single":
        lat = I.fcc_lattice(1, 2.0)
        d = dict(dim=3, lattice=lat, n=1, alpha=2.0)
        d["pos"] = I.uniform_positions(rng, lat, W, 1)
        d["q"] = np.array([-1.0])
        d["fixed_pos"], d["fixed_q"] = np.zeros((0, 3)), np.zeros(0)
    elif name == "clustered":
        # half the electrons in a ball of radius 0.25 of the mean spacing:
        # hundreds of close pairs per 32 x 32 sub-tile, more than the FP32
        # path's deferred close-pair list holds, so its rescan runs
        lat = I.sc_lattice(80, 1.5)
        spacing = abs(np.linalg.det(lat)) ** (1 / 3) / 80 ** (1 / 3)
        d = dict(dim=3, lattice=lat, n=80, alpha=5.0 / lat[0, 0])
        pos = I.uniform_positions(rng, lat, W, 80)
        for k in range(W):
            v = rng.normal(size=(40, 3))
            v *= (0.25 * spacing * rng.random((40, 1)) ** (1 / 3)) / np.linalg.norm(v, axis=1, keepdims=True)
            pos[k, :40] = pos[k, 0] + v
        d["pos"] = pos
        d["q"] = -np.ones(80)
        d["fixed_pos"], d["fixed_q"] = np.zeros((0, 3)), np.zeros(0)
    elif name == "mixed_q":
        lat = I.sc_lattice(40, 1.2)
        d = dict(dim=3, lattice=lat, n=40, alpha=5.0 / lat[0, 0])
        d["pos"] = I.uniform_positions(rng, lat, W, 40)
        d["q"] = np.where(np.arange(40) % 4 == 0, 3.0, -1.0)
        d["fixed_pos"], d["fixed_q"] = np.zeros((0, 3)), np.zeros(0)
    else:
        raise KeyError(name)
    d["n_walkers"] = W
    return d
