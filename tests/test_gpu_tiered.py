"""Tiered FP64 form (EWALD_FP64_TIERED): FP64 results with the real-space
images above erfc(alpha r) = 1e-7 evaluated in FP64 from the exact geometry
and the rest in FP32.  Held to the FP64 bar, 1e-12 of max(|E|, 1e-2 S),
against the oracle at the FP64 cutoffs, on the same cases as the other
forms (ions, charges that FP32 cannot hold, clustered particles, 2D, layers)."""
import numpy as np
import pytest

import oracle
from paper_2507_02888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def ew():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_02888_gb300 import ewald
    ewald.load()
    return ewald


def scale(c):
    return abs(c[0]) + abs(c[2]) + abs(c[1] + c[3]) + abs(c[4])


def small(name, W=4):
    rng = np.random.default_rng(404)
    if name == "sc54":
        return I.workload("heg3d_sc_n54", W)
    if name == "fcc100_odd_q":
        # charges that are not FP32 numbers, Q != 0 (background)
        lat = I.fcc_lattice(100, 1.5)
        d = dict(dim=3, lattice=lat, n=100, alpha=6.0 / abs(np.linalg.det(lat)) ** (1 / 3))
        d["pos"] = I.uniform_positions(rng, lat, W, 100)
        d["q"] = -1.0 + 0.1 * (np.arange(100) % 7) / 3.0
        d["fixed_pos"], d["fixed_q"] = np.zeros((0, 3)), np.zeros(0)
    elif name == "diamond1":
        lat, ions = I.diamond_ions(1, 6.74)
        d = dict(dim=3, lattice=lat, n=32, alpha=0.9)
        d["pos"] = I.scattered_positions(rng, ions, W, 32, 0.8)
        d["q"] = -np.ones(32)
        d["fixed_pos"], d["fixed_q"] = ions, 4.0 * np.ones(len(ions))
    elif name == "hex70":
        lat = I.hex_lattice(70, 3.0)
        d = dict(dim=2, lattice=lat, n=70, alpha=5.0 / np.sqrt(abs(np.linalg.det(lat))))
        d["pos"] = I.uniform_positions(rng, lat, W, 70)
        d["q"] = -np.ones(70)
        d["fixed_pos"], d["fixed_q"] = np.zeros((0, 2)), np.zeros(0)
    elif name == "clustered":
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
    else:
        raise KeyError(name)
    d["n_walkers"] = W
    return d


@pytest.mark.parametrize("name", ["sc54", "fcc100_odd_q", "diamond1", "hex70", "clustered"])
def test_tiered_energy_matches_oracle(ew, name):
    w = small(name)
    ctx = ew.context_for(w, precision="fp64_tiered")
    info = ctx.info()
    assert info["precision"] == 2
    b = ew.Batch(ctx, w["n_walkers"])
    b.set_positions(w["pos"])
    comp = b.components()
    e = b.energy()
    for k in range(w["n_walkers"]):
        p = np.concatenate([w["pos"][k], w["fixed_pos"]])
        q = np.concatenate([w["q"], w["fixed_q"]])
        eo, co = oracle.energy(w["dim"], w["lattice"], p, q, w["alpha"], info["r_cutoff"], info["g_cutoff"])
        fl = max(abs(eo), 1e-2 * scale(co))
        assert abs(e[k] - eo) <= TOL * fl, (k, e[k], eo, (e[k] - eo) / fl)
        assert np.all(np.abs(comp[k] - co) <= TOL * np.maximum(np.abs(co), fl))


@pytest.mark.parametrize("name,sample", [("heg3d_fcc_n1024", [0, 4095]), ("diamond_3x3x3", [7]),
                                         ("heg2d_hex_n338", [1000])])
def test_tiered_full_size_sampled(ew, name, sample):
    w = I.workload(name)
    ctx = ew.context_for(w, precision="fp64_tiered")
    b = ew.Batch(ctx, w["n_walkers"])
    b.set_positions(w["pos"])
    e = b.energy()
    rc, gc = oracle.cutoffs(w["dim"], w["alpha"])
    for k in sample:
        p = np.concatenate([w["pos"][k], w["fixed_pos"]])
        q = np.concatenate([w["q"], w["fixed_q"]])
        eo, co = oracle.energy(w["dim"], w["lattice"], p, q, w["alpha"], rc, gc)
        assert abs(e[k] - eo) <= TOL * max(abs(eo), 1e-2 * scale(co)), (k, e[k], eo)


def test_tiered_equals_fp64_on_many_walkers(ew):
    w = I.workload("heg3d_fcc_n1024", 64)
    out = {}
    for prec in ("fp64", "fp64_tiered"):
        ctx = ew.context_for(w, precision=prec)
        b = ew.Batch(ctx, 64)
        b.set_positions(w["pos"])
        out[prec] = (b.energy().copy(), b.components().copy())
    e64, c64 = out["fp64"]
    floor = np.maximum(np.abs(e64), 1e-2 * (np.abs(c64[:, 0]) + np.abs(c64[:, 2]) + np.abs(c64[:, 1] + c64[:, 3])
                                           + np.abs(c64[:, 4])))
    assert np.max(np.abs(out["fp64_tiered"][0] - e64) / floor) <= TOL


def test_tiered_layered_bilayer(ew):
    rng = np.random.default_rng(12)
    lat = I.hex_lattice(30, 2.0)
    n = 60
    w = dict(dim=2, lattice=lat, n=n, n_walkers=2, alpha=4.5 / np.sqrt(abs(np.linalg.det(lat))))
    w["pos"] = I.uniform_positions(rng, lat, 2, n)
    w["q"] = np.where(np.arange(n) < 30, -1.0, 1.0)
    w["z"] = np.where(np.arange(n) < 30, 0.0, 2.3)          # 2.3 is not an FP32 number
    w["fixed_pos"], w["fixed_q"] = np.zeros((0, 2)), np.zeros(0)
    ctx = ew.context_for(w, precision="fp64_tiered")
    info = ctx.info()
    b = ew.Batch(ctx, 2)
    b.set_positions(w["pos"])
    e = b.energy()
    for k in range(2):
        eo, co = oracle.energy_z(lat, w["pos"][k], w["z"], w["q"], w["alpha"], info["r_cutoff"], info["g_cutoff"])
        assert abs(e[k] - eo) <= TOL * max(abs(eo), 1e-2 * scale(co))


def all_of(w, k, pos):
    return np.concatenate([pos, w["fixed_pos"]]), np.concatenate([w["q"], w["fixed_q"]])


@pytest.mark.parametrize("name", ["fcc100_odd_q", "clustered", "diamond1"])
def test_tiered_moves_match_oracle(ew, name):
    """Proposed dE of the tiered kernel (real space split like the energy's,
    reciprocal in FP64) against the oracle's, through accepted and rejected
    moves, and the energy at the end against a fresh oracle energy."""
    W = 3
    w = small(name, W)
    ctx = ew.context_for(w, precision="fp64_tiered", resum_every=4)
    info = ctx.info()
    rc, gc = info["r_cutoff"], info["g_cutoff"]
    b = ew.Batch(ctx, W)
    b.set_positions(w["pos"])
    pos = w["pos"].copy()
    floors = []
    for k in range(W):
        eo, co = oracle.energy(w["dim"], w["lattice"], *all_of(w, k, pos[k]), w["alpha"], rc, gc)
        floors.append(max(abs(eo), 1e-2 * scale(co)))
    rng = np.random.default_rng(31)
    ks, disp, acc = I.move_stream(rng, W, w["n"], 10, w["dim"], 0.3)
    for m in range(ks.shape[0]):
        rn = pos[np.arange(W), ks[m]] + disp[m]
        de = b.propose(ks[m], rn).copy()
        for k in range(W):
            deo = oracle.delta_e(w["dim"], w["lattice"], *all_of(w, k, pos[k]), int(ks[m, k]), rn[k], w["alpha"],
                                 rc, gc)
            assert abs(de[k] - deo) <= TOL * floors[k], (m, k, de[k], deo)
        b.accept(acc[m])
        for k in range(W):
            if acc[m, k]:
                pos[k, ks[m, k]] = rn[k]
    e = b.energy()
    for k in range(W):
        eo, co = oracle.energy(w["dim"], w["lattice"], *all_of(w, k, pos[k]), w["alpha"], rc, gc)
        assert abs(e[k] - eo) <= TOL * max(abs(eo), 1e-2 * scale(co))


def test_tiered_moves_full_size(ew):
    """The fcc workload's 4096 walkers: every proposed dE equal to the FP64
    kernel's within the FP64 bar, and two sampled walkers against the oracle."""
    w = I.workload("heg3d_fcc_n1024")
    W = w["n_walkers"]
    rng = np.random.default_rng(8)
    ks = rng.integers(0, w["n"], size=W)
    rn = w["pos"][np.arange(W), ks] + rng.normal(scale=0.4, size=(W, 3))
    out = {}
    for prec in ("fp64", "fp64_tiered"):
        ctx = ew.context_for(w, precision=prec)
        b = ew.Batch(ctx, W)
        b.set_positions(w["pos"])
        e = b.energy().copy()
        c = b.components().copy()
        out[prec] = b.propose(ks, rn).copy()
    floor = np.maximum(np.abs(e), 1e-2 * (np.abs(c[:, 0]) + np.abs(c[:, 2]) + np.abs(c[:, 1] + c[:, 3])
                                          + np.abs(c[:, 4])))
    assert np.max(np.abs(out["fp64_tiered"] - out["fp64"]) / floor) <= TOL
    rc, gc = oracle.cutoffs(3, w["alpha"])
    for k in (5, 4090):
        deo = oracle.delta_e(3, w["lattice"], *all_of(w, k, w["pos"][k]), int(ks[k]), rn[k], w["alpha"], rc, gc)
        assert abs(out["fp64_tiered"][k] - deo) <= TOL * floor[k], (k, out["fp64_tiered"][k], deo)
