"""Layered 2D cells on the GPU (paper Sec. 2.2, Eqs. (5)-(6) with charges at
heights z != 0) against the FP64 oracle's pair definition, through the C ABI:
energies and their pieces, rho(G) per layer, move energy changes, fixed
charges in their own layer, the batched and serving forms, and argument
checks.  Tolerances as in the in-plane tests: 1e-12 (FP64) and 1e-6
(mixed) of max(|E|, 1e-2 S)."""
import numpy as np
import pytest

import oracle
from paper_2507_02888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-6, "fp64_tiered": 1e-12}


@pytest.fixture(scope="module")
def ew():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_02888_gb300 import ewald
    ewald.load()
    return ewald


def scale(comp):
    return abs(comp[0]) + abs(comp[2]) + abs(comp[1] + comp[3]) + abs(comp[4])


def bilayer(n=60, W=3, sep=2.5, seed=21, fixed=False):
    """n/2 electrons at z = 0 and n/2 holes at z = sep; with fixed=True also
    12 fixed charges (+1/2 each) in a third layer at z = -3.5."""
    rng = np.random.default_rng(seed)
    lat = I.hex_lattice(n // 2, 2.0)
    d = dict(dim=2, lattice=lat, n=n, n_walkers=W, alpha=4.5 / np.sqrt(abs(np.linalg.det(lat))))
    d["pos"] = I.uniform_positions(rng, lat, W, n)
    d["q"] = np.where(np.arange(n) < n // 2, -1.0, 1.0)
    d["z"] = np.where(np.arange(n) < n // 2, 0.0, sep)
    if fixed:
        d["fixed_pos"] = rng.random((12, 2)) @ lat
        d["fixed_q"] = np.full(12, 0.5)
        d["fixed_z"] = np.full(12, -3.5)
    else:
        d["fixed_pos"], d["fixed_q"] = np.zeros((0, 2)), np.zeros(0)
    return d


def oracle_all(w, walker, rc, gc, pos=None):
    p = w["pos"][walker] if pos is None else pos
    pz = np.concatenate([p, w["fixed_pos"]])
    z = np.concatenate([w["z"], w.get("fixed_z", np.zeros(0))])
    q = np.concatenate([w["q"], w["fixed_q"]])
    return oracle.energy_z(w["lattice"], pz, z, q, w["alpha"], rc, gc)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("fixed", [False, True])
def test_energy_matches_oracle(ew, prec, fixed):
    w = bilayer(fixed=fixed)
    ctx = ew.context_for(w, precision=prec)
    info = ctx.info()
    assert info["n_layers"] == (3 if fixed else 2)
    b = ew.Batch(ctx, w["n_walkers"])
    b.set_positions(w["pos"])
    comp = b.components()
    e = b.energy()
    for k in range(w["n_walkers"]):
        eo, co = oracle_all(w, k, info["r_cutoff"], info["g_cutoff"])
        fl = max(abs(eo), 1e-2 * scale(co))
        assert abs(e[k] - eo) <= TOL[prec] * fl, (k, e[k], eo)
        # the same five pieces: real-space, Madelung, reciprocal, self, background
        assert np.max(np.abs(comp[k] - co)) <= 2 * TOL[prec] * scale(co), (comp[k], co)
    assert abs(info["e_background"] - co[4]) <= 1e-12 * abs(co[4])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_bilayer_sampled(ew, prec):
    w = I.workload("ehbilayer2d_hex_n338", 2048)
    ctx = ew.context_for(w, precision=prec)
    info = ctx.info()
    b = ew.Batch(ctx, w["n_walkers"])
    b.set_positions(w["pos"])
    e = b.energy()
    assert np.all(np.isfinite(e))
    for k in (0, 1777):
        eo, co = oracle.energy_z(w["lattice"], w["pos"][k], w["z"], w["q"], w["alpha"], info["r_cutoff"],
                                 info["g_cutoff"])
        assert abs(e[k] - eo) <= TOL[prec] * max(abs(eo), 1e-2 * scale(co)), (k, e[k], eo)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rho_per_layer(ew, prec):
    w = bilayer(fixed=True, W=2)
    ctx = ew.context_for(w, precision=prec)
    b = ew.Batch(ctx, 2)
    b.set_positions(w["pos"])
    rho = b.rho()
    nv = ctx.gvectors()
    assert rho.shape == (2, 3, len(nv), 2)
    tol = 1e-12 if prec == "fp64" else 2e-5
    zs = sorted(set(np.concatenate([w["z"], w["fixed_z"]])))
    for k in range(2):
        p = np.concatenate([w["pos"][k], w["fixed_pos"]])
        z = np.concatenate([w["z"], w["fixed_z"]])
        q = np.concatenate([w["q"], w["fixed_q"]])
        for L, h in enumerate(zs):
            sel = z == h
            ref = oracle.rho_at(2, w["lattice"], p[sel], q[sel], nv)
            got = rho[k, L, :, 0] + 1j * rho[k, L, :, 1]
            assert np.max(np.abs(got - ref)) <= tol * np.sqrt(np.sum(q[sel] ** 2))


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_tiered"])
def test_moves_match_oracle(ew, prec):
    w = bilayer(fixed=True, W=3, seed=5)
    ctx = ew.context_for(w, precision=prec)
    info = ctx.info()
    rc, gc = info["r_cutoff"], info["g_cutoff"]
    b = ew.Batch(ctx, 3)
    b.set_positions(w["pos"])
    e = b.energy().copy()
    rng = np.random.default_rng(9)
    pos = b.get_positions().copy()
    z_all = np.concatenate([w["z"], w["fixed_z"]])
    q_all = np.concatenate([w["q"], w["fixed_q"]])
    floors = []
    for k in range(3):
        eo, co = oracle_all(w, k, rc, gc, pos[k])
        floors.append(max(abs(eo), 1e-2 * scale(co)))
    for step in range(6):
        ks = rng.integers(0, w["n"], size=3)           # electrons and holes alike
        rn = pos[np.arange(3), ks] + rng.normal(scale=0.7, size=(3, 2))
        de = b.propose(ks, rn).copy()
        acc = np.array([1, step % 2, 1], dtype=np.uint8)
        for k in range(3):
            p_all = np.concatenate([pos[k], w["fixed_pos"]])
            deo = oracle.delta_e_z(w["lattice"], p_all, z_all, q_all, ks[k], rn[k], w["alpha"], rc, gc)
            assert abs(de[k] - deo) <= TOL[prec] * floors[k], (step, k, de[k], deo)
        b.accept(acc)
        for k in range(3):
            if acc[k]:
                pos[k, ks[k]] = rn[k]
                e[k] += de[k]
    # the running energies against a fresh oracle energy of the final positions
    for k in range(3):
        eo, co = oracle_all(w, k, rc, gc, pos[k])
        assert abs(e[k] - eo) <= 4 * TOL[prec] * floors[k]
    # and rho kept by the moves equals rho rebuilt from the positions
    r1 = b.rho().copy()
    b.resum()
    assert np.max(np.abs(r1 - b.rho())) <= (2e-5 if prec == "mixed" else 1e-12) * np.sqrt(w["n"])


def test_one_height_is_the_plane(ew):
    w = bilayer(W=2)
    plain = dict(w)
    del plain["z"]
    for h in (0.0, 2.75):
        ctx = ew.context_for(w, precision="fp64", mobile_z=np.full(w["n"], h))
        assert ctx.info()["n_layers"] == 1
        b = ew.Batch(ctx, 2)
        b.set_positions(w["pos"])
        b0 = ew.Batch(ew.context_for(plain, precision="fp64"), 2)
        b0.set_positions(w["pos"])
        assert np.array_equal(b.energy(), b0.energy())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_multi_and_serving_with_a_layered_system(ew, prec):
    from paper_2507_02888_gb300 import serve
    wl = bilayer(W=3, seed=2)
    wp = I.workload("heg3d_sc_n54", 4)
    cl, cp = ew.context_for(wl, precision=prec), ew.context_for(wp, precision=prec)
    bl, bp = ew.Batch(cl, 3), ew.Batch(cp, 4)
    bl.set_positions(wl["pos"])
    bp.set_positions(wp["pos"])
    cm = np.concatenate([bl.components(), bp.components()])
    alone = cm.sum(axis=1)
    floor = np.maximum(np.abs(alone), 1e-2 * np.abs(cm).sum(axis=1))
    e = ew.Multi([bl, bp]).energy()
    # same terms, partial sums added in the persistent kernel's order
    assert np.all(np.abs(e - alone) <= (1e-13 if prec == "fp64" else 1e-6) * floor)
    # serving: a layered request alone and next to another request
    res = []
    for mix in (False, True):
        srv = serve.Server(prec, max_walkers=16)
        ids = [srv.submit(cl, wl["pos"], 15, 0.8, 0.5, seed=77)]
        if mix:
            ids.append(srv.submit(cp, wp["pos"], 9, 0.3, 0.5, seed=5))
        out = {}
        for _ in range(200):
            srv.step()
            for r in ids:
                if r not in out and srv.result(r) is not None:
                    out[r] = srv.result(r)
            if len(out) == len(ids):
                break
        res.append(out[ids[0]])
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert np.all(np.isfinite(res[0][0]))


def test_argument_checks(ew):
    w = bilayer(W=1)
    with pytest.raises(ew.EwaldError) as ei:
        ew.Context(3, np.eye(3) * 5.0, -np.ones(4), mobile_z=np.zeros(4))
    assert ei.value.code == 1
    with pytest.raises(ew.EwaldError):
        ew.context_for(w, mobile_z=np.arange(w["n"]) % 5 * 1.0)      # five heights
    with pytest.raises(ew.EwaldError):
        zz = w["z"].copy()
        zz[3] = np.nan
        ew.context_for(w, mobile_z=zz)
    with pytest.raises(ew.EwaldError):
        ew.context_for(w, mobile_z=w["z"] * 1e5)                    # |dz| g_c beyond 600


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_tiered"])
def test_served_layered_moves_match_oracle(ew, prec):
    """The serving kernel's device-drawn moves on a bilayer, replayed on the
    host (SplitMix64 + Box-Muller, as in the in-plane serving test) with the
    oracle's pair-definition dE."""
    import math
    from paper_2507_02888_gb300 import serve
    mask = (1 << 64) - 1

    def splitmix_out(seed, c):
        z = (seed + 0x9E3779B97F4A7C15 * (c + 1)) & mask
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
        return z ^ (z >> 31)

    def u53(x):
        return (x >> 11) * 2.0 ** -53

    w = bilayer(n=40, W=3, sep=1.7, seed=31)
    sigma, steps, seed, accept_p = 0.9, 10, 777, 0.5
    ctx = ew.context_for(w, precision=prec)
    info = ctx.info()
    rc, gc = info["r_cutoff"], info["g_cutoff"]
    srv = serve.Server(prec, max_walkers=8)
    rid = srv.submit(ctx, w["pos"], steps, sigma, accept_p, seed)
    res = None
    for _ in range(200):
        srv.step()
        res = srv.result(rid)
        if res is not None:
            break
    e_gpu, n_gpu, _ = res
    lat = np.asarray(w["lattice"])
    inv = np.linalg.inv(lat)
    n = w["n"]
    for walker in range(3):
        frac = (w["pos"][walker] @ inv) % 1.0
        e0, c0 = oracle.energy_z(lat, frac @ lat, w["z"], w["q"], w["alpha"], rc, gc)
        floor = max(abs(e0), 1e-2 * scale(c0))
        e, n_acc = e0, 0
        for step in range(steps):
            c = ((step << 32) + walker) * 8
            k = ((splitmix_out(seed, c) >> 32) * n) >> 32
            g = []
            for p in range(2):
                u1, u2 = u53(splitmix_out(seed, c + 1 + 2 * p)), u53(splitmix_out(seed, c + 2 + 2 * p))
                rad = math.sqrt(-2.0 * math.log(1.0 - u1))
                g += [rad * math.cos(2 * math.pi * u2), rad * math.sin(2 * math.pi * u2)]
            acc = u53(splitmix_out(seed, c + 5)) < accept_p
            pos = frac @ lat
            r_new = pos[k] + sigma * np.array(g[:2])
            de = oracle.delta_e_z(lat, pos, w["z"], w["q"], k, r_new, w["alpha"], rc, gc)
            if acc:
                e += de
                n_acc += 1
                frac[k] = (r_new @ inv) % 1.0
        assert n_gpu[walker] == n_acc
        assert abs(e_gpu[walker] - e) <= 2 * TOL[prec] * floor, (walker, e_gpu[walker], e)
