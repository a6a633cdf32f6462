"""Serving form: continuous batching of walker batches of different systems.

Checks that a request's results are bitwise the same alone and mixed with
other requests (arriving before and during it), that the device-side move
stream (counter-based SplitMix64, Box-Muller) replayed here on the host
with the FP64 oracle gives the same energies, and that admission respects
the walker budget.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2507_02888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-6, "fp64_tiered": 1e-12}
MASK = (1 << 64) - 1


@pytest.fixture(scope="module")
def mods():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_02888_gb300 import ewald, serve
    ewald.load()
    return ewald, serve


def splitmix_out(seed, c):
    """Output c (0-based) of a SplitMix64 stream seeded with `seed` (Steele, Lea & Flood 2014)."""
    z = (seed + 0x9E3779B97F4A7C15 * (c + 1)) & MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def u53(x):
    return (x >> 11) * 2.0 ** -53


def replay_move(seed, step, walker, n, dim, sigma, accept_p):
    c0 = ((step << 32) + walker) * 8
    k = ((splitmix_out(seed, c0) >> 32) * n) >> 32
    g = []
    for p in range(2):
        u1 = u53(splitmix_out(seed, c0 + 1 + 2 * p))
        u2 = u53(splitmix_out(seed, c0 + 2 + 2 * p))
        rad = math.sqrt(-2.0 * math.log(1.0 - u1))
        g += [rad * math.cos(2 * math.pi * u2), rad * math.sin(2 * math.pi * u2)]
    acc = u53(splitmix_out(seed, c0 + 5)) < accept_p
    return int(k), sigma * np.array(g[:dim]), acc


def small_hex(W, seed=5):
    rng = np.random.default_rng(seed)
    lat = I.hex_lattice(60, 3.0)
    return dict(dim=2, lattice=lat, n=60, alpha=5.0 / math.sqrt(abs(np.linalg.det(lat))), n_walkers=W,
                pos=I.uniform_positions(rng, lat, W, 60), q=-np.ones(60), fixed_pos=np.zeros((0, 2)),
                fixed_q=np.zeros(0))


def run_until_done(srv, ids, extra=None, limit=20000):
    out = {}
    for it in range(limit):
        if extra and it in extra:
            for fn in extra[it]:
                ids.append(fn())
        srv.step()
        for rid in ids:
            if rid not in out:
                r = srv.result(rid)
                if r is not None:
                    out[rid] = r
        if len(out) == len(ids) and not (extra and any(k > it for k in extra)):
            return out
    raise AssertionError("requests did not finish")


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_tiered"])
def test_request_alone_equals_in_mix(mods, prec):
    ewald, serve = mods
    wa = I.workload("heg3d_sc_n54", 6)
    wb = small_hex(5)
    wc = I.workload("heg3d_sc_n128", 3)
    ca, cb, cc = (ewald.context_for(w, precision=prec) for w in (wa, wb, wc))
    alone = serve.Server(prec, max_walkers=64)
    ra = alone.submit(ca, wa["pos"], 25, 0.3, 0.5, seed=11)
    res_alone = run_until_done(alone, [ra])[ra]
    mixed = serve.Server(prec, max_walkers=64)
    ids = [mixed.submit(cb, wb["pos"], 40, 1.0, 0.5, seed=7), mixed.submit(cc, wc["pos"], 10, 0.3, 0.5, seed=3)]
    holder = {}

    def submit_a():
        holder["a"] = mixed.submit(ca, wa["pos"], 25, 0.3, 0.5, seed=11)
        return holder["a"]

    def submit_d():
        return mixed.submit(cc, wc["pos"][:2], 30, 0.3, 0.5, seed=99)

    res = run_until_done(mixed, ids, extra={3: [submit_a], 9: [submit_d]})
    e_mix, n_mix, _ = res[holder["a"]]
    assert np.array_equal(e_mix, res_alone[0])
    assert np.array_equal(n_mix, res_alone[1])
    assert 0 < n_mix.sum() < 25 * 6


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_tiered"])
@pytest.mark.parametrize("case", ["sc54", "hex60"])
def test_served_moves_match_oracle(mods, case, prec):
    ewald, serve = mods
    w = I.workload("heg3d_sc_n54", 3) if case == "sc54" else small_hex(3, seed=8)
    sigma, steps, seed, accept_p = (0.4 if case == "sc54" else 1.2), 12, 2024, 0.5
    ctx = ewald.context_for(w, precision=prec)
    info = ctx.info()
    rc, gc = info["r_cutoff"], info["g_cutoff"]
    srv = serve.Server(prec, max_walkers=16)
    rid = srv.submit(ctx, w["pos"], steps, sigma, accept_p, seed)
    e_gpu, n_gpu, lat = run_until_done(srv, [rid])[rid]
    assert lat > 0
    lat_m = np.asarray(w["lattice"])
    inv = np.linalg.inv(lat_m)
    dim, n = w["dim"], w["n"]
    for walker in range(w["n_walkers"]):
        frac = (w["pos"][walker] @ inv) % 1.0          # positions as stored: wrapped
        e0, c0 = oracle.energy(dim, lat_m, frac @ lat_m, w["q"], w["alpha"], rc, gc)
        floor = max(abs(e0), 1e-2 * (abs(c0[0]) + abs(c0[2]) + abs(c0[1] + c0[3]) + abs(c0[4])))
        e, n_acc = e0, 0
        for step in range(steps):
            k, disp, acc = replay_move(seed, step, walker, n, dim, sigma, accept_p)
            pos = frac @ lat_m
            r_new = pos[k] + disp
            de = oracle.delta_e(dim, lat_m, pos, w["q"], k, r_new, w["alpha"], rc, gc)
            if acc:
                e += de
                n_acc += 1
                frac[k] = (r_new @ inv) % 1.0
        e_final, _ = oracle.energy(dim, lat_m, frac @ lat_m, w["q"], w["alpha"], rc, gc)
        assert n_gpu[walker] == n_acc
        assert abs(e_gpu[walker] - e) <= 2 * TOL[prec] * floor, (walker, e_gpu[walker], e)
        assert abs(e - e_final) <= 1e-10 * floor             # the oracle's own bookkeeping


def test_server_precision_must_match_context(mods):
    """A tiered server takes tiered contexts only; an FP64 server takes FP64
    and tiered ones (moving them with the plain FP64 kernel)."""
    ewald, serve = mods
    w = I.workload("heg3d_sc_n54", 2)
    c64 = ewald.context_for(w, precision="fp64")
    ct = ewald.context_for(w, precision="fp64_tiered")
    cm = ewald.context_for(w, precision="mixed")
    tiered = serve.Server("fp64_tiered", max_walkers=8)
    for c in (c64, cm):
        with pytest.raises(ewald.EwaldError) as ei:
            tiered.submit(c, w["pos"], 2, 0.3, 0.5, seed=1)
        assert ei.value.code == 1
    r = tiered.submit(ct, w["pos"], 4, 0.3, 0.5, seed=1)
    e_t, n_t, _ = run_until_done(tiered, [r])[r]
    plain = serve.Server("fp64", max_walkers=8)
    r = plain.submit(ct, w["pos"], 4, 0.3, 0.5, seed=1)
    e_p, n_p, _ = run_until_done(plain, [r])[r]
    assert np.array_equal(n_t, n_p)
    assert np.max(np.abs(e_t - e_p)) <= 1e-12 * np.max(np.abs(e_p))


def test_admission_respects_walker_budget(mods):
    ewald, serve = mods
    w = I.workload("heg3d_sc_n54", 6)
    ctx = ewald.context_for(w, precision="mixed")
    srv = serve.Server("mixed", max_walkers=8)
    ids = [srv.submit(ctx, w["pos"], 5, 0.3, 0.5, seed=s) for s in range(3)]
    seen_active = []
    out = {}
    for _ in range(1000):
        a, q = srv.step()
        seen_active.append(a)
        for rid in ids:
            if rid not in out and srv.result(rid) is not None:
                out[rid] = True
        if len(out) == 3:
            break
    assert len(out) == 3
    assert max(seen_active) == 1                            # 6 + 6 > 8 walkers: one at a time
    # every finished request is reported by completed() exactly once
    got = []
    for _ in range(100):
        srv.step()
        got += srv.completed()
        if len(got) >= 3:
            break
    assert sorted(got) == sorted(ids)
    srv.step()
    assert srv.completed() == []


def test_admission_respects_memory_budget(mods):
    """A device-memory budget that holds one request at a time: the requests
    queue and run one after another, with the results of an unconstrained
    server (bit for bit: a walker's result does not depend on the mix)."""
    ewald, serve = mods
    w = I.workload("heg3d_sc_n54", 6)
    ctx = ewald.context_for(w, precision="mixed")
    need = serve.request_bytes(ctx, 6)
    assert need > 6 * 54 * 3 * 8                             # at least the positions
    free = serve.Server("mixed", max_walkers=64)
    ids_f = [free.submit(ctx, w["pos"], 6, 0.3, 0.5, seed=40 + s) for s in range(3)]
    res_f = run_until_done(free, ids_f)
    tight = serve.Server("mixed", max_walkers=64, hbm_budget_bytes=1.5 * need)
    ids_t = [tight.submit(ctx, w["pos"], 6, 0.3, 0.5, seed=40 + s) for s in range(3)]
    seen = []
    out = {}
    for _ in range(2000):
        a, q = tight.step()
        seen.append((a, q))
        for rid in ids_t:
            if rid not in out:
                r = tight.result(rid)
                if r is not None:
                    out[rid] = r
        if len(out) == 3:
            break
    assert len(out) == 3
    assert max(a for a, _ in seen) == 1 and max(q for _, q in seen) == 2   # one at a time, two waiting
    for rf, rt in zip(ids_f, ids_t):
        assert np.array_equal(res_f[rf][0], out[rt][0]) and np.array_equal(res_f[rf][1], out[rt][1])


def test_request_over_budget_is_refused(mods):
    ewald, serve = mods
    w = I.workload("heg3d_sc_n54", 6)
    ctx = ewald.context_for(w, precision="mixed")
    need = serve.request_bytes(ctx, 6)
    srv = serve.Server("mixed", max_walkers=64, hbm_budget_bytes=need - 1)
    with pytest.raises(ewald.EwaldError) as ei:
        srv.submit(ctx, w["pos"], 3, 0.3, 0.5, seed=1)
    assert ei.value.code == 5                                # EWALD_ERR_OOM, nothing queued
    assert srv.step() == (0, 0)
    rid = srv.submit(ctx, w["pos"][:5], 3, 0.3, 0.5, seed=1)  # a smaller request fits
    e, n, _ = run_until_done(srv, [rid])[rid]
    assert np.all(np.isfinite(e))


def test_cancel_queued_and_active_requests(mods):
    """Host-side cancellation: an active and a queued request are cancelled;
    the others finish with the results they have alone, the cancelled ones
    are reported once and answer EWALD_ERR_CANCELLED."""
    ewald, serve = mods
    w = I.workload("heg3d_sc_n54", 6)
    ctx = ewald.context_for(w, precision="mixed")
    alone = serve.Server("mixed", max_walkers=64)
    ra = alone.submit(ctx, w["pos"][:4], 20, 0.3, 0.5, seed=77)
    ref = run_until_done(alone, [ra])[ra]
    srv = serve.Server("mixed", max_walkers=10)
    keep = srv.submit(ctx, w["pos"][:4], 20, 0.3, 0.5, seed=77)
    active = srv.submit(ctx, w["pos"], 50, 0.3, 0.5, seed=5)   # 4 + 6 walkers: both admitted
    queued = srv.submit(ctx, w["pos"], 50, 0.3, 0.5, seed=6)   # waits for slots
    for _ in range(3):
        a, q = srv.step()
    assert (a, q) == (2, 1)
    srv.cancel(active)
    srv.cancel(queued)
    with pytest.raises(ewald.EwaldError) as ei:
        srv.cancel(queued)
    assert ei.value.code == 8                                # already cancelled
    done, out = [], None
    for _ in range(200):
        srv.step()
        done += srv.completed()
        r = srv.result(keep)
        if r is not None:
            out = r
        if out is not None and len(done) == 3:
            break
    assert sorted(done) == sorted([keep, active, queued])
    assert np.array_equal(out[0], ref[0]) and np.array_equal(out[1], ref[1])
    for rid in (active, queued):
        with pytest.raises(ewald.EwaldError) as ei:
            srv.result(rid)
        assert ei.value.code == 9
    with pytest.raises(ewald.EwaldError) as ei:
        srv.cancel(keep)                                     # finished
    assert ei.value.code == 8
    srv.step()
    assert srv.completed() == []
