"""Single-particle moves on the 3D electron gas at full size (fcc cell,
N = 1024, 4096 walkers), in the launch configuration the benchmark times,
against the FP64 CPU oracle (paper Sec. 2.1: VMC and DMC sampling is a
stream of one-particle moves, each needing the energy change).

* test_moves_match_oracle_full_size: every walker of the batch moves; the
  proposed dE of three sampled walkers (first, middle, last) is compared
  with the oracle's over 10 rounds, with accepted and rejected moves and one
  move that carries an electron across the cell boundary.
* test_rho_drift_over_1000_moves: 1000 rounds without a re-sum; rho(G) kept
  by accepted moves is compared with a rebuild, element by element with the
  oracle's rho(G) of the final positions, and through the reciprocal energy
  and the next move's dE.

Gates: the walker floor max(|E|, 1e-2 S) at 1e-12 (FP64) / 1e-6 (mixed), and
the move's own scale max(|dE|, 1e-2 (|dE_real| + |dE_recip|)) at the DE_TOL
of test_gpu_parity.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2507_02888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-6, "fp64_tiered": 1e-12}
DE_TOL = {"fp64": 1e-12, "mixed": 3e-4, "fp64_tiered": 2e-10}
SAMPLE = [0, 2047, 4095]


@pytest.fixture(scope="module")
def ew():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_02888_gb300 import ewald
    ewald.load()
    return ewald


@pytest.fixture(scope="module")
def fcc():
    return I.workload("heg3d_fcc_n1024")


def floor_of(comp):
    return 1e-2 * (abs(comp[0]) + abs(comp[2]) + abs(comp[1] + comp[3]) + abs(comp[4]))


def oracle_jobs(fn, jobs):
    # the oracle releases the GIL (ctypes): run the sampled evaluations side by side
    with ThreadPoolExecutor(8) as ex:
        return list(ex.map(lambda a: fn(*a), jobs))


@pytest.mark.parametrize("prec", ["mixed", "fp64", "fp64_tiered"])
def test_moves_match_oracle_full_size(ew, fcc, prec):
    w = fcc
    W, N, dim, lat = w["n_walkers"], w["n"], w["dim"], w["lattice"]
    M = 10
    ks, disp, acc = I.move_stream(np.random.default_rng(31), W, N, M, dim, w["sigma"])
    # round 3: walker 0's electron nearest the a_1 face is carried across it
    f = w["pos"][0] @ np.linalg.inv(lat)
    f -= np.floor(f)
    k0 = int(np.argmax(f[:, 0]))
    ks[3, 0] = k0
    disp[3, 0] = (1.0 - f[k0, 0] + 0.004) * lat[0]
    acc[3, 0] = 1
    for wi in SAMPLE:   # each sampled walker has accepted and rejected moves
        assert 0 < acc[:, wi].sum() < M
    ctx = ew.context_for(w, precision=prec)
    info = ctx.info()
    rc, gc = info["r_cutoff"], info["g_cutoff"]
    b = ew.Batch(ctx, W)
    b.set_positions(w["pos"])
    b.energy()
    pos = w["pos"].copy()
    jobs, got = [], []
    for m in range(M):
        r_new = pos[np.arange(W), ks[m]] + disp[m]
        de = b.propose(ks[m], r_new)
        assert np.all(np.isfinite(de))
        for wi in SAMPLE:
            jobs.append((pos[wi].copy(), int(ks[m, wi]), r_new[wi].copy()))
            got.append(de[wi])
        b.accept(acc[m])
        sel = acc[m].astype(bool)
        pos[np.arange(W)[sel], ks[m][sel]] = r_new[sel]
    q = w["q"]

    def one(p, k, rn):
        e0, c0 = oracle.energy(dim, lat, p, q, w["alpha"], rc, gc)
        d_real, d_recip = oracle.delta_e_parts(dim, lat, p, q, k, rn, w["alpha"], rc, gc)
        return e0, c0, d_real, d_recip

    out = oracle_jobs(one, jobs)
    worst_w = worst_de = 0.0
    for g, (e0, c0, d_real, d_recip) in zip(got, out):
        de_o = d_real + d_recip
        wf = max(abs(e0), floor_of(c0))
        ds = max(abs(de_o), 1e-2 * (abs(d_real) + abs(d_recip)))
        assert abs(g - de_o) <= TOL[prec] * wf, (g, de_o, wf)
        assert abs(g - de_o) <= DE_TOL[prec] * ds, (g, de_o, ds)
        worst_w, worst_de = max(worst_w, abs(g - de_o) / wf), max(worst_de, abs(g - de_o) / ds)
    print("fcc N=1024 moves, %s: dE error / walker floor %.3g, / dE scale %.3g" % (prec, worst_w, worst_de))
    # the crossing electron is stored wrapped into the cell, at the oracle's position up to a lattice vector
    got_pos = b.get_positions()
    fr = (got_pos[0, k0] - pos[0, k0]) @ np.linalg.inv(lat)
    assert np.max(np.abs(fr - np.round(fr))) < 1e-12 and abs(np.round(fr[0])) == 1
    # energies after the moves (re-summed rho) against the oracle
    e = b.energy()
    ens = oracle_jobs(lambda p: oracle.energy(dim, lat, p, q, w["alpha"], rc, gc), [(pos[wi],) for wi in SAMPLE])
    for wi, (e_o, c_o) in zip(SAMPLE, ens):
        assert abs(e[wi] - e_o) <= TOL[prec] * max(abs(e_o), floor_of(c_o)), (wi, e[wi], e_o)
    b.close()
    ctx.close()


def recip_from_rho(ctx, w, rho_w):
    """E_recip = (2 pi / Omega) sum over the half space of 2 f(G) |rho(G)|^2,
    f(G) = exp(-G^2/4 alpha^2) / G^2 (paper Eq. (3)), from a stored rho."""
    lat = np.asarray(w["lattice"])
    B = 2 * np.pi * np.linalg.inv(lat).T
    G = ctx.gvectors() @ B
    g2 = np.sum(G * G, axis=1)
    f = np.exp(-g2 / (4 * w["alpha"] ** 2)) / g2
    r2 = rho_w[0, :, 0] ** 2 + rho_w[0, :, 1] ** 2
    return 2 * np.pi / abs(np.linalg.det(lat)) * np.sum(2 * f * r2)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_rho_drift_over_1000_moves(ew, fcc, prec):
    """rho(G) under 1000 rounds of accepted-or-rejected moves with no re-sum:
    the running sum (FP64 in the FP64 path; the float pair hi + lo updated
    by two-sums in the mixed path) against a rebuild and against the oracle."""
    torch = pytest.importorskip("torch")
    w = fcc
    W, N, dim, lat, q = w["n_walkers"], w["n"], w["dim"], w["lattice"], w["q"]
    ctx = ew.context_for(w, precision=prec, resum_every=10 ** 9)
    info = ctx.info()
    rc, gc = info["r_cutoff"], info["g_cutoff"]
    b = ew.Batch(ctx, W)
    b.set_positions(w["pos"])
    b.energy()
    MM = 1000
    ks, disp, acc = I.move_stream(np.random.default_rng(99), W, N, MM, dim, w["sigma"])
    pos_d = torch.tensor(w["pos"], device="cuda")
    ar = torch.arange(W, device="cuda")
    k_d, d_d, a_d = (torch.tensor(x, device="cuda") for x in (ks, disp, acc))
    de_d = torch.empty(W, dtype=torch.float64, device="cuda")
    for m in range(MM):
        kk = k_d[m].long()
        rn = pos_d[ar, kk] + d_d[m]
        b.propose(k_d[m], rn, de_d)
        b.accept(a_d[m])
        sel = a_d[m].bool()
        pos_d[ar[sel], kk[sel]] = rn[sel]
    torch.cuda.synchronize()
    pos = pos_d.cpu().numpy()
    kn = np.full(W, 5, dtype=np.int32)
    rnn = pos[:, 5] + 0.3
    r_run = b.rho()
    de_run = b.propose(kn, rnn)          # from the running rho
    b.resum()
    r_new = b.rho()
    de_new = b.propose(kn, rnn)          # from the rebuilt rho
    rho_tol = 1e-12 if prec == "fp64" else 2e-5   # per unit sqrt(sum q^2), as for a rebuilt rho
    rq = np.sqrt(np.sum(q ** 2))
    assert np.max(np.abs(r_run - r_new)) <= rho_tol * rq
    nv = ctx.gvectors()

    def one(p, rn):
        e0, c0 = oracle.energy(dim, lat, p, q, w["alpha"], rc, gc)
        d_real, d_recip = oracle.delta_e_parts(dim, lat, p, q, 5, rn, w["alpha"], rc, gc)
        return oracle.rho_at(dim, lat, p, q, nv), e0, c0, d_real, d_recip

    out = oracle_jobs(one, [(pos[wi], rnn[wi]) for wi in SAMPLE])
    for wi, (ro, e0, c0, d_real, d_recip) in zip(SAMPLE, out):
        for r in (r_run, r_new):
            got = r[wi, 0, :, 0] + 1j * r[wi, 0, :, 1]
            assert np.max(np.abs(got - ro)) <= rho_tol * rq, (wi, np.max(np.abs(got - ro)))
        wf = max(abs(e0), floor_of(c0))
        # the reciprocal energy of the running rho against the oracle's piece
        assert abs(recip_from_rho(ctx, w, r_run[wi]) - c0[2]) <= TOL[prec] * wf
        de_o = d_real + d_recip
        ds = max(abs(de_o), 1e-2 * (abs(d_real) + abs(d_recip)))
        for de in (de_run, de_new):
            assert abs(de[wi] - de_o) <= TOL[prec] * wf, (wi, de[wi], de_o)
            assert abs(de[wi] - de_o) <= DE_TOL[prec] * ds, (wi, de[wi], de_o)
    b.close()
    ctx.close()
