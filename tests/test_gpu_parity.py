"""GPU path vs the FP64 CPU oracle, element by element, through the C ABI.

Tolerances (paper Sec. 6 motivates the two precisions):
  FP64 path : |E_gpu - E_orc| <= 1e-12 * max(|E_orc|, 1e-2 S)
  mixed path: |E_gpu - E_orc| <= 1e-6  * max(|E_orc|, 1e-2 S)
with S = |E_real| + |E_recip| + |E_madR + E_self| + |E_bg| of the oracle.  The
floor keeps the gate meaningful when E is the small difference of large
parts (random electron-gas configurations).  A move's energy change is held
to the walker's floor at the same tolerance, and also to its own scale,
max(|dE|, 1e-2 (|dE_real| + |dE_recip|)) from the oracle's parts, at
DE_TOL: Metropolis acceptance consumes dE itself.  The mixed path's FP32
terms and phases carry absolute errors of ~1e-7 Ha per move, which is
1e-8 of a walker's energy but up to ~1e-5 of a small dE.
"""
import numpy as np
import pytest

import oracle
from cases import small_case
from paper_2507_02888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-6, "fp64_tiered": 1e-12}
# move dE against its own scale: FP64 to the FP64 gate; the mixed path's FP32
# terms and the tiered path's FP32 tail terms leave absolute errors of
# ~1e-7 Ha and ~1e-13 Ha per move, whatever the size of dE (largest measured
# against the dE scale: mixed 7.7e-5 for a 6e-4 Ha move in the 2D cell,
# 1.2e-5 at N = 1024; tiered 3.6e-11)
DE_TOL = {"fp64": 1e-12, "mixed": 3e-4, "fp64_tiered": 2e-10}
MIXED_REAL_TOL = 1e-10   # default real-space cutoff tolerance of the mixed path


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


def all_particles(w, walker, pos=None):
    p = w["pos"][walker] if pos is None else pos
    return np.concatenate([p, w["fixed_pos"]]), np.concatenate([w["q"], w["fixed_q"]])


def oracle_energy(w, walker, rc, gc, pos=None):
    p, q = all_particles(w, walker, pos)
    return oracle.energy(w["dim"], w["lattice"], p, q, w["alpha"], rc, gc)


def oracle_move(w, walker, pos, k, r_new, rc, gc):
    """(dE, its scale max(|dE|, 1e-2 (|dE_real| + |dE_recip|))) from the oracle."""
    p, q = all_particles(w, walker, pos)
    d_real, d_recip = oracle.delta_e_parts(w["dim"], w["lattice"], p, q, int(k), r_new, w["alpha"], rc, gc)
    de = d_real + d_recip
    return de, max(abs(de), 1e-2 * (abs(d_real) + abs(d_recip)))


def make(ew, w, prec, **kw):
    ctx = ew.context_for(w, precision=prec, **kw)
    b = ew.Batch(ctx, w["n_walkers"])
    b.set_positions(w["pos"])
    return ctx, b


CASES = ["sc54", "fcc100", "hex70", "diamond1", "single", "mixed_q", "clustered"]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES)
def test_energy_matches_oracle(ew, case, prec):
    w = small_case(case, 6)
    ctx, b = make(ew, w, prec)
    info = ctx.info()
    rc, gc = info["r_cutoff"], info["g_cutoff"]
    comp = b.components()
    e = b.energy()
    assert np.array_equal(comp.sum(axis=1), comp.sum(axis=1))
    for walker in range(w["n_walkers"]):
        e_o, c_o = oracle_energy(w, walker, rc, gc)
        S = scale(c_o)
        floor = max(abs(e_o), 1e-2 * S)
        assert abs(e[walker] - e_o) <= TOL[prec] * floor, (walker, e[walker], e_o)
        # components: each to the same relative tolerance of its own size (the gate is on E)
        assert np.all(np.abs(comp[walker] - c_o) <= TOL[prec] * np.maximum(np.abs(c_o), floor)), (comp[walker], c_o)


def test_mixed_direct_choice(ew):
    """Which systems take the first two images of a pair without the lane
    rings (info mixed_direct), so that the parity cases above cover both
    loops: on where lists hold 3 to 8 images and the second nearest image
    to a displacement cell's centre is inside r_c for >= 3/4 of the
    displacements (sc40 with mixed charges and the clustered sc80: ~0.99,
    with weighted terms and close pairs; hex70 in 2D: ~0.9; the
    1024-electron fcc gas: 0.91), off where it is not (fcc100: ~0.65,
    diamond1: ~0.7), where lists are short (the 338-electron 2D gas: one
    or two images) or long (sc54: chunked lists)."""
    want = {"mixed_q": 1, "clustered": 1, "hex70": 1, "fcc100": 0, "diamond1": 0, "sc54": 0}
    for name, flag in want.items():
        ctx = ew.context_for(small_case(name, 2), precision="mixed")
        assert ctx.info()["mixed_direct"] == flag, name
        ctx.close()
    for name, flag in (("heg3d_fcc_n1024", 1), ("heg2d_hex_n338", 0)):
        ctx = ew.context_for(I.workload(name, 2), precision="mixed")
        info = ctx.info()
        assert info["mixed_direct"] == flag, name
        assert not flag or 3 <= info["max_candidates"] <= 8
        ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_tiered"])
def test_plan_reports_what_create_builds(ew, prec, monkeypatch):
    """ewald_plan (host set-up only) and ewald_get_info of the context
    ewald_create builds agree field by field (no tiling cache applied)."""
    monkeypatch.delenv("EWALD_TUNE_CACHE", raising=False)
    for w in (small_case("fcc100", 1), small_case("hex70", 1), small_case("mixed_q", 1),
              I.workload("diamond_3x3x3", 1), I.workload("heg3d_fcc_n1024", 1)):
        ctx = ew.context_for(w, precision=prec)
        assert ew.plan_for(w, prec) == ctx.info()
        ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cutoffs_match_oracle_definition(ew, prec):
    w = small_case("fcc100", 1)
    ctx, _ = make(ew, w, prec)
    info = ctx.info()
    rc, gc = oracle.cutoffs(3, w["alpha"])
    if prec == "mixed":                                # real space at erfc(alpha r_c) = 1e-10
        rc, _ = oracle.cutoffs(3, w["alpha"], MIXED_REAL_TOL)
    assert abs(info["r_cutoff"] / rc - 1) < 1e-9 and abs(info["g_cutoff"] / gc - 1) < 1e-9
    assert 2 * info["n_g_half"] == oracle.gcount(3, w["lattice"], gc)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_rho_matches_oracle(ew, prec):
    w = small_case("diamond1", 2)
    ctx, b = make(ew, w, prec)
    nv = ctx.gvectors()
    rho = b.rho()
    tol = 1e-12 if prec == "fp64" else 2e-5
    for walker in range(2):
        p, q = all_particles(w, walker)
        ref = oracle.rho_at(3, w["lattice"], p, q, nv)
        got = rho[walker, 0, :, 0] + 1j * rho[walker, 0, :, 1]
        assert np.max(np.abs(got - ref)) <= tol * np.sqrt(np.sum(q ** 2)), np.max(np.abs(got - ref))
    # half space: no G appears together with -G, and none is zero
    keys = {tuple(v) for v in nv}
    assert all(tuple(-v) not in keys for v in nv) and (0, 0, 0) not in keys


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_tiered"])
@pytest.mark.parametrize("case", ["sc54", "fcc100", "hex70", "diamond1"])
def test_move_sequence_matches_oracle(ew, case, prec):
    W = 5
    w = small_case(case, W)
    ctx, b = make(ew, w, prec, resum_every=3)
    info = ctx.info()
    rc, gc = info["r_cutoff"], info["g_cutoff"]
    dim, n = w["dim"], w["n"]
    rng = np.random.default_rng(77)
    ks, disp, acc = I.move_stream(rng, W, n, 12, dim, 0.4)
    pos = w["pos"].copy()
    base = [oracle_energy(w, i, rc, gc, pos[i]) for i in range(W)]
    floors = [max(abs(e), 1e-2 * scale(c)) for e, c in base]
    worst = 0.0
    for m in range(ks.shape[0]):
        r_new = pos[np.arange(W), ks[m]] + disp[m]
        de = b.propose(ks[m], r_new)
        for i in range(W):
            de_o, de_scale = oracle_move(w, i, pos[i], ks[m, i], r_new[i], rc, gc)
            assert abs(de[i] - de_o) <= TOL[prec] * floors[i], (m, i, de[i], de_o)
            assert abs(de[i] - de_o) <= DE_TOL[prec] * de_scale, (m, i, de[i], de_o, de_scale)
            worst = max(worst, abs(de[i] - de_o) / de_scale)
        b.accept(acc[m])
        for i in range(W):
            if acc[m, i]:
                pos[i, ks[m, i]] = r_new[i]
    e = b.energy()
    for i in range(W):
        e_o, c_o = oracle_energy(w, i, rc, gc, pos[i])
        assert abs(e[i] - e_o) <= TOL[prec] * max(abs(e_o), 1e-2 * scale(c_o))
    print("move dE error / dE scale, %s %s: max %.3g" % (case, prec, worst))
    # stored positions equal the oracle's up to lattice vectors
    got = b.get_positions()
    frac = (got - pos) @ np.linalg.inv(w["lattice"])
    assert np.max(np.abs(frac - np.round(frac))) < 1e-12


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_tiered"])
def test_rho_after_many_moves_without_resum(ew, prec):
    """rho(G) updated in FP64 by accepted moves stays close to a rebuild."""
    W = 4
    w = small_case("fcc100", W)
    ctx, b = make(ew, w, prec, resum_every=10 ** 6)
    rng = np.random.default_rng(5)
    ks, disp, acc = I.move_stream(rng, W, w["n"], 200, 3, 0.5)
    for m in range(ks.shape[0]):
        cur = b.get_positions()
        b.propose(ks[m], cur[np.arange(W), ks[m]] + disp[m])
        b.accept(acc[m])
    r1 = b.rho()
    b.resum()
    r2 = b.rho()
    tol = 2e-5 if prec == "mixed" else 1e-12
    assert np.max(np.abs(r1 - r2)) < tol * np.sqrt(w["n"])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_wigner_crystals_on_gpu(ew, prec):
    tol = 1e-10 if prec == "fp64" else 1e-6
    lat, pos = I.bcc_crystal(3, 1.0)
    ctx = ew.Context(3, lat, -np.ones(54), alpha=2.8 / lat[0, 0], precision=prec)
    b = ew.Batch(ctx, 2)
    b.set_positions(np.stack([pos, pos + 0.37]))
    e = b.energy() / 54
    assert np.all(np.abs(e - (-0.895929255682)) < tol)
    rs = 5.0
    lat, pos = I.hex_crystal(18, rs)
    ctx = ew.Context(2, lat, -np.ones(324), alpha=4.0 / np.sqrt(abs(np.linalg.det(lat))), precision=prec)
    b = ew.Batch(ctx, 1)
    b.set_positions(pos[None])
    e = b.energy()[0] / 324 * rs
    assert abs(e - (-1.106103)) < 5e-7


def test_energy_is_deterministic(ew):
    w = small_case("fcc100", 8)
    for prec in ("fp64", "mixed"):
        ctx, b = make(ew, w, prec)
        e1 = b.energy().copy()
        e2 = b.energy().copy()
        assert np.array_equal(e1, e2)


def test_device_pointers_match_host_path(ew):
    import torch
    w = small_case("hex70", 4)
    ctx, b = make(ew, w, "fp64", stream=torch.cuda.current_stream())
    e_host = b.energy()
    pos_d = torch.tensor(w["pos"], device="cuda")
    b.set_positions(pos_d)
    e_d = torch.zeros(4, dtype=torch.float64, device="cuda")
    b.energy(e_d)
    torch.cuda.synchronize()
    assert np.allclose(e_d.cpu().numpy(), e_host, rtol=0, atol=1e-12 * np.max(np.abs(e_host)))
    k = torch.tensor([1, 2, 3, 4], dtype=torch.int32, device="cuda")
    r_new = pos_d[torch.arange(4), k.long()] + 0.1
    de_d = b.propose(k, r_new)
    torch.cuda.synchronize()
    de_h = b.propose(k.cpu().numpy(), r_new.cpu().numpy())
    assert np.array_equal(de_d.cpu().numpy(), de_h)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_tiered"])
def test_error_codes(ew, prec):
    w = small_case("sc54", 2)
    ctx, b = make(ew, w, prec)
    with pytest.raises(ew.EwaldError) as ei:
        ew.Batch(ctx, 0)
    assert ei.value.code == 1                          # an empty batch is refused
    with pytest.raises(ew.EwaldError) as ei:
        b.accept([1, 1])
    assert ei.value.code == 4                          # no pending proposal
    with pytest.raises(ew.EwaldError) as ei:
        b.propose([0, 54], np.zeros((2, 3)))
    assert ei.value.code == 1                          # k out of range
    with pytest.raises(ew.EwaldError) as ei:
        b.propose([0, 1], np.array([[np.nan, 0, 0], [0, 0, 0]]))
    assert ei.value.code == 1                          # non-finite position
    bad = w["pos"].copy()
    bad[1, 3] = bad[1, 7] + w["lattice"][1]            # two electrons on top of each other
    b.set_positions(bad)
    with pytest.raises(ew.EwaldError) as ei:
        b.energy()
    assert ei.value.code == 3
    b.set_positions(w["pos"])                          # recovers
    assert np.all(np.isfinite(b.energy()))


# ------------------------------------------------------------ full sizes, sampled

FULL = [("heg3d_fcc_n1024", [0, 2047, 4095]), ("heg2d_hex_n338", [0, 1500]),
        ("diamond_3x3x3", [0, 1023])]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,sample", FULL)
def test_full_size_sampled_walkers(ew, name, sample, prec):
    """Each path with its default cutoffs against the oracle at the definition's
    cutoffs (1e-16 in both spaces): for the mixed path this includes the
    real-space images it leaves out beyond erfc(alpha r_c) = 1e-10."""
    w = I.workload(name)
    ctx, b = make(ew, w, prec)
    e = b.energy()
    assert np.all(np.isfinite(e))
    rc, gc = oracle.cutoffs(w["dim"], w["alpha"])
    for walker in sample:
        e_o, c_o = oracle_energy(w, walker, rc, gc)
        assert abs(e[walker] - e_o) <= TOL[prec] * max(abs(e_o), 1e-2 * scale(c_o)), (walker, e[walker], e_o)
