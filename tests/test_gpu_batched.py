"""Batched form: walkers of several systems (3D/2D, with and without ions,
different N) in one persistent launch, against each batch alone and against
the oracle."""
import numpy as np
import pytest

import oracle
from paper_2507_02888_gb300 import inputs as I

pytestmark = pytest.mark.gpu


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


def small_diamond(W):
    rng = np.random.default_rng(31)
    lat, ions = I.diamond_ions(1, 6.74)
    d = dict(name="diamond1", dim=3, lattice=lat, n=32, alpha=0.9, n_walkers=W)
    d["pos"] = I.scattered_positions(rng, ions, W, 32, 0.8)
    d["q"] = -np.ones(32)
    d["fixed_pos"], d["fixed_q"] = ions, 4.0 * np.ones(len(ions))
    return d


def mix(W=(5, 7, 3, 4)):
    return [I.workload("heg3d_sc_n54", W[0]), I.workload("heg2d_hex_n338", W[1]), small_diamond(W[2]),
            I.workload("heg3d_sc_n128", W[3])]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_multi_equals_single_batches(ew, prec):
    ws = mix()
    ctxs = [ew.context_for(w, precision=prec) for w in ws]
    bs = []
    for c, w in zip(ctxs, ws):
        b = ew.Batch(c, w["n_walkers"])
        b.set_positions(w["pos"])
        bs.append(b)
    comps = np.concatenate([b.components() for b in bs])
    alone = comps.sum(axis=1)
    floor = np.maximum(np.abs(alone), 1e-2 * np.abs(comps).sum(axis=1))
    m = ew.Multi(bs)
    e1 = m.energy().copy()
    e2 = m.energy().copy()       # graph replay gives the same bits as the first launch
    # the same terms as the single-batch kernels; the persistent kernel splits
    # each 32 x 32 sub-tile into j slices to keep its 8 warps busy, so its
    # partial sums are added in another (fixed) order: equal to rounding
    tol = 1e-13 if prec == "fp64" else 1e-6
    assert np.all(np.abs(e1 - alone) <= tol * floor), np.max(np.abs(e1 - alone) / floor)
    assert np.array_equal(e1, e2)
    # each batch is still usable on its own afterwards
    assert np.allclose(bs[1].energy(), alone[5:12], rtol=0, atol=tol * floor[5:12].max())


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_multi_matches_oracle(ew, prec):
    tol = 1e-12 if prec == "fp64" else 1e-6
    ws = mix((2, 2, 2, 2))
    ctxs = [ew.context_for(w, precision=prec) for w in ws]
    bs = []
    for c, w in zip(ctxs, ws):
        b = ew.Batch(c, w["n_walkers"])
        b.set_positions(w["pos"])
        bs.append(b)
    e = ew.Multi(bs).energy()
    k = 0
    for c, w in zip(ctxs, ws):
        info = c.info()
        for i in range(w["n_walkers"]):
            p = np.concatenate([w["pos"][i], w["fixed_pos"]])
            q = np.concatenate([w["q"], w["fixed_q"]])
            e_o, c_o = oracle.energy(w["dim"], w["lattice"], p, q, w["alpha"], info["r_cutoff"], info["g_cutoff"])
            assert abs(e[k] - e_o) <= tol * max(abs(e_o), 1e-2 * scale(c_o)), (w["name"], i, e[k], e_o)
            k += 1


def test_multi_rejects_mixed_precisions(ew):
    w = I.workload("heg3d_sc_n54", 2)
    b1 = ew.Batch(ew.context_for(w, precision="fp64"), 2)
    b2 = ew.Batch(ew.context_for(w, precision="mixed"), 2)
    b1.set_positions(w["pos"])
    b2.set_positions(w["pos"])
    with pytest.raises(ew.EwaldError):
        ew.Multi([b1, b2])
