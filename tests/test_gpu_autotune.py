"""The autotuner (ewald_autotune): real-space tiling, the mixed form's CTA
size and the structure-factor chunking chosen by timing, stored in and read
back from its JSON cache; a tuned context computes the oracle's energies."""
import json

import numpy as np
import pytest

import oracle
from paper_2507_02888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-6}


@pytest.fixture(scope="module")
def ew():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_02888_gb300 import ewald
    ewald.load()
    return ewald


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_autotune_choice_cache_and_energies(ew, prec, tmp_path, monkeypatch):
    w = I.workload("heg3d_sc_n128", 64)
    ctx = ew.context_for(w, precision=prec)
    b = ew.Batch(ctx, 64)
    b.set_positions(w["pos"])
    e0 = b.energy().copy()
    cache = str(tmp_path / "tune.json")
    r = b.autotune(cache)
    assert r["from_cache"] == 0 and r["n_tried"] >= 2 and r["ms"] > 0 and r["sfac_ms"] > 0
    assert r["pair_tile"] in (32, 64, 128, 256) and r["sfac_chunks"] >= 1
    assert r["real_threads"] in ((256, 512) if prec == "mixed" else (128,))
    info = ctx.info()
    assert info["pair_tile"] == r["pair_tile"] and info["subcell_bits"] == r["subcell_bits"]
    # the tuned configuration computes the oracle's energies
    e1 = b.energy()
    rc, gc = info["r_cutoff"], info["g_cutoff"]
    for i in (0, 31, 63):
        e_o, c = oracle.energy(3, w["lattice"], w["pos"][i], w["q"], w["alpha"], rc, gc)
        floor = max(abs(e_o), 1e-2 * (abs(c[0]) + abs(c[2]) + abs(c[1] + c[3]) + abs(c[4])))
        assert abs(e1[i] - e_o) <= TOL[prec] * floor
        assert abs(e1[i] - e0[i]) <= 2 * TOL[prec] * floor
    # the cache holds the choice and gives it back without timing
    entries = json.load(open(cache))["entries"]
    assert len(entries) == 1 and entries[0]["tile"] == r["pair_tile"] and entries[0]["chunks"] >= 1
    r2 = b.autotune(cache)
    assert r2["from_cache"] == 1 and r2["pair_tile"] == r["pair_tile"] and r2["subcell_bits"] == r["subcell_bits"]
    assert r2["real_threads"] == r["real_threads"] and r2["sfac_chunks"] == r["sfac_chunks"]
    b.close()
    ctx.close()
    # a new context of the same system takes the cached tiling at creation
    monkeypatch.setenv("EWALD_TUNE_CACHE", cache)
    ctx2 = ew.context_for(w, precision=prec)
    i2 = ctx2.info()
    assert i2["pair_tile"] == r["pair_tile"] and i2["subcell_bits"] == r["subcell_bits"]
    b2 = ew.Batch(ctx2, 64)
    b2.set_positions(w["pos"])
    assert np.array_equal(b2.energy(), e1)
    ctx2.close()
