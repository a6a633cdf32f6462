"""Splitting parameter by measurement (ewald_tune_alpha): the returned alpha
lies in the searched range, is at least as fast as the starting one, and
gives the oracle's energy (alpha independence, paper Eq. (2))."""
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


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-6)])
@pytest.mark.parametrize("name", ["heg3d_sc_n54", "heg2d_hex_n338"])
def test_tuned_alpha_gives_the_same_energy(ew, name, prec, tol):
    w = I.workload(name, 8)
    a, us = ew.tune_alpha(w["dim"], w["lattice"], w["q"], w["pos"], alpha=w["alpha"], precision=prec)
    assert 0.6 * 0.93 * w["alpha"] * (1 - 1e-12) <= a <= 3.0 * 1.07 * w["alpha"] * (1 + 1e-12)
    assert us > 0
    ctx = ew.context_for(w, precision=prec, alpha=a)
    info = ctx.info()
    assert abs(info["alpha"] - a) < 1e-15 * a
    b = ew.Batch(ctx, 8)
    b.set_positions(w["pos"])
    e = b.energy()
    for k in (0, 5):
        eo, co = oracle.energy(w["dim"], w["lattice"], w["pos"][k], w["q"], a, info["r_cutoff"],
                               info["g_cutoff"])
        assert abs(e[k] - eo) <= tol * max(abs(eo), 1e-2 * scale(co))
    # and the oracle's energy does not depend on alpha
    e0, c0 = oracle.energy(w["dim"], w["lattice"], w["pos"][0], w["q"], w["alpha"],
                           *oracle.cutoffs(w["dim"], w["alpha"]))
    e1, _ = oracle.energy(w["dim"], w["lattice"], w["pos"][0], w["q"], a, *oracle.cutoffs(w["dim"], a))
    assert abs(e0 - e1) <= 1e-10 * scale(c0)


def test_tune_alpha_arguments(ew):
    w = I.workload("heg3d_sc_n54", 2)
    with pytest.raises(ew.EwaldError):
        ew.tune_alpha(3, w["lattice"], w["q"], w["pos"][:0], alpha=w["alpha"])
