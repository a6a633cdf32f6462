"""A large system: 4096 electrons in a simple-cubic cell (64 pair tiles of
64 per side, 31918 G vectors), against the oracle on a sampled walker, in
both precisions: full energy and one move energy change.  Also the Jastrow
u term's refusal when the walker's particles do not fit its shared-memory
tile (EWALD_ERR_ARG, no launch)."""
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


def big(W=3):
    n = 4096
    lat = I.sc_lattice(n, 2.0)
    rng = np.random.default_rng(5)
    alpha = 2.0 * (4000.0 * 6.0 * np.pi ** 2 / abs(np.linalg.det(lat))) ** (1.0 / 3.0) / 12.1394
    return dict(dim=3, lattice=lat, n=n, alpha=alpha, n_walkers=W, pos=I.uniform_positions(rng, lat, W, n),
                q=-np.ones(n), fixed_pos=np.zeros((0, 3)), fixed_q=np.zeros(0))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_4096_electrons(ew, prec):
    w = big()
    ctx = ew.context_for(w, precision=prec)
    info = ctx.info()
    b = ew.Batch(ctx, w["n_walkers"])
    b.set_positions(w["pos"])
    e = b.energy()
    rc16, gc = oracle.cutoffs(3, w["alpha"])
    eo, co = oracle.energy(3, w["lattice"], w["pos"][1], w["q"], w["alpha"], rc16, gc)
    floor = max(abs(eo), 1e-2 * (abs(co[0]) + abs(co[2]) + abs(co[1] + co[3]) + abs(co[4])))
    assert abs(e[1] - eo) <= TOL[prec] * floor, (e[1], eo)
    # one move of electron 4000 of every walker
    pos = b.get_positions()
    rng = np.random.default_rng(3)
    rn = pos[:, 4000] + rng.normal(scale=0.3, size=(w["n_walkers"], 3))
    de = b.propose(np.full(w["n_walkers"], 4000), rn)
    deo = oracle.delta_e(3, w["lattice"], pos[1], w["q"], 4000, rn[1], w["alpha"], info["r_cutoff"],
                         info["g_cutoff"])
    assert abs(de[1] - deo) <= TOL[prec] * floor, (de[1], deo)


def test_u_term_refuses_a_walker_larger_than_its_tile(ew):
    n = 16384
    lat = I.sc_lattice(n, 2.0)
    ctx = ew.Context(3, lat, -np.ones(n), alpha=0.12, precision="fp64")
    with pytest.raises(ew.EwaldError) as ei:
        ctx.set_jastrow_u(n // 2, 0.45 * lat[0, 0], 3, [0.1, 0.0, 0.01], [0.2, 0.0, 0.01])
    assert ei.value.code == 1
