"""Two-body plane-wave Jastrow term on the GPU (paper Sec. 2.3, Eqs. (7),
(9), (10)) against the FP64 oracle's direct pair sums: values, gradients and
Laplacians, both precisions, through the C ABI."""
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


def case(name, W):
    rng = np.random.default_rng(99)
    if name == "fcc100":
        lat = I.fcc_lattice(100, 1.5)
        d = dict(dim=3, lattice=lat, n=100, alpha=6.0 / abs(np.linalg.det(lat)) ** (1 / 3))
        d["pos"] = I.uniform_positions(rng, lat, W, 100)
    elif name == "hex70":
        lat = I.hex_lattice(70, 3.0)
        d = dict(dim=2, lattice=lat, n=70, alpha=5.0 / np.sqrt(abs(np.linalg.det(lat))))
        d["pos"] = I.uniform_positions(rng, lat, W, 70)
    else:
        d = I.workload(name, W)
        return d
    d["q"] = -np.ones(d["n"])
    d["fixed_pos"], d["fixed_q"] = np.zeros((0, d["dim"])), np.zeros(0)
    d["n_walkers"] = W
    return d


def scales(w, k, a):
    """Magnitude scales of J_p, its gradient and Laplacian for walker k (the
    sums of absolute values of what the GPU adds up)."""
    nv, st = oracle.jastrow_stars(w["dim"], w["lattice"], len(a))
    B = 2 * np.pi * np.linalg.inv(np.asarray(w["lattice"])).T
    G = nv @ B
    rho = np.exp(1j * (w["pos"][k] @ G.T)).sum(axis=0)
    aa = np.abs(np.asarray(a)[st]) * 0.5
    n = w["n"]
    sj = np.sum(aa * 0.5 * (np.abs(rho) ** 2 + n))
    sg = np.sum(aa * np.linalg.norm(G, axis=1) * (np.abs(rho) + 1))
    sl = np.sum(aa * np.sum(G * G, axis=1) * (np.abs(rho) + 1))
    return sj, sg, sl


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,a", [("fcc100", [0.4, -0.2, 0.1, 0.05, -0.02]), ("hex70", [0.3, 0.1, -0.05]),
                                    ("heg3d_sc_n54", [0.25, -0.1, 0.04, 0.01, -0.01, 0.005])])
def test_jastrow_p_matches_oracle(ew, name, a, prec):
    w = case(name, 4)
    ctx = ew.context_for(w, precision=prec)
    n_g = ctx.set_jastrow_p(a)
    nv, _ = oracle.jastrow_stars(w["dim"], w["lattice"], len(a))
    assert 2 * n_g == len(nv)                      # one of each +-G pair
    b = ew.Batch(ctx, w["n_walkers"])
    b.set_positions(w["pos"])
    j, g, lap = b.jastrow_p()
    for k in range(w["n_walkers"]):
        jo, go, lo = oracle.jastrow_p(w["dim"], w["lattice"], w["pos"][k], a)
        sj, sg, sl = scales(w, k, a)
        assert abs(j[k] - jo) <= TOL[prec] * sj, (k, j[k], jo)
        assert np.max(np.abs(g[k] - go)) <= TOL[prec] * sg
        assert np.max(np.abs(lap[k] - lo)) <= TOL[prec] * sl
    # values only: same J
    j2, g2, l2 = b.jastrow_p(derivatives=False)
    assert g2 is None and l2 is None and np.array_equal(j2, j)


def test_jastrow_p_full_size_sampled(ew):
    w = I.workload("heg3d_fcc_n1024", 8)
    a = [0.2, -0.08, 0.03, 0.01, -0.005, 0.002, 0.001, -0.0005]
    for prec in ("fp64", "mixed"):
        ctx = ew.context_for(w, precision=prec)
        ctx.set_jastrow_p(a)
        b = ew.Batch(ctx, w["n_walkers"])
        b.set_positions(w["pos"])
        j, g, lap = b.jastrow_p()
        jo, go, lo = oracle.jastrow_p(3, w["lattice"], w["pos"][5], a)
        sj, sg, sl = scales(w, 5, a)
        assert abs(j[5] - jo) <= TOL[prec] * sj
        assert np.max(np.abs(g[5] - go)) <= TOL[prec] * sg
        assert np.max(np.abs(lap[5] - lo)) <= TOL[prec] * sl


def test_jastrow_p_errors(ew):
    w = case("fcc100", 2)
    ctx = ew.context_for(w, precision="fp64")
    b = ew.Batch(ctx, 2)
    b.set_positions(w["pos"])
    with pytest.raises(ew.EwaldError) as ei:
        b.jastrow_p()
    assert ei.value.code == 8                      # no stars set
    with pytest.raises(ew.EwaldError) as ei:
        ctx.set_jastrow_p(np.zeros(65))
    assert ei.value.code == 1
    with pytest.raises(ew.EwaldError):
        ctx.set_jastrow_p([np.nan])
    ctx.set_jastrow_p([0.1])
    assert np.all(np.isfinite(b.jastrow_p()[0]))
