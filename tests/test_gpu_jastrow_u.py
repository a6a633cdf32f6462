"""Polynomial two-body Jastrow term u on the GPU (paper Sec. 2.3, Eqs. (7),
(8)) against the FP64 oracle's direct pair sum: values, gradients and
Laplacians, both precisions, through the C ABI.  Tolerances are relative to
the sums of absolute values of the added terms (1e-12 FP64, 1e-6 mixed)."""
import itertools

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


def half_shortest(lat):
    dim = lat.shape[0]
    best = min(np.linalg.norm(np.array(m) @ lat)
               for m in itertools.product(range(-2, 3), repeat=dim) if any(m))
    return best / 2


def scales(w, k, L, C, a_like, a_unlike, n_up):
    """Sums of |u|, per particle of |u'| and of |u''| + (d-1)|u'|/r over the
    pairs inside L (nearest images by brute force): the magnitudes the GPU
    adds up, for the tolerances only."""
    lat = np.asarray(w["lattice"])
    dim = lat.shape[0]
    pos = w["pos"][k]
    n = len(pos)
    inv = np.linalg.inv(lat)
    d = pos[:, None, :] - pos[None, :, :]
    f = d @ inv
    f -= np.round(f)
    best = np.full((n, n), np.inf)
    for m in itertools.product((-1, 0, 1), repeat=dim):
        r = np.linalg.norm((f + np.array(m)) @ lat, axis=2)
        best = np.minimum(best, r)
    np.fill_diagonal(best, np.inf)
    like = (np.arange(n)[:, None] < n_up) == (np.arange(n)[None, :] < n_up)
    su, sg, sl = 0.0, np.zeros(n), np.zeros(n)
    for mask, a, gamma in ((like, a_like, 0.25 if dim == 3 else 1 / 3), (~like, a_unlike, 0.5 if dim == 3 else 1.0)):
        a = np.abs(np.asarray(a, dtype=float))
        a[1] = gamma / L ** C + C * a[0] / L              # bound of the cusp-fixed |alpha_1|
        r = np.where(mask & (best < L), best, np.nan)
        P = sum(al * r ** l for l, al in enumerate(a))
        dP = sum(l * al * r ** (l - 1) for l, al in enumerate(a) if l)
        d2P = sum(l * (l - 1) * al * r ** (l - 2) for l, al in enumerate(a) if l > 1)
        t = np.abs(r - L)
        u = t ** C * P
        du = C * t ** (C - 1) * P + t ** C * dP
        d2u = C * (C - 1) * t ** max(C - 2, 0) * P + 2 * C * t ** (C - 1) * dP + t ** C * d2P
        su += 0.5 * np.nansum(u)
        sg += np.nansum(du, axis=1)
        sl += np.nansum(d2u + (dim - 1) * du / r, axis=1)
    return su, sg, sl


def case(name, W, seed=17):
    rng = np.random.default_rng(seed)
    if name == "fcc100":
        lat = I.fcc_lattice(100, 1.5)
        d = dict(dim=3, lattice=lat, n=100, alpha=6.0 / abs(np.linalg.det(lat)) ** (1 / 3))
    elif name == "hex70":
        lat = I.hex_lattice(70, 3.0)
        d = dict(dim=2, lattice=lat, n=70, alpha=5.0 / np.sqrt(abs(np.linalg.det(lat))))
    else:
        return I.workload(name, W)
    d["pos"] = I.uniform_positions(rng, lat, W, d["n"])
    d["q"] = -np.ones(d["n"])
    d["fixed_pos"], d["fixed_q"] = np.zeros((0, d["dim"])), np.zeros(0)
    d["n_walkers"] = W
    return d


B_LIKE = [0.31, 0.0, -0.2, 0.4, 0.1, -0.2, 0.3]
B_UNLIKE = [0.55, 0.0, 0.3, -0.6, 0.5, 0.1, -0.1]


def coefs(L, C):
    """alpha_l = b_l / L^(l + C): u = (x - 1)^C sum_l b_l x^l in x = r / L, of order one."""
    return ([b / L ** (l + C) for l, b in enumerate(B_LIKE)], [b / L ** (l + C) for l, b in enumerate(B_UNLIKE)])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name,C,frac_up", [("fcc100", 3, 0.5), ("hex70", 2, 0.5), ("heg3d_sc_n54", 3, 1.0),
                                           ("fcc100", 2, 0.3)])
def test_jastrow_u_matches_oracle(ew, name, C, frac_up, prec):
    w = case(name, 3)
    L = 0.97 * half_shortest(np.asarray(w["lattice"]))
    n_up = int(frac_up * w["n"])
    ctx = ew.context_for(w, precision=prec)
    al, au = coefs(L, C)
    ctx.set_jastrow_u(n_up, L, C, al, au)
    b = ew.Batch(ctx, w["n_walkers"])
    b.set_positions(w["pos"])
    j, g, lap = b.jastrow_u()
    for k in range(w["n_walkers"]):
        jo, go, lo = oracle.jastrow_u(w["dim"], w["lattice"], w["pos"][k], n_up, L, C, al, au)
        su, sg, sl = scales(w, k, L, C, al, au, n_up)
        assert abs(j[k] - jo) <= TOL[prec] * su, (k, j[k], jo, su)
        assert np.all(np.abs(g[k] - go) <= TOL[prec] * sg[:, None])
        assert np.all(np.abs(lap[k] - lo) <= TOL[prec] * sl)
    j2, g2, l2 = b.jastrow_u(derivatives=False)
    assert g2 is None and l2 is None and np.array_equal(j2, j)


def test_jastrow_u_full_size_sampled(ew):
    w = I.workload("heg3d_fcc_n1024", 8)
    L = 0.99 * half_shortest(np.asarray(w["lattice"]))
    al, au = coefs(L, 3)
    for prec in ("fp64", "mixed"):
        ctx = ew.context_for(w, precision=prec)
        ctx.set_jastrow_u(512, L, 3, al, au)
        b = ew.Batch(ctx, w["n_walkers"])
        b.set_positions(w["pos"])
        j, g, lap = b.jastrow_u()
        jo, go, lo = oracle.jastrow_u(3, w["lattice"], w["pos"][6], 512, L, 3, al, au)
        su, sg, sl = scales(w, 6, L, 3, al, au, 512)
        assert abs(j[6] - jo) <= TOL[prec] * su
        assert np.all(np.abs(g[6] - go) <= TOL[prec] * sg[:, None])
        assert np.all(np.abs(lap[6] - lo) <= TOL[prec] * sl)


def test_jastrow_u_errors(ew):
    w = case("fcc100", 2)
    lat = np.asarray(w["lattice"])
    ctx = ew.context_for(w, precision="fp64")
    b = ew.Batch(ctx, 2)
    b.set_positions(w["pos"])
    with pytest.raises(ew.EwaldError) as ei:
        b.jastrow_u()
    assert ei.value.code == 8                                   # no u term set
    for args in ((50, 1.01 * half_shortest(lat), 3), (50, 0.5, 0), (50, 0.5, 9), (101, 0.5, 3), (-1, 0.5, 3)):
        with pytest.raises(ew.EwaldError) as ei:
            ctx.set_jastrow_u(args[0], args[1], args[2], B_LIKE, B_UNLIKE)
        assert ei.value.code == 1
    with pytest.raises(ew.EwaldError):
        ctx.set_jastrow_u(50, 0.5, 3, [np.nan, 0.0], [0.1, 0.0])
    ctx.set_jastrow_u(50, 0.9 * half_shortest(lat), 3, [0.1, 0.0], [0.2, 0.0])
    assert np.all(np.isfinite(b.jastrow_u()[0]))
