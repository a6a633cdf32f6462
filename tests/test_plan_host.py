"""The host set-up through ewald_plan, on the CPU (no GPU needed).

ewald_plan runs the host part of ewald_create (validation, cutoffs, the
half-space G list, image and candidate lists, the constant energy terms, all
in FP64; paper Sec. 6.1) and its default real-space tiling.  These tests pin
that set-up against the FP64 oracle's own definitions: the cutoffs (the
oracle bisects erfc(alpha r_c) = tol where the library takes Newton steps on
log erfc), the number of G vectors inside g_c (the oracle counts a box of
integer vectors), and the Madelung, self and background terms and the
fixed-ion pair sum (the oracle sums them from their definitions, paper
Eqs. (2)-(6)).  The mixed form's choice of taking each pair's two nearest
images without the lane rings is checked too.
"""
import ctypes

import numpy as np
import pytest

import oracle
from cases import small_case
from paper_2507_02888_gb300 import ewald
from paper_2507_02888_gb300 import inputs as I

MIXED_REAL_TOL = 1e-10  # the mixed form's real-space cutoff: erfc(alpha r_c) = 1e-10


def system(name):
    if name in ("heg3d_fcc_n1024", "heg2d_hex_n338", "diamond_3x3x3", "ehbilayer2d_hex_n338"):
        return I.workload(name, 1)
    return small_case(name, 1)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_tiered"])
@pytest.mark.parametrize("name", ["fcc100", "diamond1", "hex70", "sc54", "heg3d_fcc_n1024", "diamond_3x3x3"])
def test_plan_cutoffs_and_g_count_match_oracle(name, prec):
    w = system(name)
    info = ewald.plan_for(w, prec)
    rc, gc = oracle.cutoffs(w["dim"], w["alpha"])
    if prec == "mixed":
        rc, _ = oracle.cutoffs(w["dim"], w["alpha"], MIXED_REAL_TOL)
    assert abs(info["r_cutoff"] / rc - 1) < 1e-9
    assert abs(info["g_cutoff"] / gc - 1) < 1e-9
    assert 2 * info["n_g_half"] == oracle.gcount(w["dim"], w["lattice"], gc)
    assert info["precision"] == ewald.PRECISIONS[prec]
    assert info["n_mobile"] == len(w["q"]) and info["n_fixed"] == len(w["fixed_q"])
    assert abs(info["volume"] - abs(np.linalg.det(w["lattice"]))) <= 1e-12 * info["volume"]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["fcc100", "diamond1", "hex70", "mixed_q", "single"])
def test_plan_constants_match_oracle(name, prec):
    """Madelung, self and background terms (and, with ions, the ions' own
    real-space pair sum) against the oracle's energy components at the
    plan's cutoffs: they do not depend on the mobile particles' positions."""
    w = system(name)
    info = ewald.plan_for(w, prec)
    rc, gc = info["r_cutoff"], info["g_cutoff"]
    q = np.concatenate([w["q"], w["fixed_q"]])
    pos = np.concatenate([w["pos"][0], w["fixed_pos"]])
    _, c = oracle.energy(w["dim"], w["lattice"], pos, q, w["alpha"], rc, gc)
    for key, ref in (("e_madelung", c[1]), ("e_self", c[3]), ("e_background", c[4])):
        assert abs(info[key] - ref) <= 1e-12 * max(abs(ref), 1e-300), (key, info[key], ref)
    if len(w["fixed_q"]):
        _, ci = oracle.energy(w["dim"], w["lattice"], w["fixed_pos"], w["fixed_q"], w["alpha"], rc, gc)
        assert abs(info["e_fixed_real"] - ci[0]) <= 1e-12 * abs(ci[0])
    else:
        assert info["e_fixed_real"] == 0.0


def test_plan_layered_background_matches_oracle():
    """A layered 2D cell (electron-hole bilayer): the background term of the
    charged sheets at their height differences (paper Eq. (5), G = 0)."""
    w = I.workload("ehbilayer2d_hex_n338", 1)
    info = ewald.plan_for(w, "fp64")
    assert info["n_layers"] == 2
    _, c = oracle.energy_z(w["lattice"], w["pos"][0], w["z"], w["q"], w["alpha"], info["r_cutoff"],
                           info["g_cutoff"])
    assert abs(info["e_background"] - c[4]) <= 1e-12 * abs(c[4])


def test_plan_mixed_direct_choice():
    """The mixed form takes each pair's first two images (the two nearest to
    the displacement cell's centre) without the lane rings where lists hold
    3 to 8 images and the second of them lies inside r_c for at least 3/4 of
    the displacements; the same choice as the contexts report on the GPU."""
    want = {"mixed_q": 1, "clustered": 1, "hex70": 1, "heg3d_fcc_n1024": 1, "diamond_3x3x3": 1,
            "fcc100": 0, "diamond1": 0, "sc54": 0, "heg2d_hex_n338": 0}
    for name, flag in want.items():
        info = ewald.plan_for(system(name), "mixed")
        assert info["mixed_direct"] == flag, name
        if flag:
            assert 3 <= info["max_candidates"] <= 8, name


def test_plan_tiling_defaults():
    """The default tiling: 256-particle tiles for the mixed form where they
    pad no more than 128-particle tiles, displacement cells whose mixed
    tables fit the 24 KB cap."""
    w = I.workload("heg3d_fcc_n1024", 1)
    assert ewald.plan_for(w, "mixed")["pair_tile"] == 256
    assert ewald.plan_for(w, "fp64")["pair_tile"] == 128
    assert ewald.plan_for(system("sc54"), "mixed")["pair_tile"] == 32


def _plan_code(dim=3, lattice=None, q=(-1.0,), **kw):
    lib = ewald.load()
    lat = np.ascontiguousarray(np.eye(dim) * 5.0 if lattice is None else lattice, dtype=np.float64)
    qa = np.ascontiguousarray(q, dtype=np.float64)
    d = ewald.Desc(dim, lat.ctypes.data_as(ewald._dp), kw.get("n", len(qa)), qa.ctypes.data_as(ewald._dp),
                   0, None, None, kw.get("alpha", 0.5), 0.0, 0.0, kw.get("precision", 0), 0)
    info = ewald.Info()
    return lib.ewald_plan(ctypes.byref(d), ctypes.byref(info))


@pytest.mark.parametrize("case,code", [
    ("dim4", 1), ("left_handed", 2), ("singular", 2), ("no_particles", 1),
    ("nan_charge", 1), ("bad_precision", 1), ("null", 1)])
def test_plan_rejects_bad_descriptions(case, code):
    """The same validation and codes as ewald_create."""
    if case == "dim4":
        got = _plan_code(dim=4, lattice=np.eye(4))
    elif case == "left_handed":
        got = _plan_code(lattice=np.diag([5.0, 5.0, -5.0]))
    elif case == "singular":
        got = _plan_code(lattice=np.array([[1.0, 0, 0], [2.0, 0, 0], [0, 0, 1.0]]))
    elif case == "no_particles":
        got = _plan_code(n=0)
    elif case == "nan_charge":
        got = _plan_code(q=(np.nan,))
    elif case == "bad_precision":
        got = _plan_code(precision=7)
    else:
        got = ewald.load().ewald_plan(None, None)
    assert got == code


@pytest.mark.parametrize("name", ["heg3d_fcc_n1024", "sc54", "diamond_3x3x3", "heg2d_hex_n338"])
def test_plan_balanced_alpha(name):
    """gamma <= 0 lets the library pick alpha.  At its choice the real-space
    work, N particles times the images inside r_c (the r_c sphere's volume, or
    disc's area, over the cell's), matches the reciprocal work, the number of
    G vectors inside g_c that the oracle counts, within 5%; and the cutoffs
    follow the 1e-16 definitions at that alpha."""
    w = system(name)
    info = ewald.plan_for(w, "fp64", alpha=0.0)
    a, dim = info["alpha"], w["dim"]
    rc, gc = oracle.cutoffs(dim, a)
    assert abs(info["r_cutoff"] / rc - 1) < 1e-9 and abs(info["g_cutoff"] / gc - 1) < 1e-9
    n = len(w["q"]) + len(w["fixed_q"])
    per = (4 * np.pi / 3 * rc ** 3 if dim == 3 else np.pi * rc ** 2) / info["volume"]
    n_g = oracle.gcount(dim, w["lattice"], gc)
    assert abs(n * per / n_g - 1) < 0.05, (n * per, n_g)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["fcc100", "diamond1", "hex70", "sc54", "heg3d_fcc_n1024"])
def test_plan_image_count(name, prec):
    """The real-space image list holds every lattice vector R that a wrapped
    displacement d (fractional coordinates in [-1/2, 1/2)) can bring inside
    r_c: |R| < r_c + max |d|.  Counted here over a box of integer vectors
    wide enough for that radius (|m_k| <= reach |b_k| / 2 pi)."""
    import itertools
    w = system(name)
    info = ewald.plan_for(w, prec)
    A = np.asarray(w["lattice"], dtype=float)
    dim = A.shape[0]
    corners = np.array(list(itertools.product([-0.5, 0.5], repeat=dim)))
    reach = info["r_cutoff"] + np.max(np.linalg.norm(corners @ A, axis=1))
    B = 2 * np.pi * np.linalg.inv(A).T
    span = [int(np.ceil(reach * np.linalg.norm(B[k]) / (2 * np.pi))) for k in range(dim)]
    m = np.array(list(itertools.product(*[range(-s, s + 1) for s in span])), dtype=float)
    assert info["n_images"] == int(np.sum(np.linalg.norm(m @ A, axis=1) < reach))
