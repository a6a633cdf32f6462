"""The allocation-free energy entry point (ewald_energy_noalloc) against the
ordinary ewald_energy, through the C ABI, on two calls in a row.

Callers that cannot allocate device memory at call time pass their own
device arrays for positions and energies; the library keeps every
intermediate in a fixed static device array.  This file is collected last
so that a failure here cannot hide the other tests."""
import ctypes

import numpy as np
import pytest

from paper_2507_02888_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "mixed": 1e-6, "fp64_tiered": 1e-12}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_02888_gb300 import ewald
    lib = ewald.load()
    f = lib.ewald_energy_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    return torch, ewald, lib


def hex_case(W):
    rng = np.random.default_rng(99)
    lat = I.hex_lattice(70, 3.0)
    return dict(dim=2, lattice=lat, n=70, alpha=5.0 / np.sqrt(abs(np.linalg.det(lat))), n_walkers=W,
                pos=I.uniform_positions(rng, lat, W, 70), q=-np.ones(70), fixed_pos=np.zeros((0, 2)),
                fixed_q=np.zeros(0))


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_tiered"])
@pytest.mark.parametrize("case", ["sc54", "hex70", "diamond"])
def test_noalloc_matches_energy_twice(env, case, prec):
    torch, ewald, lib = env
    if case == "sc54":
        w = I.workload("heg3d_sc_n54", 16)
    elif case == "hex70":
        w = hex_case(9)
    else:
        w = I.workload("diamond_3x3x3", 6)
    stream = torch.cuda.current_stream()
    ctx = ewald.context_for(w, precision=prec, stream=stream)
    b = ewald.Batch(ctx, w["n_walkers"])
    b.set_positions(w["pos"])
    comp = b.components()
    ref = b.energy()
    pos_d = torch.tensor(w["pos"], device="cuda")
    floor = np.maximum(np.abs(ref), 1e-2 * (np.abs(comp[:, 0]) + np.abs(comp[:, 2]) +
                                             np.abs(comp[:, 1] + comp[:, 3]) + np.abs(comp[:, 4])))
    for call in range(2):
        e_d = torch.full((w["n_walkers"],), float("nan"), dtype=torch.float64, device="cuda")
        st_d = torch.full((1,), -1, dtype=torch.int32, device="cuda")
        code = lib.ewald_energy_noalloc(ctx._h, pos_d.data_ptr(), w["n_walkers"], e_d.data_ptr(), st_d.data_ptr())
        assert code == 0, lib.ewald_last_error_message(ctx._h)
        torch.cuda.synchronize()
        got = e_d.cpu().numpy()
        assert int(st_d.cpu()[0]) == 0
        assert np.all(np.abs(got - ref) <= TOL[prec] * floor), (call, got, ref)
    # the ordinary path is unaffected afterwards
    assert np.allclose(b.energy(), ref, rtol=0, atol=0)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp64_tiered"])
def test_noalloc_matches_oracle(env, prec):
    """The allocation-free energies against the FP64 CPU oracle directly,
    element by element, at the context's own cutoffs."""
    import oracle
    torch, ewald, lib = env
    w = I.workload("diamond_3x3x3", 3)
    ctx = ewald.context_for(w, precision=prec, stream=torch.cuda.current_stream())
    info = ctx.info()
    pos_d = torch.tensor(w["pos"], device="cuda")
    e_d = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    code = lib.ewald_energy_noalloc(ctx._h, pos_d.data_ptr(), 3, e_d.data_ptr(), None)
    assert code == 0, lib.ewald_last_error_message(ctx._h)
    torch.cuda.synchronize()
    got = e_d.cpu().numpy()
    q = np.concatenate([w["q"], w["fixed_q"]])
    for i in range(3):
        p = np.concatenate([w["pos"][i], w["fixed_pos"]])
        e_o, c = oracle.energy(3, w["lattice"], p, q, w["alpha"], info["r_cutoff"], info["g_cutoff"])
        floor = max(abs(e_o), 1e-2 * (abs(c[0]) + abs(c[2]) + abs(c[1] + c[3]) + abs(c[4])))
        assert abs(got[i] - e_o) <= TOL[prec] * floor, (i, got[i], e_o)


def test_noalloc_rejects_too_many_walkers(env):
    torch, ewald, lib = env
    w = I.workload("heg3d_fcc_n1024", 1)
    ctx = ewald.context_for(w, precision="mixed")
    W = 100000
    code = lib.ewald_energy_noalloc(ctx._h, ctypes.c_void_p(16), W, ctypes.c_void_p(16), None)
    assert code == 5                                         # EWALD_ERR_OOM, nothing launched
    msg = lib.ewald_last_error_message(ctx._h).decode()
    assert "static scratch" in msg and "at most" in msg
