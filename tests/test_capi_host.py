"""Host-only checks of the C ABI (no GPU): the library loads, exports every
entry point that include/*.h declares, and rejects bad descriptions before
touching the device."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2507_02888_gb300 import ewald, serve

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(ewald_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    lib = ewald.load()
    names = declared_functions()
    assert len(names) >= 17
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    bound = {n for n, _, _ in ewald.SIGNATURES} | {n for n, _, _ in serve.SIGNATURES}
    assert set(names) <= bound | {"ewald_energy_noalloc"}


def test_strerror_names_every_code():
    lib = ewald.load()
    for code in range(10):
        assert lib.ewald_strerror(code) not in (None, b"unknown error")


def test_build_flags_tell_the_debug_library_apart():
    """The release library reports no debug checks; the debug library
    (-DEWALD_DEBUG, index checks in every kernel) reports them and exports
    the same entry points."""
    from paper_2507_02888_gb300 import build
    assert ewald.load().ewald_build_flags() & 1 == 0
    if not os.path.exists(build.LIB_DEBUG):
        pytest.skip("debug library not built (python -m paper_2507_02888_gb300.build --all)")
    dbg = ctypes.CDLL(build.LIB_DEBUG)
    dbg.ewald_build_flags.restype = ctypes.c_int
    assert dbg.ewald_build_flags() & 1 == 1
    missing = [n for n in declared_functions() if not hasattr(dbg, n)]
    assert not missing, missing


def _create(dim=3, lattice=None, q=(-1.0,), **kw):
    lib = ewald.load()
    lat = np.ascontiguousarray(np.eye(dim) * 5.0 if lattice is None else lattice, dtype=np.float64)
    qa = np.ascontiguousarray(q, dtype=np.float64)
    d = ewald.Desc(dim, lat.ctypes.data_as(ewald._dp), kw.get("n", len(qa)), qa.ctypes.data_as(ewald._dp),
                   0, None, None, kw.get("alpha", 0.5), 0.0, 0.0, kw.get("precision", 0), 0)
    h = ctypes.c_void_p()
    code = lib.ewald_create(ctypes.byref(d), None, ctypes.byref(h))
    return code, h


@pytest.mark.parametrize("case,code", [
    ("dim4", 1), ("left_handed", 2), ("singular", 2), ("no_particles", 1),
    ("nan_charge", 1), ("bad_precision", 1)])
def test_create_rejects_bad_descriptions(case, code):
    if case == "dim4":
        got, h = _create(dim=4, lattice=np.eye(4))
    elif case == "left_handed":
        got, h = _create(lattice=np.diag([5.0, 5.0, -5.0]))
    elif case == "singular":
        got, h = _create(lattice=np.array([[1.0, 0, 0], [2.0, 0, 0], [0, 0, 1.0]]))
    elif case == "no_particles":
        got, h = _create(n=0)
    elif case == "nan_charge":
        got, h = _create(q=(np.nan,))
    else:
        got, h = _create(precision=7)
    assert got == code
    assert not h.value


def _create_z(dim, n, z, zf=None, nf=0, precision=0, alpha=0.5):
    lib = ewald.load()
    lat = np.ascontiguousarray(np.eye(dim) * 9.0, dtype=np.float64)
    q = np.ascontiguousarray(-np.ones(n))
    zz = np.ascontiguousarray(z, dtype=np.float64)
    fp = np.ascontiguousarray(np.zeros((max(nf, 1), dim)))
    fq = np.ascontiguousarray(np.ones(max(nf, 1)))
    zfa = None if zf is None else np.ascontiguousarray(zf, dtype=np.float64)
    d = ewald.Desc(dim, lat.ctypes.data_as(ewald._dp), n, q.ctypes.data_as(ewald._dp), nf,
                   fp.ctypes.data_as(ewald._dp), fq.ctypes.data_as(ewald._dp), alpha, 0.0, 0.0, precision, 0,
                   zz.ctypes.data_as(ewald._dp), None if zfa is None else zfa.ctypes.data_as(ewald._dp))
    h = ctypes.c_void_p()
    return lib.ewald_create(ctypes.byref(d), None, ctypes.byref(h)), h


@pytest.mark.parametrize("case", ["heights_in_3d", "nan_height", "five_heights", "far_layers", "nan_fixed_height"])
def test_create_rejects_bad_heights(case):
    # layered 2D cells (Eqs. (5)-(6) at z != 0): every check runs on the host
    if case == "heights_in_3d":
        got, h = _create_z(3, 4, [0.0, 1.0, 0.0, 1.0])
    elif case == "nan_height":
        got, h = _create_z(2, 4, [0.0, np.nan, 0.0, 1.0])
    elif case == "five_heights":
        got, h = _create_z(2, 5, [0.0, 1.0, 2.0, 3.0, 4.0])
    elif case == "far_layers":
        got, h = _create_z(2, 4, [0.0, 1e6, 0.0, 1e6])      # |dz| g_c far beyond 600
    else:
        got, h = _create_z(2, 4, [0.0, 1.0, 0.0, 1.0], zf=[np.nan], nf=1)
    assert got == 1
    assert not h.value
