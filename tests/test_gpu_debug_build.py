"""The debug library (built with -DEWALD_DEBUG) against the release library.

In the debug build every kernel checks the indices it derives on the device
(lane rings and warp queues within their capacity, displacement-cell and
candidate-list ids within their tables, the moved particle's partners within
the particle arrays) and reports a miss through the batch's status word,
which the host turns into EWALD_ERR_STATE.  Each build runs the same cases in
a child process (3D and 2D gases, the 2D bilayer, diamond with fixed ions,
every precision form; energies, components, three rounds of moves, one
batched launch over two systems):

* the debug run finishes with no status raised;
* the debug library reports EWALD_BUILD_DEBUG_CHECKS and the release one
  does not;
* the results agree: the checks change no arithmetic, so the two builds
  differ at most by the compiler's different instruction choices, held to
  1e-12 (FP64 forms) and 1e-7 (mixed form) of each walker's energy scale.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
TOL = {"fp64": 1e-12, "mixed": 1e-7, "fp64_tiered": 1e-12}


def run_child(variant, path):
    env = dict(os.environ, EWALD_LIBRARY=variant)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_lib_child.py"), path], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, "%s build run failed:\n%s%s" % (variant, r.stdout[-3000:], r.stderr[-3000:])
    return dict(np.load(path))


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_02888_gb300 import build
    if not os.path.exists(build.LIB_DEBUG) or not os.path.exists(build.LIB):
        pytest.fail("both libraries are built by __graft_entry__.build()")
    d = tmp_path_factory.mktemp("dbg")
    return run_child("release", str(d / "rel.npz")), run_child("debug", str(d / "dbg.npz"))


def test_build_flags(results):
    rel, dbg = results
    assert int(rel["build_flags"]) & 1 == 0
    assert int(dbg["build_flags"]) & 1 == 1


def test_debug_matches_release(results):
    rel, dbg = results
    assert set(rel) == set(dbg)
    worst = {}
    for key in sorted(rel):
        if key == "build_flags" or key.endswith(".comp"):
            continue
        parts = key.split(".")
        prec = parts[1]
        comp = rel.get(parts[0] + "." + prec + ".comp")
        a, g = np.asarray(rel[key], dtype=float), np.asarray(dbg[key], dtype=float)
        if comp is not None:
            # each walker's scale |E_real| + |E_recip| + |E_mad + E_self| + |E_bg|
            c = np.asarray(comp)
            sc = np.abs(c[:, 0]) + np.abs(c[:, 2]) + np.abs(c[:, 1] + c[:, 3]) + np.abs(c[:, 4])
        else:
            sc = np.maximum(np.abs(a), 1.0)
        assert np.all(np.isfinite(g)), key
        err = float(np.max(np.abs(a - g) / sc))
        worst[key] = err
        assert err <= TOL[prec], (key, err)
    print("debug vs release, worst relative difference: %.3g" % max(worst.values()))
