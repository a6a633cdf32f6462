"""Every ABI entry point opens an NVTX range named after itself, so that a
profiler's timeline shows the library calls around their kernels.  Checked
with a small injection library (tests/nvtx/nvtx_record.c) that records the
ranges; ewald_create pushes and pops its range even where it then fails
for want of a GPU."""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

CHILD = r'''
import sys
sys.path.insert(0, %r)
import numpy as np
from paper_2507_02888_gb300 import ewald, inputs as I
w = I.workload("heg3d_sc_n54", 2)
try:
    ctx = ewald.context_for(w, precision="mixed")
    ctx.close()
except ewald.EwaldError:
    pass                       # no GPU here: the range is still recorded
'''


def test_entry_points_open_nvtx_ranges(tmp_path):
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    if not os.path.exists(os.path.join(cuda, "include", "nvtx3", "nvToolsExt.h")):
        pytest.skip("no NVTX headers")
    lib = str(tmp_path / "librecord.so")
    subprocess.check_call(["gcc", "-O1", "-fPIC", "-shared", "-I", os.path.join(cuda, "include"), "-o", lib,
                           os.path.join(HERE, "nvtx", "nvtx_record.c")])
    log = str(tmp_path / "nvtx.log")
    env = dict(os.environ, NVTX_INJECTION64_PATH=lib, EWALD_NVTX_LOG=log)
    subprocess.run([sys.executable, "-c", CHILD % ROOT], env=env, check=True, timeout=300)
    lines = open(log).read().split("\n")
    assert "push ewald_create" in lines
    pushes = [l for l in lines if l.startswith("push ")]
    assert len(pushes) == lines.count("pop")                 # every range closed
