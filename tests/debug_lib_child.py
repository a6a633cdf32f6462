"""Child process of test_gpu_debug_build: runs the cases of that test through
whichever library EWALD_LIBRARY selects and saves the results to the .npz
named on the command line (energies, components, proposed dE of three move
rounds, batched energies).  Any status the kernels raise (in the debug build:
an index caught out of range) comes back as an EwaldError and a non-zero
exit."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2507_02888_gb300 import ewald  # noqa: E402
from paper_2507_02888_gb300 import inputs as I  # noqa: E402

# (workload, walkers): 3D gas, 2D gas, 2D bilayer, diamond (fixed ions)
CASES = [("heg3d_sc_n54", 16), ("heg2d_hex_n338", 4), ("ehbilayer2d_hex_n338", 4), ("diamond_3x3x3", 2)]
PRECISIONS = ["fp64", "mixed", "fp64_tiered"]


def run_case(name, W, prec, out):
    w = I.workload(name, n_walkers=W)
    ctx = ewald.context_for(w, precision=prec)
    b = ewald.Batch(ctx, W)
    b.set_positions(w["pos"])
    tag = "%s.%s" % (name, prec)
    out[tag + ".energy"] = b.energy().copy()
    out[tag + ".comp"] = b.components().copy()
    ks, disp, acc = I.move_stream(np.random.default_rng(5), W, w["n"], 3, w["dim"], w["sigma"])
    pos = w["pos"].copy()
    des = []
    for m in range(3):
        r_new = pos[np.arange(W), ks[m]] + disp[m]
        des.append(b.propose(ks[m], r_new).copy())
        b.accept(acc[m])
        sel = acc[m].astype(bool)
        pos[np.arange(W)[sel], ks[m][sel]] = r_new[sel]
    out[tag + ".de"] = np.array(des)
    out[tag + ".after"] = b.energy().copy()
    b.close()
    ctx.close()


def run_multi(prec, out):
    # one persistent launch over two systems of different composition
    ws = [I.workload("diamond_3x3x3", n_walkers=2), I.workload("heg3d_sc_n54", n_walkers=8)]
    ctxs = [ewald.context_for(w, precision=prec) for w in ws]
    bs = [ewald.Batch(c, w["n_walkers"]) for c, w in zip(ctxs, ws)]
    for b, w in zip(bs, ws):
        b.set_positions(w["pos"])
    m = ewald.Multi(bs)
    out["multi.%s" % prec] = m.energy().copy()
    m.close()
    for b in bs:
        b.close()
    for c in ctxs:
        c.close()


def main(path):
    ewald.load(build_if_missing=False)
    out = {"build_flags": np.array(ewald.build_flags())}
    errors = []
    # every case runs, so one run names every check that fires
    for name, W in CASES:
        for prec in PRECISIONS:
            try:
                run_case(name, W, prec, out)
            except ewald.EwaldError as e:
                errors.append("%s %s: %s" % (name, prec, e))
    for prec in PRECISIONS:
        try:
            run_multi(prec, out)
        except ewald.EwaldError as e:
            errors.append("multi %s: %s" % (prec, e))
    np.savez(path, **out)
    if errors:
        sys.exit("\n".join(errors))


if __name__ == "__main__":
    main(sys.argv[1])
