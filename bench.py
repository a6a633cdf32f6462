#!/usr/bin/env python3
"""Benchmark of the Ewald hot path on GB300.

One step = one full Ewald energy of every walker of the batch (structure
factor + reciprocal energy, real-space pair sum, combine) followed by
--moves rounds of single-electron propose + accept for every walker.  The
headline value is walker Ewald energies per second of the mixed-precision
batched form; move dE/s, the plain-FP64 form, the end-to-end numbers through
host buffers, the roofline of the dominant kernel, the CPU oracle baseline
and the SM clocks are reported on the same JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

For N > 1 it is launched with torch.distributed.run, one rank per GPU; each
rank evaluates its own batch (walkers are independent: weak scaling, no
data-path collective).  Timing: CUDA events on the library's stream, barrier
and synchronize on both sides, max over ranks.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "walker Ewald energies/s + move ΔE/s, mixed batched vs plain FP64; p50/p99 ms"
FLOP_REAL_TERM = 25   # per real-space term inside r_c
FLOP_G_TERM = 16      # per (electron, G) structure-factor term
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="heg3d_fcc_n1024")
    p.add_argument("--walkers", type=int, default=0, help="0 = the workload's walker count")
    p.add_argument("--moves", type=int, default=4, help="propose+accept rounds per step")
    p.add_argument("--fp64-steps", type=int, default=2)
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-seconds", type=float, default=12.0)
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--no-configs", action="store_true", help="skip the per-config table (c0, c2, c3)")
    p.add_argument("--no-jastrow", action="store_true", help="skip the two-body plane-wave Jastrow term")
    p.add_argument("--no-tune-alpha", action="store_true", help="skip the measured alpha balancing leg")
    p.add_argument("--serve-requests", type=int, default=2000)
    p.add_argument("--serve-requests-fp64", type=int, default=120,
                   help="plain-FP64 serving leg (2000 takes ~6 min: run it on request)")
    p.add_argument("--serve-requests-tiered", type=int, default=2000)
    return p.parse_args()


# ----------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) of the GPU in use while the timed region runs."""
    Q = ("pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id):
        self.bus = bus_id.lower() if bus_id else ""
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9 or (self.bus and not c[0].lower().endswith(self.bus)):
                continue
            try:
                rows.append((float(c[1]), float(c[2]), c[5:9]))
            except ValueError:
                pass
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": reasons}


# ------------------------------------------------------------------ CPU oracle

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_walker_energies(w, walkers, rc, gc, threads):
    """Oracle energies of the given walkers on `threads` host threads (ctypes releases the GIL)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle
    pos_all = np.concatenate([w["pos"][list(walkers)], np.broadcast_to(
        w["fixed_pos"], (len(walkers),) + w["fixed_pos"].shape)], axis=1)
    q = np.concatenate([w["q"], w["fixed_q"]])

    def one(i):
        return oracle.energy(w["dim"], w["lattice"], pos_all[i], q, w["alpha"], rc, gc)[0]

    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(one, range(len(walkers))))


def cpu_model():
    """Host CPU model name (lscpu; /proc/cpuinfo as a fallback), for the baseline's record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_oracle_rate(w, rc, gc, seconds):
    """Walker energies/s of the oracle on one host thread and on all host
    cores (one walker per thread at a time), on bounded samples."""
    import oracle
    cores = host_cores()
    oracle.build()
    oracle_walker_energies(w, [0], rc, gc, 1)          # load the library outside the timing
    t0 = time.perf_counter()
    oracle_walker_energies(w, [1, 2], rc, gc, 1)
    t1 = (time.perf_counter() - t0) / 2                  # one walker on one thread
    rounds = max(1, min(4, int(seconds / max(t1, 1e-3))))
    n = cores * rounds
    walkers = [i % w["n_walkers"] for i in range(n)]
    t0 = time.perf_counter()
    oracle_walker_energies(w, walkers, rc, gc, cores)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "walker energies/s", "cores": cores, "kind": "oracle",
            "one_thread": 1.0 / t1, "nproc": os.cpu_count(), "cpu_model": cpu_model(),
            "sample": "%d walkers of %s (%d per host thread) on %d threads, plain FP64 C oracle, %.1f s wall; "
                      "one thread: 2 walkers, %.2f s each" % (n, w["name"], rounds, cores, dt, t1)}


# ------------------------------------------------------------------- our arm

def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


# the sources of the mixed-precision real-space kernel k_real_mixed: the
# committed DRAM traffic counts only while none of them has changed
REAL_SOURCES = ["paper_2507_02888_gb300/csrc/real_mixed.cu", "paper_2507_02888_gb300/csrc/real_mixed.cuh",
                "paper_2507_02888_gb300/csrc/ewald_internal.h", "paper_2507_02888_gb300/csrc/device_common.cuh"]


def real_kernel_name(info, w):
    """The k_real_mixed instantiation the library launches for this system:
    candidate slots rounded up to 2, 4, 6 or 8 (0: longer lists, walked in
    chunks), whether the pair weights vary (the mobile or the fixed charges
    not all equal in FP32) and whether the first two images of a pair are
    evaluated without the lane rings (mixed_direct)."""
    cm = next((c for c in (2, 4, 6, 8) if info["max_candidates"] <= c), 0)
    qw = int(any(len(q) and np.ptp(np.asarray(q, dtype=np.float32)) != 0 for q in (w["q"], w["fixed_q"])))
    return "k_real_mixed<%d,%d,%d,%d>" % (info["dim"], cm, qw, int(info.get("mixed_direct", 0)))


def profiled_traffic(workload, precision):
    """DRAM bytes per launch of the real-space kernel from the committed ncu summary, if current."""
    p = os.path.join(ROOT, "profiles", "real_%s_%s.json" % (precision, workload))
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_hash") != source_hash(REAL_SOURCES):
        return None
    return d.get("dram_bytes_per_launch")


def measured_hbm():
    """HBM copy bandwidth measured on this machine (MEASURED_PEAKS.json), else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(p))["hbm_gbs"]), "of measured (MEASURED_PEAKS.json copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "of fallback (6.8 TB/s)"


def move_roofline(info, w, W, moves_per_s, accept_frac, peaks, hbm_peak, hbm_basis):
    """Algorithmic bytes and flops of one propose + accept of one walker, and
    the fractions of HBM bandwidth and FP32 FMA rate they reach."""
    if not moves_per_s:
        return None
    n, nf, dim, ngh = w["n"], len(w["fixed_q"]), w["dim"], info["n_g_half"]
    # propose: rho(G) of the walker (the mixed path reads its FP32 leading
    # pair, 8 bytes a G) and every particle's position; accept: rho(G)
    # read-modify-write (16 bytes a G each way) and the moved position, for
    # accepted moves
    bytes_move = ngh * 8 + (n + nf) * dim * 8 + accept_frac * (2 * ngh * 16 + dim * 8)
    dim_ball = 4.0 / 3.0 * math.pi * info["r_cutoff"] ** 3 if dim == 3 else math.pi * info["r_cutoff"] ** 2
    terms = 2 * (n - 1 + nf) * dim_ball / info["volume"]      # old and new position against all others
    flop_move = terms * FLOP_REAL_TERM + 2 * ngh * FLOP_G_TERM
    gbs = bytes_move * moves_per_s / 1e9
    tf = flop_move * moves_per_s / 1e12
    return {"bytes_per_move": bytes_move, "achieved_gbs": gbs, "hbm_peak_gbs": hbm_peak,
            "hbm_frac": gbs / hbm_peak, "hbm_basis": hbm_basis, "flop_per_move": flop_move,
            "achieved_tflops": tf, "fp32_frac_of_measured": tf / peaks["fp32_tflops"]}


def de_stats(de, de_fp64, floor):
    """A form's move dE against the FP64 path's, every walker: relative to
    the walker's floor max(|E|, 1e-2 S) and to |dE| itself."""
    d = np.abs(de - de_fp64)
    rel = d / np.maximum(np.abs(de_fp64), 1e-300)
    return {"walkers": int(d.size), "abs_max_ha": float(np.max(d)), "abs_median_ha": float(np.median(d)),
            "vs_walker_floor_max": float(np.max(d / floor)),
            "vs_abs_de_mean": float(np.mean(rel)),
            "vs_abs_de_median": float(np.median(rel)), "vs_abs_de_p99": float(np.percentile(rel, 99)),
            "vs_abs_de_max": float(np.max(rel)), "frac_within_1e-6_of_abs_de": float(np.mean(rel <= 1e-6)),
            "abs_de_median_ha": float(np.median(np.abs(de_fp64)))}


def ranks_max(vals, world):
    """Element-wise maximum of per-rank timings over all ranks (host tensors:
    the process group is gloo, used for the barrier and this maximum only)."""
    if world == 1:
        return list(vals)
    import torch
    t = torch.tensor(vals, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def expected_real_terms(info, w):
    """Mean number of real-space terms per walker for uniform random displacements.

    A uniformly distributed displacement has on average V_ball(r_c)/V_cell
    lattice images inside the cutoff sphere.
    """
    dim, rc, vol = w["dim"], info["r_cutoff"], info["volume"]
    ball = 4.0 / 3.0 * math.pi * rc ** 3 if dim == 3 else math.pi * rc ** 2
    n, nf = w["n"], len(w["fixed_q"])
    return (n * (n - 1) / 2 + n * nf) * ball / vol


def workload_config(args, w, world):
    """The workload both arms report: sizes and parameters of the synthetic
    input only, so that the two lines name the same configuration."""
    return {"workload": args.workload, "walkers_per_gpu": int(w["n_walkers"]), "n_electrons": int(w["n"]),
            "n_fixed": len(w["fixed_q"]), "dim": int(w["dim"]), "alpha": float(w["alpha"]),
            "moves_per_step": args.moves, "l2": "flushed before every timed step (256 MB write)",
            "parallelism": "walker replicas, %d GPU(s)" % world}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2507_02888_gb300 import ewald, inputs

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = inputs.workload(args.workload, args.walkers or None)
    W, N, dim = w["n_walkers"], w["n"], w["dim"]
    stream = torch.cuda.Stream(device=dev)
    pos_d = torch.tensor(w["pos"], device=dev)
    rng = np.random.default_rng(1000 + rank)
    M = args.moves
    ks, disp, acc = inputs.move_stream(rng, W, N, max(M, 1), dim, w["sigma"])
    k_d = torch.tensor(ks, device=dev)
    rn_d = torch.tensor(w["pos"][np.arange(W)[None, :], ks] + disp, device=dev)
    acc_d = torch.tensor(acc, device=dev)
    e_d = torch.empty(W, dtype=torch.float64, device=dev)
    de_d = torch.empty((max(M, 1), W), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    def make(prec, **kw):
        ctx = ewald.context_for(w, precision=prec, stream=stream, **kw)
        b = ewald.Batch(ctx, W)
        b.set_positions(pos_d)
        return ctx, b

    def timed_steps(b, ctx, steps, warmup, moves, clocks=None):
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
        with torch.cuda.stream(stream):
            for s in range(warmup):
                b.energy(e_d)
                for m in range(moves):
                    b.propose(k_d[m], rn_d[m], de_d[m])
                    b.accept(acc_d[m])
            torch.cuda.synchronize()
            if world > 1:
                torch.distributed.barrier()
            ctx.timing()          # drop warm-up timers
            ctx.set_timing(True)
            if clocks:
                clocks.start()
            for s in range(steps):
                flush.fill_(float(s))            # evict the previous step's data from L2
                ev[s][0].record(stream)
                b.energy(e_d)
                ev[s][1].record(stream)
                for m in range(moves):
                    b.propose(k_d[m], rn_d[m], de_d[m])
                    b.accept(acc_d[m])
                ev[s][2].record(stream)
            torch.cuda.synchronize()
            clk = clocks.stop() if clocks else None
            if world > 1:
                torch.distributed.barrier()
        ctx.set_timing(False)
        t_e = sum(ev[s][0].elapsed_time(ev[s][1]) for s in range(steps))
        t_m = sum(ev[s][1].elapsed_time(ev[s][2]) for s in range(steps))
        return t_e, t_m, ctx.timing(), clk

    def max_over_ranks(vals):
        return ranks_max(vals, world)

    def first_round_de(b):
        """dE of every walker's first move from the workload's configuration
        (before any step: every move proposes a real displacement)."""
        with torch.cuda.stream(stream):
            b.propose(k_d[0], rn_d[0], de_d[0])
            torch.cuda.synchronize()
        return de_d[0].cpu().numpy().copy()

    # measured arithmetic peaks (a few ms, before any timed region)
    peaks = ewald.measure_peaks()
    hbm_peak, hbm_basis = measured_hbm()

    # ---- mixed precision, batched: the headline
    ctx, b = make("mixed")
    info = ctx.info()
    de0_mixed = first_round_de(b)
    props = torch.cuda.get_device_properties(dev)
    bus = ("%02x:%02x.0" % (props.pci_bus_id, props.pci_device_id)
           if isinstance(getattr(props, "pci_bus_id", None), int) else "")
    clocks = ClockSampler(bus)
    t_e, t_m, timers, clk = timed_steps(b, ctx, args.steps, args.warmup, M, clocks)
    t_e, t_m = max_over_ranks([t_e, t_m])
    # every step's moves put the same particles at the same places, so each
    # timed step evaluates the same configurations: keep them for the FP64 leg
    e_mixed = e_d.cpu().numpy().copy()
    K = args.steps
    energies_per_s = world * W * K / (t_e / 1e3)
    moves_per_s = world * W * M * K / (t_m / 1e3) if M else None
    launches = sum(n for _, n in timers.values())

    # dominant kernel: real-space pair sum
    real_ms, real_n = timers["real"]
    terms = expected_real_terms(info, w) * W
    achieved = terms * FLOP_REAL_TERM / (real_ms / real_n / 1e3) / 1e12
    peak = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    traffic = profiled_traffic(args.workload, "mixed")
    sf_ms, sf_n = timers["sfac"]
    kernel_ms = {k: round(v[0] / max(v[1], 1), 4) for k, v in timers.items() if v[1]}

    result = {
        "metric": METRIC, "value": energies_per_s, "unit": "walker energies/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": (t_e + t_m) / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": workload_config(args, w, world),
        "moves": {"value": moves_per_s, "unit": "move dE/s (propose+accept)",
                  "ms_per_round": t_m / max(K * M, 1),
                  "roofline": move_roofline(info, w, W, moves_per_s, float(np.mean(acc)), peaks, hbm_peak,
                                            hbm_basis)},
        "kernel_ms_per_launch": kernel_ms,
        "roofline": {"bound": "alu", "kernel": real_kernel_name(info, w), "precision": "mixed",
                     "r_cutoff": info["r_cutoff"], "n_g_half": info["n_g_half"], "achieved": achieved,
                     "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_basis": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (nominal)",
                     "work": "%d flop per real-space term inside r_c, %.4g terms per launch"
                             % (FLOP_REAL_TERM, terms),
                     "sfac_tflops": FLOP_G_TERM * N * info["n_g_half"] * W / (sf_ms / sf_n / 1e3) / 1e12,
                     "peak_measured": peaks["fp32_tflops"], "frac_of_measured": achieved / peaks["fp32_tflops"],
                     "peaks_measured": dict(peaks, basis="multiply-add chains, all SMs (ewald_measure_peaks)")},
        "clocks": clk, "gpu_launches": launches,
    }
    b.close()
    ctx.close()

    # ---- the mixed path at the FP64 path's real-space cutoff (erfc = 1e-16)
    # instead of its own (1e-10): the same kernels doing the extra images
    if not args.no_fp64:
        c64 = ewald.context_for(w, precision="fp64", stream=stream)
        rc16 = c64.info()["r_cutoff"]
        c64.close()
        ctx, b = make("mixed", r_cutoff=rc16)
        i16 = ctx.info()
        m_e, _, m_t, _ = timed_steps(b, ctx, 3, 1, 0)
        m_e = max_over_ranks([m_e])[0]
        r_ms, r_n = m_t["real"]
        t16 = expected_real_terms(i16, w) * W
        a16 = t16 * FLOP_REAL_TERM / (r_ms / r_n / 1e3) / 1e12
        result["mixed_at_fp64_cutoff"] = {"value": world * W * 3 / (m_e / 1e3), "unit": "walker energies/s",
                                          "r_cutoff": rc16, "real_ms_per_launch": round(r_ms / r_n, 4),
                                          "real_tflops": a16, "real_frac": a16 / peak}
        b.close()
        ctx.close()

    # ---- plain FP64 form, same workload
    if not args.no_fp64:
        ctx, b = make("fp64")
        de0_fp64 = first_round_de(b)
        fs = max(1, args.fp64_steps)
        f_e, f_m, f_t, _ = timed_steps(b, ctx, fs, 1, M)
        f_e, f_m = max_over_ranks([f_e, f_m])
        e_fp64 = e_d.cpu().numpy().copy()
        de_fp64 = de_d.cpu().numpy().copy()
        comp = b.components()
        floor = np.maximum(np.abs(comp.sum(axis=1)),
                           1e-2 * (np.abs(comp[:, 0]) + np.abs(comp[:, 2]) + np.abs(comp[:, 1] + comp[:, 3])
                                   + np.abs(comp[:, 4])))
        rel = (e_mixed - e_fp64) / floor
        result["accuracy"] = {"mixed_vs_fp64_max": float(np.max(np.abs(rel))), "mixed_vs_fp64_mean": float(np.mean(rel)),
                              "gate": 1e-6, "walkers": int(W),
                              "measure": "|E_mixed - E_fp64| / max(|E|, 1e-2 S) per walker; the FP64 path "
                                         "(cutoffs at 1e-16) is within 1e-12 of the oracle",
                              "move_de_mixed": de_stats(de0_mixed, de0_fp64, floor)}
        i64 = ctx.info()
        r64_ms, r64_n = f_t["real"]
        a64 = expected_real_terms(i64, w) * W * FLOP_REAL_TERM / (r64_ms / r64_n / 1e3) / 1e12
        result["fp64"] = {"value": world * W * fs / (f_e / 1e3), "unit": "walker energies/s",
                          "moves": world * W * M * fs / (f_m / 1e3) if M else None,
                          "steps": fs, "kernel_ms_per_launch":
                              {k: round(v[0] / max(v[1], 1), 3) for k, v in f_t.items() if v[1]},
                          "roofline": {"bound": "alu", "kernel": "k_real<double,%d>" % dim, "achieved": a64,
                                       "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                                       "frac": a64 / peaks["fp64_tflops"],
                                       "peak_basis": "measured FP64 FMA rate (ewald_measure_peaks)"}}
        result["mixed_over_fp64"] = energies_per_s / result["fp64"]["value"]
        b.close()
        ctx.close()

        # ---- tiered FP64 form: FP64 results, the real-space images below
        # erfc(alpha r) = 1e-7 in FP32 (EWALD_FP64_TIERED)
        ctx, b = make("fp64_tiered")
        de0_tiered = first_round_de(b)
        g_e, g_m, g_t, _ = timed_steps(b, ctx, fs, 1, M)
        g_e, g_m = max_over_ranks([g_e, g_m])
        rel_g = (e_d.cpu().numpy() - e_fp64) / floor
        rel_de = (de_d.cpu().numpy() - de_fp64) / floor[None, :] if M else np.zeros(1)
        result["accuracy"]["move_de_fp64_tiered"] = de_stats(de0_tiered, de0_fp64, floor)
        result["fp64_tiered"] = {"value": world * W * fs / (g_e / 1e3), "unit": "walker energies/s",
                                 "moves": world * W * M * fs / (g_m / 1e3) if M else None,
                                 "steps": fs, "vs_fp64_max": float(np.max(np.abs(rel_g))),
                                 "move_de_vs_fp64_max": float(np.max(np.abs(rel_de))), "gate": 1e-12,
                                 "kernel_ms_per_launch": {k: round(v[0] / max(v[1], 1), 3)
                                                          for k, v in g_t.items() if v[1]}}
        b.close()
        ctx.close()

        # ---- alpha balanced by measurement (ewald_tune_alpha), both forms:
        # the same energies (alpha independence) at the fastest split
        if not args.no_tune_alpha:
            tuned = {"note": "alpha from ewald_tune_alpha on a sample of the walkers; energies compared with "
                             "the FP64 path at the workload's alpha"}
            for prec, sample, steps in (("mixed", 256, 3), ("fp64", 32, 1), ("fp64_tiered", 64, 1)):
                a_t, _ = ewald.tune_alpha(dim, w["lattice"], w["q"], w["pos"][:sample],
                                          w["fixed_pos"] if len(w["fixed_q"]) else None,
                                          w["fixed_q"] if len(w["fixed_q"]) else None, alpha=w["alpha"],
                                          precision=prec, stream=stream)
                ctx, b = make(prec, alpha=a_t)
                it = ctx.info()
                # with the same moves as the other legs, so that the energies are of the
                # same (moved) configurations as e_fp64
                t_e, _, t_t, _ = timed_steps(b, ctx, steps, 1, M)
                t_e = max_over_ranks([t_e])[0]
                rel_t = (e_d.cpu().numpy() - e_fp64) / floor
                tuned[prec] = {"alpha": a_t, "alpha_over_workload": a_t / w["alpha"],
                               "value": world * W * steps / (t_e / 1e3), "unit": "walker energies/s",
                               "n_g_half": it["n_g_half"], "r_cutoff": it["r_cutoff"],
                               "kernel_ms_per_launch": {k: round(v[0] / max(v[1], 1), 3)
                                                        for k, v in t_t.items() if v[1]},
                               "vs_fp64_at_workload_alpha_max": float(np.max(np.abs(rel_t)))}
                b.close()
                ctx.close()
            result["tuned_alpha"] = tuned

    # ---- end to end through the C ABI with host buffers
    if not args.no_e2e:
        ctx = ewald.context_for(w, precision="mixed", stream=stream)
        b = ewald.Batch(ctx, W)
        keep = []

        def pinned(a):
            # page-locked host copy (the library copies such arrays by DMA)
            t = torch.empty(a.shape, dtype=getattr(torch, str(a.dtype)), pin_memory=True)
            keep.append(t)
            t.numpy()[...] = a
            return t.numpy()

        pos_h = pinned(np.ascontiguousarray(w["pos"]))
        pos_t = keep[-1]                     # the same page-locked positions as a tensor
        ks_h, rn_h = pinned(np.ascontiguousarray(ks)), pinned(np.ascontiguousarray(rn_d.cpu().numpy()))
        acc_h = pinned(np.ascontiguousarray(acc))
        e_h, de_h = pinned(np.zeros(W)), pinned(np.zeros(W))
        e_steps = max(2, K // 2)

        def moves():
            for m in range(M):
                b.propose(ks_h[m], rn_h[m], de_h)
                b.accept(acc_h[m])

        # serial: each step uploads its positions, then computes
        for _ in range(2):
            b.set_positions(pos_h)
            b.energy(e_h)
        if world > 1:
            torch.distributed.barrier()
        te_serial = 0.0
        for s in range(e_steps):
            t0 = time.perf_counter()
            b.set_positions(pos_h)
            b.energy(e_h)
            te_serial += time.perf_counter() - t0
            moves()

        # pipelined: step s + 1's positions go up from page-locked memory on a
        # copy stream into one of two device buffers while step s computes;
        # the batch takes them from that buffer (device to device, on its own
        # stream) once the copy has landed.  Every step still uploads its
        # positions and reads its energies back inside the timed region.
        cstream = torch.cuda.Stream(device=dev)
        stage = [torch.empty_like(pos_d) for _ in range(2)]
        copied = [torch.cuda.Event() for _ in range(2)]
        consumed = [torch.cuda.Event() for _ in range(2)]
        for i in range(2):
            consumed[i].record(stream)

        def upload(i):
            cstream.wait_event(consumed[i])  # the buffer's previous positions are in the batch
            with torch.cuda.stream(cstream):
                stage[i].copy_(pos_t, non_blocking=True)
                copied[i].record(cstream)

        def energy_step(s):
            i = s % 2
            stream.wait_event(copied[i])
            b.set_positions(stage[i])
            consumed[i].record(stream)
            upload(1 - i)                    # the next step's positions, under this step's energy
            b.energy(e_h)                    # read back to page-locked memory (synchronises)

        upload(0)
        for s in range(2):
            energy_step(s)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        te = tm = 0.0
        t_prev = time.perf_counter()
        upload(0)                            # the first step's positions, inside the timed region
        for s in range(e_steps):
            energy_step(s)
            t1 = time.perf_counter()
            te += t1 - t_prev
            moves()
            t_prev = time.perf_counter()
            tm += t_prev - t1
        torch.cuda.synchronize()             # the last prefetch (not a step's input) settles untimed
        te, tm, te_serial = max_over_ranks([te, tm, te_serial])
        result["e2e"] = {"value": world * W * e_steps / te, "unit": "walker energies/s",
                         "h2d_bytes_per_step": W * N * dim * 8 + M * W * (4 + dim * 8 + 1),
                         "d2h_bytes_per_step": W * 8 + M * W * 8,
                         "moves": world * W * M * e_steps / tm if M else None,
                         "serial_value": world * W * e_steps / te_serial,
                         "note": "positions uploaded from page-locked host memory and energies and dE read "
                                 "back to it, every step; the next step's upload overlaps this step's energy "
                                 "(serial_value: upload, then compute)"}
        b.close()
        ctx.close()

    # ---- batched form (uneven systems in one persistent launch) and serving form
    if not args.no_configs:
        result["configs"] = run_configs(stream)
    if not args.no_jastrow:
        result["jastrow_p"] = run_jastrow(stream, args.workload)
        result["jastrow_u"] = run_jastrow_u(stream, args.workload)
    if not args.no_batched:
        result["batched"] = run_batched(stream, 5)
    if not args.no_serving:
        sv = run_serving(stream, "mixed", args.serve_requests)
        sv["fp64"] = run_serving(stream, "fp64", args.serve_requests_fp64)
        sv["fp64_tiered"] = run_serving(stream, "fp64_tiered", args.serve_requests_tiered)
        result["serving"] = sv

    # ---- the numbers that qualify the headline, on the object of the line
    # that carries the measurement (roofline)
    rf = result["roofline"]
    mv = result["moves"]["roofline"]
    if mv:
        rf["moves"] = {"bound": "hbm", "kernels": "k_propose + k_accept", "achieved": mv["achieved_gbs"],
                       "peak": hbm_peak, "unit": "GB/s", "frac": mv["hbm_frac"], "peak_basis": hbm_basis,
                       "bytes_per_move": mv["bytes_per_move"], "moves_per_s": moves_per_s,
                       "fp32_frac_of_measured": mv["fp32_frac_of_measured"]}
    if "mixed_at_fp64_cutoff" in result and "fp64" in result:
        eq = result["mixed_at_fp64_cutoff"]
        rf["equal_cutoff"] = {"mixed_value": eq["value"], "fp64_value": result["fp64"]["value"],
                              "mixed_over_fp64": eq["value"] / result["fp64"]["value"],
                              "real_frac": eq["real_frac"], "r_cutoff": eq["r_cutoff"],
                              "unit": "walker energies/s", "note": "both forms at erfc(alpha r_c) = 1e-16"}
    if "accuracy" in result:
        a = result["accuracy"]
        acc_cfg = {"energy_mixed_vs_fp64_max": a["mixed_vs_fp64_max"], "gate": a["gate"],
                   "measure": "relative to max(|E|, 1e-2 S) per walker, all walkers"}
        for key in ("move_de_mixed", "move_de_fp64_tiered"):
            if key in a:
                acc_cfg[key] = {k: a[key][k] for k in ("vs_walker_floor_max", "vs_abs_de_median", "vs_abs_de_p99",
                                                      "vs_abs_de_max", "abs_max_ha")}
        if "fp64_tiered" in result:
            acc_cfg["energy_fp64_tiered_vs_fp64_max"] = result["fp64_tiered"]["vs_fp64_max"]
        rf["accuracy"] = acc_cfg

    # ---- CPU oracle on the host cores (rank 0 only)
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        import oracle
        rc16, gc16 = oracle.cutoffs(w["dim"], w["alpha"])   # the definition's cutoffs
        result["cpu_baseline"] = cpu_oracle_rate(w, rc16, gc16, args.cpu_seconds)
    return result


def run_batched(stream, steps):
    """Batched form: the bulk-solid cell (diamond, 864 e + 216 ions, 1024
    walkers) with the 3D electron gas at N = 1024 (fcc, 4096 walkers) in one
    persistent launch per energy call, tilings autotuned; against the same
    walkers as one energy launch sequence per batch."""
    import torch
    from paper_2507_02888_gb300 import ewald, inputs
    ws = [inputs.workload("diamond_3x3x3"), inputs.workload("heg3d_fcc_n1024")]
    ctxs = [ewald.context_for(w, precision="mixed", stream=stream) for w in ws]
    bs = []
    tune = []
    for c, w in zip(ctxs, ws):
        b = ewald.Batch(c, w["n_walkers"])
        b.set_positions(w["pos"])
        tune.append(b.autotune())
        bs.append(b)
    m = ewald.Multi(bs)
    Wt = sum(b.W for b in bs)
    out = torch.empty(Wt, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(stream):
        for _ in range(2):
            m.energy(out)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        ev[0].record(stream)
        for _ in range(steps):
            m.energy(out)
        ev[1].record(stream)
        torch.cuda.synchronize()
        t_multi = ev[0].elapsed_time(ev[1])
        # the same walkers, one energy launch sequence per batch
        ev[0].record(stream)
        for _ in range(steps):
            for b in bs:
                b.energy(out[:b.W])
        ev[1].record(stream)
        torch.cuda.synchronize()
        t_sep = ev[0].elapsed_time(ev[1])
    m.close()
    return {"value": Wt * steps / (t_multi / 1e3), "unit": "walker energies/s",
            "workload": "diamond_3x3x3 (W=1024) + heg3d_fcc_n1024 (W=4096), one persistent launch",
            "separate_batches": Wt * steps / (t_sep / 1e3), "steps": steps,
            "tiling": [{"pair_tile": t["pair_tile"], "subcell_bits": t["subcell_bits"]} for t in tune]}


def run_configs(stream, steps=3, moves=4):
    """The other single-system workloads at their own sizes (with the 2D
    electron-hole bilayer, charges at two heights), each in both
    precisions: walker energies/s, move dE/s (propose + accept rounds) and the
    mixed path's per-walker error against the FP64 path (floor as in the
    tests).  Device-resident inputs; every step re-evaluates the same
    configurations (each round's moves put the same particles at the same
    places)."""
    import torch
    from paper_2507_02888_gb300 import ewald, inputs
    out = {}
    for name in ["heg3d_sc_n54", "heg2d_hex_n338", "diamond_3x3x3", "ehbilayer2d_hex_n338"]:
        w = inputs.workload(name)
        W, N, dim = w["n_walkers"], w["n"], w["dim"]
        rng = np.random.default_rng(77)
        ks, disp, acc = inputs.move_stream(rng, W, N, moves, dim, w["sigma"])
        k_d = torch.tensor(ks, device="cuda")
        rn_d = torch.tensor(w["pos"][np.arange(W)[None, :], ks] + disp, device="cuda")
        acc_d = torch.tensor(acc, device="cuda")
        pos_d = torch.tensor(w["pos"], device="cuda")
        e_d = torch.empty(W, dtype=torch.float64, device="cuda")
        de_d = torch.empty(W, dtype=torch.float64, device="cuda")
        row, energies = {"walkers": W, "n": N, "n_fixed": len(w["fixed_q"]), "dim": dim}, {}
        if "z" in w:
            row["layers"] = int(len(set(w["z"])))
        for prec in ("mixed", "fp64"):
            ctx = ewald.context_for(w, precision=prec, stream=stream)
            b = ewald.Batch(ctx, W)
            b.set_positions(pos_d)
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            with torch.cuda.stream(stream):
                for _ in range(2):                      # warm-up, and the moved configuration
                    b.energy(e_d)
                    for m in range(moves):
                        b.propose(k_d[m], rn_d[m], de_d)
                        b.accept(acc_d[m])
                ev[0].record(stream)
                for _ in range(steps):
                    b.energy(e_d)
                ev[1].record(stream)
                for _ in range(steps):
                    for m in range(moves):
                        b.propose(k_d[m], rn_d[m], de_d)
                        b.accept(acc_d[m])
                ev[2].record(stream)
                torch.cuda.synchronize()
            comp = b.components()
            energies[prec] = (e_d.cpu().numpy().copy(), comp)
            row[prec] = {"walker_energies_per_s": W * steps / (ev[0].elapsed_time(ev[1]) / 1e3),
                         "move_de_per_s": W * moves * steps / (ev[1].elapsed_time(ev[2]) / 1e3),
                         "r_cutoff": ctx.info()["r_cutoff"]}
            b.close()
            ctx.close()
        em, (ef, cf) = energies["mixed"][0], energies["fp64"]
        floor = np.maximum(np.abs(cf.sum(axis=1)),
                           1e-2 * (np.abs(cf[:, 0]) + np.abs(cf[:, 2]) + np.abs(cf[:, 1] + cf[:, 3]) + np.abs(cf[:, 4])))
        rel = (em - ef) / floor
        row["mixed_vs_fp64"] = {"max": float(np.max(np.abs(rel))), "mean": float(np.mean(rel))}
        out[name] = row
    return out


def run_jastrow(stream, workload, n_stars=8, steps=3):
    """Two-body plane-wave Jastrow term p (Sec. 2.3, Eq. (9)) of every walker
    with gradients and Laplacians, both precisions: walker evaluations/s and
    phase evaluations/s (each (electron, G) phase is evaluated twice: once for
    rho(G), once for the electron's derivatives)."""
    import torch
    from paper_2507_02888_gb300 import ewald, inputs
    w = inputs.workload(workload)
    W, N, dim = w["n_walkers"], w["n"], w["dim"]
    a = 0.2 * (-0.4) ** np.arange(n_stars)
    pos_d = torch.tensor(w["pos"], device="cuda")
    j = torch.empty(W, dtype=torch.float64, device="cuda")
    g = torch.empty((W, N, dim), dtype=torch.float64, device="cuda")
    lap = torch.empty((W, N), dtype=torch.float64, device="cuda")
    out = {"workload": workload, "walkers": W, "n_stars": n_stars}
    for prec in ("mixed", "fp64"):
        ctx = ewald.context_for(w, precision=prec, stream=stream)
        n_g = ctx.set_jastrow_p(a)
        b = ewald.Batch(ctx, W)
        b.set_positions(pos_d)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        with torch.cuda.stream(stream):
            b.jastrow_p(j, g, lap)
            ev[0].record(stream)
            for _ in range(steps):
                b.jastrow_p(j, g, lap)
            ev[1].record(stream)
            torch.cuda.synchronize()
        t = ev[0].elapsed_time(ev[1]) / 1e3
        out[prec] = {"walker_evaluations_per_s": W * steps / t, "n_g_half": n_g,
                     "phase_evaluations_per_s": 2.0 * W * N * n_g * steps / t}
        b.close()
        ctx.close()
    return out


def run_jastrow_u(stream, workload, C=3, steps=3):
    """Polynomial two-body Jastrow term u (Sec. 2.3, Eq. (8)) of every walker
    with gradients and Laplacians, both precisions: walker evaluations/s and
    pairs/s (every unordered pair is visited once; those inside L_u are
    evaluated).  L_u = 0.99 of half the shortest lattice vector, N_u = 8, half
    the electrons spin up."""
    import itertools
    import torch
    from paper_2507_02888_gb300 import ewald, inputs
    w = inputs.workload(workload)
    W, N, dim = w["n_walkers"], w["n"], w["dim"]
    lat = np.asarray(w["lattice"])
    L = 0.99 * min(np.linalg.norm(np.array(m) @ lat)
                   for m in itertools.product(range(-2, 3), repeat=dim) if any(m)) / 2
    b_like = [0.3, 0.0, -0.2, 0.4, 0.1, -0.2, 0.3, -0.1, 0.05]
    b_unlike = [0.55, 0.0, 0.3, -0.6, 0.5, 0.1, -0.1, 0.05, -0.02]
    al = [c / L ** (l + C) for l, c in enumerate(b_like)]
    au = [c / L ** (l + C) for l, c in enumerate(b_unlike)]
    pos_d = torch.tensor(w["pos"], device="cuda")
    j = torch.empty(W, dtype=torch.float64, device="cuda")
    g = torch.empty((W, N, dim), dtype=torch.float64, device="cuda")
    lap = torch.empty((W, N), dtype=torch.float64, device="cuda")
    out = {"workload": workload, "walkers": W, "L_u": L, "C": C, "N_u": len(b_like) - 1}
    for prec in ("mixed", "fp64"):
        ctx = ewald.context_for(w, precision=prec, stream=stream)
        ctx.set_jastrow_u(N // 2, L, C, al, au)
        b = ewald.Batch(ctx, W)
        b.set_positions(pos_d)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        n_steps = steps if prec == "mixed" else 1
        with torch.cuda.stream(stream):
            b.jastrow_u(j, g, lap)
            ev[0].record(stream)
            for _ in range(n_steps):
                b.jastrow_u(j, g, lap)
            ev[1].record(stream)
            torch.cuda.synchronize()
        t = ev[0].elapsed_time(ev[1]) / 1e3
        out[prec] = {"walker_evaluations_per_s": W * n_steps / t,
                     "pairs_per_s": float(W) * N * (N - 1) / 2 * n_steps / t}
        b.close()
        ctx.close()
    return out


SERVE_SYSTEMS = ["heg3d_sc_n54", "heg3d_sc_n128", "heg2d_hex_n338", "heg3d_sc_n512", "heg3d_fcc_n1024",
                 "diamond_3x3x3"]


def run_serving(stream, precision, n_requests, seed=4242):
    """Serving form: Poisson stream of requests over the six systems of the mix,
    W ~ U{1..512} walkers, M ~ U{1..200} moves, rate 0.8 x the saturated rate."""
    from paper_2507_02888_gb300 import ewald, inputs, serve
    rng = np.random.default_rng(seed)
    ws = {}
    for name in SERVE_SYSTEMS:
        w = inputs.workload(name, 512)
        ws[name] = (ewald.context_for(w, precision=precision, stream=stream), w["pos"], w["sigma"])

    def make(n, rate):
        reqs, t = [], 0.0
        for i in range(n):
            name = SERVE_SYSTEMS[rng.integers(len(SERVE_SYSTEMS))]
            ctx, pos, sigma = ws[name]
            W, M = int(rng.integers(1, 513)), int(rng.integers(1, 201))
            t = 0.0 if rate is None else t + rng.exponential(1.0 / rate)
            reqs.append((t, ctx, pos[:W], M, sigma, int(rng.integers(1, 2 ** 62))))
        return reqs

    srv = serve.Server(precision, max_walkers=16384)
    sat = serve.run_stream(srv, make(max(20, n_requests // 8), None))
    sat_rate = len(sat["results"]) / sat["elapsed_s"]
    lam = 0.8 * sat_rate
    res = serve.run_stream(srv, make(n_requests, lam))
    srv.close()
    lat = np.asarray(res["latency_ms"])
    return {"moves_per_s": res["moves"] / res["elapsed_s"], "unit": "walker moves/s (propose+accept)",
            "p50_ms": res["p50_ms"], "p99_ms": res["p99_ms"], "requests": n_requests,
            "latencies_above_p99": int(np.sum(lat > res["p99_ms"])),
            "arrival_rate_per_s": lam, "saturated_moves_per_s": sat["moves"] / sat["elapsed_s"],
            "saturated_requests_per_s": sat_rate, "elapsed_s": res["elapsed_s"]}


def run_reference(args, rank, world):
    """The oracle as the reference arm: walker energies/s on the host cores."""
    from paper_2507_02888_gb300 import inputs
    import oracle
    if rank != 0:
        return None
    w = inputs.workload(args.workload, args.walkers or None)
    rc, gc = oracle.cutoffs(w["dim"], w["alpha"])
    oracle.build()
    cores = host_cores()
    per_step = cores
    for s in range(args.warmup):
        oracle_walker_energies(w, [s % w["n_walkers"]], rc, gc, 1)
    t = 0.0
    for s in range(args.steps):
        walkers = [(s * per_step + i) % w["n_walkers"] for i in range(per_step)]
        t0 = time.perf_counter()
        oracle_walker_energies(w, walkers, rc, gc, cores)
        t += time.perf_counter() - t0
    value = per_step * args.steps / t
    return {"metric": METRIC, "value": value, "unit": "walker energies/s", "impl": "reference",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, w, world),
            "cpu_baseline": {"value": value, "unit": "walker energies/s", "cores": cores, "kind": "oracle",
                             "sample": "%d walkers per step of %s on %d host threads" % (per_step, w["name"], cores)},
            "e2e": {"value": value, "unit": "walker energies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")   # host-side barrier and timing max only
    if args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, rank, world, local_rank)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
