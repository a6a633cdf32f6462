"""Thin ctypes binding of libewald_gb300.so (C ABI in include/ewald.h).

This module only marshals arguments: every step of the computation runs in
the library's CUDA kernels.  Arrays may be NumPy arrays (host memory) or
CUDA torch tensors (device memory, passed by pointer with on_device=1 and
accessed on the context's stream).  The library must be built
(``paper_2507_02888_gb300.build``); loading fails loudly when it is not.
"""
import atexit
import ctypes
import os
import weakref

import numpy as np

from . import build as _build

EWALD_FP64, EWALD_MIXED, EWALD_FP64_TIERED = 0, 1, 2
PRECISIONS = {"fp64": EWALD_FP64, "mixed": EWALD_MIXED, "fp64_tiered": EWALD_FP64_TIERED}
ERR_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_LATTICE", 3: "ERR_COINCIDENT", 4: "ERR_NO_PROPOSAL",
             5: "ERR_OOM", 6: "ERR_CUDA", 7: "ERR_TIMEOUT", 8: "ERR_STATE", 9: "ERR_CANCELLED"}

_c_int, _c_double, _vp = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)


class EwaldError(RuntimeError):
    def __init__(self, code, what=""):
        self.code = code
        super().__init__("%s (%d)%s" % (ERR_NAMES.get(code, "?"), code, (": " + what) if what else ""))


class Desc(ctypes.Structure):
    _fields_ = [("dim", _c_int), ("lattice", _dp), ("n_mobile", _c_int), ("mobile_charge", _dp),
                ("n_fixed", _c_int), ("fixed_pos", _dp), ("fixed_charge", _dp), ("gamma", _c_double),
                ("g_cutoff", _c_double), ("r_cutoff", _c_double), ("precision", _c_int),
                ("resum_every", _c_int), ("mobile_z", _dp), ("fixed_z", _dp)]


class TuneResult(ctypes.Structure):
    _fields_ = [("pair_tile", _c_int), ("subcell_bits", _c_int), ("ms", _c_double), ("n_tried", _c_int),
                ("from_cache", _c_int), ("real_threads", _c_int), ("sfac_chunks", _c_int), ("sfac_ms", _c_double)]


class Info(ctypes.Structure):
    _fields_ = [("dim", _c_int), ("n_mobile", _c_int), ("n_fixed", _c_int), ("precision", _c_int),
                ("alpha", _c_double), ("r_cutoff", _c_double), ("g_cutoff", _c_double),
                ("volume", _c_double), ("n_g_half", _c_int), ("n_images", _c_int),
                ("subcell_bits", _c_int), ("pair_tile", _c_int), ("max_candidates", _c_int), ("n_runs", _c_int),
                ("run_len", _c_int), ("e_madelung", _c_double), ("e_self", _c_double),
                ("e_background", _c_double), ("e_fixed_real", _c_double), ("n_layers", _c_int),
                ("mixed_direct", _c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_live_batches = weakref.WeakSet()
_live_contexts = weakref.WeakSet()
_live_multis = weakref.WeakSet()


@atexit.register
def _close_all():
    """Free library objects while the CUDA runtime is still up (interpreter exit)."""
    for m in list(_live_multis):
        m.close()
    for b in list(_live_batches):
        b.close()
    for c in list(_live_contexts):
        c.close()

# (name, restype, argtypes) of every entry point declared in include/ewald.h
SIGNATURES = [
    ("ewald_create", _c_int, [ctypes.POINTER(Desc), _vp, ctypes.POINTER(_vp)]),
    ("ewald_destroy", None, [_vp]),
    ("ewald_get_info", _c_int, [_vp, ctypes.POINTER(Info)]),
    ("ewald_plan", _c_int, [ctypes.POINTER(Desc), ctypes.POINTER(Info)]),
    ("ewald_get_gvectors", _c_int, [_vp, _vp]),
    ("ewald_last_error", _c_int, [_vp]),
    ("ewald_strerror", ctypes.c_char_p, [_c_int]),
    ("ewald_last_error_message", ctypes.c_char_p, [_vp]),
    ("ewald_batch_create", _c_int, [_vp, _c_int, ctypes.POINTER(_vp)]),
    ("ewald_batch_destroy", None, [_vp]),
    ("ewald_batch_set_positions", _c_int, [_vp, _vp, _c_int]),
    ("ewald_batch_get_positions", _c_int, [_vp, _vp, _c_int]),
    ("ewald_batch_sync", _c_int, [_vp]),
    ("ewald_energy", _c_int, [_vp, _vp, _c_int]),
    ("ewald_energy_components", _c_int, [_vp, _vp, _c_int]),
    ("ewald_propose_move", _c_int, [_vp, _vp, _vp, _vp, _c_int]),
    ("ewald_accept_move", _c_int, [_vp, _vp, _c_int]),
    ("ewald_resum", _c_int, [_vp]),
    ("ewald_batch_get_rho", _c_int, [_vp, _vp, _c_int]),
    ("ewald_multi_create", _c_int, [_vp, _c_int, ctypes.POINTER(_vp)]),
    ("ewald_multi_energy", _c_int, [_vp, _vp, _c_int]),
    ("ewald_multi_destroy", None, [_vp]),
    ("ewald_autotune", _c_int, [_vp, ctypes.c_char_p, _vp]),
    ("ewald_set_timing", _c_int, [_vp, _c_int]),
    ("ewald_get_timing", _c_int, [_vp, _vp, _vp]),
    ("ewald_measure_peaks", _c_int, [_vp, _vp, _vp]),
    ("ewald_pair_terms", _c_int, [_c_int, _vp, _c_double, _vp, _vp]),
    ("ewald_pair_terms_df", _c_int, [_c_int, _vp, _c_double, _vp]),
    ("ewald_jastrow_p_set", _c_int, [_vp, _c_int, _vp]),
    ("ewald_jastrow_p_count", _c_int, [_vp, ctypes.POINTER(_c_int)]),
    ("ewald_jastrow_p", _c_int, [_vp, _vp, _vp, _vp, _c_int]),
    ("ewald_jastrow_u_set", _c_int, [_vp, _c_int, _c_double, _c_int, _c_int, _vp, _vp]),
    ("ewald_jastrow_u", _c_int, [_vp, _vp, _vp, _vp, _c_int]),
    ("ewald_tune_alpha", _c_int, [_vp, _vp, _c_int, _vp, _vp, _vp]),
    ("ewald_build_flags", _c_int, []),
]

KERNELS = ["ingest", "sfac", "real", "combine", "propose", "accept", "resum"]


def library_path():
    """The release library, or the debug one (kernels check their indices)
    when the environment sets EWALD_LIBRARY=debug."""
    return _build.LIB_DEBUG if os.environ.get("EWALD_LIBRARY") == "debug" else _build.LIB


def load(build_if_missing=True):
    """Load the shared library (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if build_if_missing and not _build.up_to_date(path):
        _build.build_variants(("debug",) if path == _build.LIB_DEBUG else ("release",))
    if not os.path.exists(path):
        raise ImportError("%s is not built; run python -m paper_2507_02888_gb300.build" % os.path.basename(path))
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def build_flags():
    """EWALD_BUILD_* bits of the loaded library (1: the debug build)."""
    return int(load().ewald_build_flags())


def _check(code, ctx=None):
    if code != 0:
        what = _lib.ewald_strerror(code).decode()
        if ctx is not None and getattr(ctx, "_h", None):
            what += " - " + _lib.ewald_last_error_message(ctx._h).decode()
        raise EwaldError(code, what)


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _is_dev(x):
    return hasattr(x, "is_cuda") and x.is_cuda


def _ptr(x):
    """(pointer, on_device) of a NumPy array or a CUDA torch tensor."""
    if _is_dev(x):
        if not x.is_contiguous():
            raise ValueError("device tensors must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), 1
    if not x.flags["C_CONTIGUOUS"]:
        raise ValueError("host arrays must be C-contiguous")
    return ctypes.c_void_p(x.ctypes.data), 0


def _desc(dim, lattice, mobile_charge, fixed_pos=None, fixed_charge=None, alpha=0.0, g_cutoff=0.0, r_cutoff=0.0,
          precision="fp64", resum_every=0, mobile_z=None, fixed_z=None):
    """An ewald_desc and the arrays it points into (keep them alive while it is used)."""
    dim = int(dim)
    lat = _f64(lattice, dim * dim)
    qm = _f64(mobile_charge)
    nf = 0 if fixed_charge is None else len(fixed_charge)
    fp = _f64(fixed_pos if nf else np.zeros(1))
    fq = _f64(fixed_charge if nf else np.zeros(1))
    prec = PRECISIONS.get(precision, precision)
    # heights of a layered 2D cell (None: every particle in the plane)
    zm = None if mobile_z is None else _f64(mobile_z)
    zf = None if fixed_z is None or nf == 0 else _f64(fixed_z)
    d = Desc(dim, lat.ctypes.data_as(_dp), len(qm), qm.ctypes.data_as(_dp), nf, fp.ctypes.data_as(_dp),
             fq.ctypes.data_as(_dp), float(alpha), float(g_cutoff), float(r_cutoff), int(prec), int(resum_every),
             None if zm is None else zm.ctypes.data_as(_dp), None if zf is None else zf.ctypes.data_as(_dp))
    return d, (lat, qm, fp, fq, zm, zf)


def plan(dim, lattice, mobile_charge, fixed_pos=None, fixed_charge=None, alpha=0.0, g_cutoff=0.0, r_cutoff=0.0,
         precision="fp64", resum_every=0, mobile_z=None, fixed_z=None):
    """ewald_plan: the info dict a context of this description would report,
    from the host set-up alone (no GPU needed)."""
    lib = load()
    d, keep = _desc(dim, lattice, mobile_charge, fixed_pos, fixed_charge, alpha, g_cutoff, r_cutoff, precision,
                    resum_every, mobile_z, fixed_z)
    i = Info()
    _check(lib.ewald_plan(ctypes.byref(d), ctypes.byref(i)))
    del keep
    return i.as_dict()


def plan_for(workload, precision="fp64", **kw):
    """ewald_plan for a workload dict from paper_2507_02888_gb300.inputs."""
    w = workload
    if "z" in w and "mobile_z" not in kw:
        kw["mobile_z"] = w["z"]
        if len(w["fixed_q"]) and "fixed_z" in w:
            kw["fixed_z"] = w["fixed_z"]
    alpha = kw.pop("alpha", w["alpha"])
    nf = len(w["fixed_q"])
    return plan(w["dim"], w["lattice"], w["q"], w["fixed_pos"] if nf else None, w["fixed_q"] if nf else None,
                alpha=alpha, precision=precision, **kw)


class Context:
    """One periodic system: cell, charges, alpha, cutoffs and precision."""

    def __init__(self, dim, lattice, mobile_charge, fixed_pos=None, fixed_charge=None, alpha=0.0,
                 g_cutoff=0.0, r_cutoff=0.0, precision="fp64", resum_every=0, stream=None, mobile_z=None,
                 fixed_z=None):
        lib = load()
        self.dim = int(dim)
        d, keep = _desc(dim, lattice, mobile_charge, fixed_pos, fixed_charge, alpha, g_cutoff, r_cutoff,
                        precision, resum_every, mobile_z, fixed_z)
        self._lat, self._qm, self._fp, self._fq, self._zm, self._zf = keep
        nf = 0 if fixed_charge is None else len(fixed_charge)
        prec = PRECISIONS.get(precision, precision)
        h = _vp()
        if stream is None:
            st = None
        elif isinstance(stream, int):
            st = _vp(stream)
        else:
            st = _vp(stream.cuda_stream)
        _check(lib.ewald_create(ctypes.byref(d), st, ctypes.byref(h)))
        self._h = h
        _live_contexts.add(self)
        self.n_mobile = len(self._qm)
        self.n_fixed = nf
        self.precision = prec

    def info(self):
        i = Info()
        _check(_lib.ewald_get_info(self._h, ctypes.byref(i)))
        return i.as_dict()

    def gvectors(self):
        n = self.info()["n_g_half"]
        out = np.zeros((n, self.dim), dtype=np.int32)
        _check(_lib.ewald_get_gvectors(self._h, ctypes.c_void_p(out.ctypes.data)))
        return out

    def set_jastrow_p(self, a):
        """Stars of the two-body plane-wave Jastrow term with coefficients a[n_stars];
        returns the number of G vectors kept (one of each +-G pair)."""
        a = _f64(a)
        _check(_lib.ewald_jastrow_p_set(self._h, a.size, ctypes.c_void_p(a.ctypes.data)), self)
        n = _c_int()
        _check(_lib.ewald_jastrow_p_count(self._h, ctypes.byref(n)), self)
        return n.value

    def set_jastrow_u(self, n_up, L_u, C, alpha_like, alpha_unlike):
        """Polynomial two-body Jastrow term: cutoff L_u, order C at the cutoff,
        coefficients alpha_l (l = 0..N_u) for like and unlike spins; alpha[1]
        is set by the cusp condition.  Mobile particles below n_up are spin up."""
        al, au = _f64(alpha_like), _f64(alpha_unlike)
        if al.size != au.size:
            raise ValueError("coefficient sets of different length")
        _check(_lib.ewald_jastrow_u_set(self._h, int(n_up), float(L_u), int(C), al.size - 1,
                                        ctypes.c_void_p(al.ctypes.data), ctypes.c_void_p(au.ctypes.data)), self)

    def set_timing(self, enable=True):
        _check(_lib.ewald_set_timing(self._h, int(bool(enable))))

    def timing(self):
        """{kernel: (device ms, launches)} accumulated since the last call."""
        ms = np.zeros(len(KERNELS))
        n = np.zeros(len(KERNELS), dtype=np.int64)
        _check(_lib.ewald_get_timing(self._h, ctypes.c_void_p(ms.ctypes.data), ctypes.c_void_p(n.ctypes.data)))
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNELS)}

    def last_error(self):
        return _lib.ewald_last_error(self._h)

    def close(self):
        if getattr(self, "_h", None):
            _lib.ewald_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """W walkers of a Context with device-resident positions and rho(G)."""

    def __init__(self, ctx, n_walkers):
        self.ctx = ctx
        self.W = int(n_walkers)
        h = _vp()
        _check(_lib.ewald_batch_create(ctx._h, self.W, ctypes.byref(h)), ctx)
        self._h = h
        _live_batches.add(self)

    # -- positions
    def set_positions(self, pos):
        if not _is_dev(pos):
            pos = _f64(pos, self.W * self.ctx.n_mobile * self.ctx.dim)
        p, dev = _ptr(pos)
        _check(_lib.ewald_batch_set_positions(self._h, p, dev), self.ctx)

    def get_positions(self, out=None):
        if out is None:
            out = np.zeros((self.W, self.ctx.n_mobile, self.ctx.dim))
        p, dev = _ptr(out)
        _check(_lib.ewald_batch_get_positions(self._h, p, dev), self.ctx)
        return out

    # -- energies
    def energy(self, out=None):
        if out is None:
            out = np.zeros(self.W)
        p, dev = _ptr(out)
        _check(_lib.ewald_energy(self._h, p, dev), self.ctx)
        return out

    def components(self, out=None):
        if out is None:
            out = np.zeros((self.W, 5))
        p, dev = _ptr(out)
        _check(_lib.ewald_energy_components(self._h, p, dev), self.ctx)
        return out

    # -- moves
    def propose(self, k, r_new, out=None):
        if _is_dev(k):
            if out is None:
                import torch
                out = torch.empty(self.W, dtype=torch.float64, device=k.device)
        else:
            k = np.ascontiguousarray(np.asarray(k, dtype=np.int32))
            r_new = _f64(r_new, self.W * self.ctx.dim)
            if out is None:
                out = np.zeros(self.W)
        pk, dev = _ptr(k)
        pr, _ = _ptr(r_new)
        po, _ = _ptr(out)
        _check(_lib.ewald_propose_move(self._h, pk, pr, po, dev), self.ctx)
        return out

    def accept(self, accept):
        if not _is_dev(accept):
            accept = np.ascontiguousarray(np.asarray(accept, dtype=np.uint8))
        p, dev = _ptr(accept)
        _check(_lib.ewald_accept_move(self._h, p, dev), self.ctx)

    def resum(self):
        _check(_lib.ewald_resum(self._h), self.ctx)

    def rho(self, out=None):
        """rho(G) [W][n_layers][n_g_half][2] (the layer axis has length 1 unless the cell is layered)."""
        inf = self.ctx.info()
        n = inf["n_g_half"]
        if out is None:
            out = np.zeros((self.W, inf["n_layers"], n, 2))
        p, dev = _ptr(out)
        _check(_lib.ewald_batch_get_rho(self._h, p, dev), self.ctx)
        return out

    def jastrow_p(self, j=None, grad=None, lap=None, derivatives=True):
        """J_p per walker and (derivatives=True) its gradient [W][N][dim] and
        Laplacian [W][N] per electron; host arrays unless device tensors are given."""
        N, dim = self.ctx.n_mobile, self.ctx.dim
        if j is None:
            j = np.zeros(self.W)
            if derivatives:
                grad, lap = np.zeros((self.W, N, dim)), np.zeros((self.W, N))
        pj, dev = _ptr(j)
        pg = _ptr(grad)[0] if grad is not None else None
        pl = _ptr(lap)[0] if lap is not None else None
        _check(_lib.ewald_jastrow_p(self._h, pj, pg, pl, dev), self.ctx)
        return j, grad, lap

    def jastrow_u(self, j=None, grad=None, lap=None, derivatives=True):
        """J_u per walker and (derivatives=True) its gradient [W][N][dim] and
        Laplacian [W][N] per particle; host arrays unless device tensors are given."""
        N, dim = self.ctx.n_mobile, self.ctx.dim
        if j is None:
            j = np.zeros(self.W)
            if derivatives:
                grad, lap = np.zeros((self.W, N, dim)), np.zeros((self.W, N))
        pj, dev = _ptr(j)
        pg = _ptr(grad)[0] if grad is not None else None
        pl = _ptr(lap)[0] if lap is not None else None
        _check(_lib.ewald_jastrow_u(self._h, pj, pg, pl, dev), self.ctx)
        return j, grad, lap

    def sync(self):
        _check(_lib.ewald_batch_sync(self._h), self.ctx)

    def autotune(self, cache_path=None):
        """Pick the fastest real-space tiling for this batch's system (see ewald_autotune)."""
        r = TuneResult()
        _check(_lib.ewald_autotune(self._h, cache_path.encode() if cache_path else None,
                                   ctypes.byref(r)))
        return {k: getattr(r, k) for k, _ in r._fields_}

    def close(self):
        if getattr(self, "_h", None):
            _lib.ewald_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multi:
    """Batches of different systems evaluated by one persistent launch (graph-replayed)."""

    def __init__(self, batches):
        self.batches = list(batches)
        arr = (_vp * len(self.batches))(*[b._h for b in self.batches])
        h = _vp()
        _check(_lib.ewald_multi_create(arr, len(self.batches), ctypes.byref(h)), self.batches[0].ctx)
        self._h = h
        self.W = sum(b.W for b in self.batches)
        _live_multis.add(self)

    def energy(self, out=None):
        """Energies of every walker, batches concatenated in order."""
        if out is None:
            out = np.zeros(self.W)
        p, dev = _ptr(out)
        _check(_lib.ewald_multi_energy(self._h, p, dev), self.batches[0].ctx)
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.ewald_multi_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_peaks():
    """Measured FP32 FMA and FP64 FMA TFLOP/s and rsqrt Tops/s of the current GPU."""
    load()
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(_lib.ewald_measure_peaks(ctypes.addressof(a), ctypes.addressof(b), ctypes.addressof(c)))
    return {"fp32_tflops": a.value, "fp64_tflops": b.value, "rsqrt_tops": c.value}


def pair_terms(r2, alpha):
    """The FP32 term erfc(alpha r)/r for float32 r^2 values on the GPU: (scalar, paired) float32 arrays."""
    load()
    r2 = np.ascontiguousarray(r2, dtype=np.float32)
    sc = np.empty_like(r2)
    pa = np.empty_like(r2)
    _check(_lib.ewald_pair_terms(int(r2.size), r2.ctypes.data, float(alpha), sc.ctypes.data, pa.ctypes.data))
    return sc, pa


def pair_terms_df(r2, alpha):
    """The tiered form's double-float erfc(alpha r)/r for FP64 r^2 values on the GPU, as FP64."""
    load()
    r2 = np.ascontiguousarray(r2, dtype=np.float64)
    out = np.empty_like(r2)
    _check(_lib.ewald_pair_terms_df(int(r2.size), r2.ctypes.data, float(alpha), out.ctypes.data))
    return out


def tune_alpha(dim, lattice, mobile_charge, pos, fixed_pos=None, fixed_charge=None, alpha=0.0, precision="fp64",
               stream=None, mobile_z=None, fixed_z=None):
    """Fastest splitting parameter for this system and precision, timed on the
    sample configurations pos [W][N][dim] (host): (alpha, microseconds per walker)."""
    lib = load()
    lat = _f64(lattice, int(dim) * int(dim))
    qm = _f64(mobile_charge)
    nf = 0 if fixed_charge is None else len(fixed_charge)
    fp = _f64(fixed_pos if nf else np.zeros(1))
    fq = _f64(fixed_charge if nf else np.zeros(1))
    zm = None if mobile_z is None else _f64(mobile_z)
    zf = None if fixed_z is None or nf == 0 else _f64(fixed_z)
    prec = PRECISIONS.get(precision, precision)
    d = Desc(int(dim), lat.ctypes.data_as(_dp), len(qm), qm.ctypes.data_as(_dp), nf, fp.ctypes.data_as(_dp),
             fq.ctypes.data_as(_dp), float(alpha), 0.0, 0.0, int(prec), 0,
             None if zm is None else zm.ctypes.data_as(_dp), None if zf is None else zf.ctypes.data_as(_dp))
    p = _f64(pos)
    W = p.size // (len(qm) * int(dim))
    st = None if stream is None else (_vp(stream) if isinstance(stream, int) else _vp(stream.cuda_stream))
    a, us = ctypes.c_double(), ctypes.c_double()
    _check(lib.ewald_tune_alpha(ctypes.byref(d), st, W, ctypes.c_void_p(p.ctypes.data), ctypes.byref(a),
                                ctypes.byref(us)))
    return a.value, us.value


def context_for(workload, precision="fp64", stream=None, **kw):
    """Context for a workload dict from paper_2507_02888_gb300.inputs."""
    w = workload
    if "z" in w and "mobile_z" not in kw:
        kw["mobile_z"] = w["z"]
        if len(w["fixed_q"]) and "fixed_z" in w:
            kw["fixed_z"] = w["fixed_z"]
    alpha = kw.pop("alpha", w["alpha"])
    return Context(w["dim"], w["lattice"], w["q"], w["fixed_pos"] if len(w["fixed_q"]) else None,
                   w["fixed_q"] if len(w["fixed_q"]) else None, alpha=alpha, precision=precision,
                   stream=stream, **kw)
