"""ctypes loader for the plain FP64 Ewald oracle (TEST INFRASTRUCTURE).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never imports it and
the oracle imports nothing from the GPU library.

Functions follow the paper's Sec. 2.2, Eqs. (2)-(6) (``energy_z`` and
``delta_e_z``: 2D cells with charges at heights z != 0), and for the two-body
plane-wave Jastrow term Sec. 2.3, Eqs. (7) and (9), and for the polynomial
two-body term Eq. (8); see ``ewald_oracle.c`` for
the formulas.  Every call takes positions as a ``(n, dim)`` float64 array
of Cartesian coordinates and charges as an ``(n,)`` float64 array.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ewald_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

ERRORS = {0: "ok", 1: "bad argument", 2: "bad lattice", 3: "coincident particles"}


class OracleError(RuntimeError):
    pass


def build(force=False):
    """Compile the oracle with gcc (plain -O2, IEEE arithmetic, libm)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            c_int, c_double = ctypes.c_int, ctypes.c_double
            lib.oracle_energy.argtypes = [c_int, dp, c_int, dp, dp, c_double, c_double, c_double, dp, dp]
            lib.oracle_delta_e.argtypes = [c_int, dp, c_int, dp, dp, c_int, dp, c_double, c_double,
                                           c_double, dp]
            lib.oracle_delta_e_parts.argtypes = [c_int, dp, c_int, dp, dp, c_int, dp, c_double, c_double,
                                                 c_double, dp, dp]
            lib.oracle_rho_at.argtypes = [c_int, dp, c_int, dp, dp, c_int, ip, dp]
            lib.oracle_recip_pairsum.argtypes = [c_int, dp, c_int, dp, dp, c_double, c_double, dp]
            lib.oracle_gcount.argtypes = [c_int, dp, c_double]
            lib.oracle_gcount.restype = ctypes.c_long
            lib.oracle_cutoffs.argtypes = [c_int, c_double, c_double, dp, dp]
            lib.oracle_jastrow_stars.argtypes = [c_int, dp, c_int, c_int, ip, ip, ip]
            lib.oracle_jastrow_p.argtypes = [c_int, dp, c_int, dp, c_int, dp, dp, dp, dp]
            lib.oracle_energy_z.argtypes = [dp, c_int, dp, dp, dp, c_double, c_double, c_double, dp, dp]
            lib.oracle_delta_e_z.argtypes = [dp, c_int, dp, dp, dp, c_int, dp, c_double, c_double, c_double, dp]
            lib.oracle_energy_z.restype = ctypes.c_int
            lib.oracle_delta_e_z.restype = ctypes.c_int
            lib.oracle_jastrow_u.argtypes = [c_int, dp, c_int, dp, c_int, c_double, c_int, c_int, dp, dp, dp, dp,
                                             dp]
            lib.oracle_jastrow_u.restype = ctypes.c_int
            lib.oracle_jastrow_stars.restype = ctypes.c_int
            lib.oracle_jastrow_p.restype = ctypes.c_int
            for f in (lib.oracle_energy, lib.oracle_delta_e, lib.oracle_delta_e_parts, lib.oracle_rho_at,
                      lib.oracle_recip_pairsum, lib.oracle_cutoffs):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _check(st):
    if st != 0:
        raise OracleError(ERRORS.get(st, "error %d" % st))


def cutoffs(dim, alpha, tol=1e-16):
    """(r_c, g_c): erfc(alpha r_c) = tol; exp(-g_c^2/4alpha^2) = tol (3D) or erfc(g_c/2alpha) = tol (2D)."""
    rc, gc = ctypes.c_double(), ctypes.c_double()
    _check(_load().oracle_cutoffs(dim, alpha, tol, ctypes.byref(rc), ctypes.byref(gc)))
    return rc.value, gc.value


def energy(dim, lattice, pos, q, alpha, r_c, g_c):
    """Return (E, components) with components = [E_real, E_madR, E_recip, E_self, E_bg]."""
    lat = _f64(lattice, (dim, dim))
    pos = _f64(pos)
    n = pos.shape[0]
    pos = pos.reshape(n, dim)
    q = _f64(q, (n,))
    comp = np.zeros(5)
    e = ctypes.c_double()
    _check(_load().oracle_energy(dim, _dp(lat), n, _dp(pos), _dp(q), alpha, r_c, g_c, _dp(comp),
                                 ctypes.byref(e)))
    return e.value, comp


def delta_e(dim, lattice, pos, q, k, r_new, alpha, r_c, g_c):
    """Energy change when particle k moves to r_new (direct definition)."""
    lat = _f64(lattice, (dim, dim))
    pos = _f64(pos)
    n = pos.shape[0]
    pos = pos.reshape(n, dim)
    q = _f64(q, (n,))
    rn = _f64(r_new, (dim,))
    de = ctypes.c_double()
    _check(_load().oracle_delta_e(dim, _dp(lat), n, _dp(pos), _dp(q), int(k), _dp(rn), alpha, r_c,
                                  g_c, ctypes.byref(de)))
    return de.value


def delta_e_parts(dim, lattice, pos, q, k, r_new, alpha, r_c, g_c):
    """(dE_real, dE_recip): the real-space and reciprocal-space parts of delta_e."""
    lat = _f64(lattice, (dim, dim))
    pos = _f64(pos)
    n = pos.shape[0]
    pos = pos.reshape(n, dim)
    q = _f64(q, (n,))
    rn = _f64(r_new, (dim,))
    dr, dk = ctypes.c_double(), ctypes.c_double()
    _check(_load().oracle_delta_e_parts(dim, _dp(lat), n, _dp(pos), _dp(q), int(k), _dp(rn), alpha, r_c,
                                        g_c, ctypes.byref(dr), ctypes.byref(dk)))
    return dr.value, dk.value


def rho_at(dim, lattice, pos, q, nvec):
    """rho(G) = sum_i q_i exp(i G.r_i) at integer reciprocal coordinates nvec (n_g, dim)."""
    lat = _f64(lattice, (dim, dim))
    pos = _f64(pos)
    n = pos.shape[0]
    pos = pos.reshape(n, dim)
    q = _f64(q, (n,))
    nv = np.ascontiguousarray(np.asarray(nvec, dtype=np.int32).reshape(-1, dim))
    out = np.zeros((nv.shape[0], 2))
    _check(_load().oracle_rho_at(dim, _dp(lat), n, _dp(pos), _dp(q), nv.shape[0],
                                 nv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(out)))
    return out[:, 0] + 1j * out[:, 1]


def recip_pairsum(dim, lattice, pos, q, alpha, g_c):
    """E_recip written as sum_G f(G) sum_{i,j} q_i q_j cos(G.(r_i-r_j)) times the prefactor."""
    lat = _f64(lattice, (dim, dim))
    pos = _f64(pos)
    n = pos.shape[0]
    pos = pos.reshape(n, dim)
    q = _f64(q, (n,))
    e = ctypes.c_double()
    _check(_load().oracle_recip_pairsum(dim, _dp(lat), n, _dp(pos), _dp(q), alpha, g_c,
                                        ctypes.byref(e)))
    return e.value


def gcount(dim, lattice, g_c):
    """Number of G != 0 with |G| <= g_c, counting +G and -G."""
    lat = _f64(lattice, (dim, dim))
    return int(_load().oracle_gcount(dim, _dp(lat), g_c))


def jastrow_stars(dim, lattice, n_stars):
    """Every G of the first n_stars shells of equal |G| (both signs):
    (nvec (n_g, dim) integer reciprocal coordinates, star (n_g,) shell index)."""
    lat = _f64(lattice, (dim, dim))
    n_g = ctypes.c_int()
    ip = ctypes.POINTER(ctypes.c_int)
    _check(_load().oracle_jastrow_stars(dim, _dp(lat), int(n_stars), 0, ctypes.byref(n_g), None, None))
    nv = np.zeros((n_g.value, dim), dtype=np.int32)
    st = np.zeros(n_g.value, dtype=np.int32)
    _check(_load().oracle_jastrow_stars(dim, _dp(lat), int(n_stars), n_g.value, ctypes.byref(n_g),
                                        nv.ctypes.data_as(ip), st.ctypes.data_as(ip)))
    return nv, st


def jastrow_p(dim, lattice, pos, a):
    """J_p = sum_{i<j} p(r_i - r_j) with p(r) = sum_m a_m sum_{G in star m, one of +-G} cos(G.r),
    and its gradient (n, dim) and Laplacian (n,) with respect to each particle."""
    lat = _f64(lattice, (dim, dim))
    pos = _f64(pos)
    n = pos.shape[0]
    pos = pos.reshape(n, dim)
    a = _f64(a).reshape(-1)
    j = ctypes.c_double()
    grad = np.zeros((n, dim))
    lap = np.zeros(n)
    _check(_load().oracle_jastrow_p(dim, _dp(lat), n, _dp(pos), a.size, _dp(a), ctypes.byref(j), _dp(grad),
                                    _dp(lap)))
    return j.value, grad, lap


def energy_z(lattice, pos, z, q, alpha, r_c, g_c):
    """2D cell, charges at in-plane positions pos (n, 2) and heights z (n,):
    (E, [E_real, E_madR, E_recip, E_self, E_bg]) from the pair definition."""
    lat = _f64(lattice, (2, 2))
    pos = _f64(pos)
    n = pos.shape[0]
    pos = pos.reshape(n, 2)
    z = _f64(z, (n,))
    q = _f64(q, (n,))
    comp = np.zeros(5)
    e = ctypes.c_double()
    _check(_load().oracle_energy_z(_dp(lat), n, _dp(pos), _dp(z), _dp(q), alpha, r_c, g_c, _dp(comp),
                                   ctypes.byref(e)))
    return e.value, comp


def delta_e_z(lattice, pos, z, q, k, r_new, alpha, r_c, g_c):
    """Energy change when particle k moves in the plane to r_new (height unchanged)."""
    lat = _f64(lattice, (2, 2))
    pos = _f64(pos)
    n = pos.shape[0]
    pos = pos.reshape(n, 2)
    z = _f64(z, (n,))
    q = _f64(q, (n,))
    rn = _f64(r_new, (2,))
    de = ctypes.c_double()
    _check(_load().oracle_delta_e_z(_dp(lat), n, _dp(pos), _dp(z), _dp(q), int(k), _dp(rn), alpha, r_c, g_c,
                                    ctypes.byref(de)))
    return de.value


def jastrow_u(dim, lattice, pos, n_up, L, C, alpha_like, alpha_unlike):
    """J_u = sum_{i<j} u(r_ij), u(r) = (r - L)^C sum_l alpha_l r^l (r < L), nearest images, like /
    unlike spin coefficients (particles < n_up spin up); alpha[1] is replaced by its cusp value.
    Returns (J_u, gradient (n, dim), Laplacian (n,))."""
    lat = _f64(lattice, (dim, dim))
    pos = _f64(pos)
    n = pos.shape[0]
    pos = pos.reshape(n, dim)
    al = _f64(alpha_like).reshape(-1)
    au = _f64(alpha_unlike).reshape(-1)
    if al.size != au.size:
        raise ValueError("coefficient sets of different length")
    j = ctypes.c_double()
    grad = np.zeros((n, dim))
    lap = np.zeros(n)
    _check(_load().oracle_jastrow_u(dim, _dp(lat), n, _dp(pos), int(n_up), float(L), int(C), al.size - 1, _dp(al),
                                    _dp(au), ctypes.byref(j), _dp(grad), _dp(lap)))
    return j.value, grad, lap
