"""Thin binding of the serving entry points (ewald_server_* in include/ewald.h)
and a host loop that feeds a Poisson stream of requests to a server.

The request loop itself - admission by walker slots and device memory,
one persistent launch per step for every active request, retirement - runs
in the library; this module only submits requests at their arrival times,
calls step() and collects results and latencies.
"""
import ctypes
import time

import numpy as np

from . import ewald

_vp, _c_int, _c_double = ctypes.c_void_p, ctypes.c_int, ctypes.c_double

SIGNATURES = [
    ("ewald_server_create", _c_int, [_c_int, _c_int, _c_double, _vp, ctypes.POINTER(_vp)]),
    ("ewald_server_destroy", None, [_vp]),
    ("ewald_server_submit", _c_int, [_vp, _vp, _vp, _c_int, _c_int, _c_double, _c_double,
                                     ctypes.c_ulonglong, ctypes.POINTER(_c_int)]),
    ("ewald_server_step", _c_int, [_vp, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int)]),
    ("ewald_server_result", _c_int, [_vp, _c_int, _vp, _vp, ctypes.POINTER(_c_double)]),
    ("ewald_server_completed", _c_int, [_vp, _vp, _c_int, ctypes.POINTER(_c_int)]),
    ("ewald_server_drain", _c_int, [_vp]),
    ("ewald_server_cancel", _c_int, [_vp, _c_int]),
    ("ewald_server_request_bytes", _c_int, [_vp, _c_int, ctypes.POINTER(_c_double)]),
    ("ewald_server_error_message", ctypes.c_char_p, [_vp]),
]
_bound = False


def _lib():
    global _bound
    lib = ewald.load()
    if not _bound:
        for name, res, args in SIGNATURES:
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _bound = True
    return lib


class Server:
    def __init__(self, precision="mixed", max_walkers=65536, hbm_budget_bytes=0.0, stream=None):
        lib = _lib()
        prec = {"fp64": ewald.EWALD_FP64, "mixed": ewald.EWALD_MIXED,
                "fp64_tiered": ewald.EWALD_FP64_TIERED}[precision]
        h = _vp()
        st = None if stream is None else _vp(stream if isinstance(stream, int) else stream.cuda_stream)
        code = lib.ewald_server_create(prec, int(max_walkers), float(hbm_budget_bytes), st, ctypes.byref(h))
        if code:
            raise ewald.EwaldError(code, "server create")
        self._h = h
        self._W = {}
        self.contexts = []      # keep the contexts alive as long as the server

    def _check(self, code):
        if code:
            raise ewald.EwaldError(code, _lib().ewald_server_error_message(self._h).decode())

    def submit(self, ctx, pos, n_steps, sigma=0.3, accept_prob=0.5, seed=0):
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64))
        W = pos.shape[0]
        rid = _c_int()
        self.contexts.append(ctx)
        self._check(_lib().ewald_server_submit(self._h, ctx._h, _vp(pos.ctypes.data), W, int(n_steps), float(sigma),
                                               float(accept_prob), int(seed) & (2 ** 64 - 1), ctypes.byref(rid)))
        self._W[rid.value] = W
        return rid.value

    def step(self):
        a, q = _c_int(), _c_int()
        self._check(_lib().ewald_server_step(self._h, ctypes.byref(a), ctypes.byref(q)))
        return a.value, q.value

    def completed(self, max_ids=4096):
        """Ids of the requests that finished since the last call."""
        ids = np.zeros(max_ids, dtype=np.int32)
        n = _c_int()
        self._check(_lib().ewald_server_completed(self._h, _vp(ids.ctypes.data), max_ids, ctypes.byref(n)))
        return ids[:n.value].tolist()

    def result(self, rid):
        """(energies [W], accepted [W], latency ms) once done, else None."""
        W = self._W[rid]
        e = np.zeros(W)
        n = np.zeros(W, dtype=np.int32)
        lat = _c_double()
        code = _lib().ewald_server_result(self._h, rid, _vp(e.ctypes.data), _vp(n.ctypes.data), ctypes.byref(lat))
        if code == 8:
            return None
        self._check(code)
        return e, n, lat.value

    def cancel(self, rid):
        """Cancel a queued or active request (ewald_server_cancel)."""
        self._check(_lib().ewald_server_cancel(self._h, int(rid)))

    def drain(self):
        self._check(_lib().ewald_server_drain(self._h))

    def close(self):
        if getattr(self, "_h", None):
            _lib().ewald_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def request_bytes(ctx, n_walkers):
    """Device bytes a request of n_walkers walkers of ctx counts against a server's budget."""
    b = _c_double()
    code = _lib().ewald_server_request_bytes(ctx._h, int(n_walkers), ctypes.byref(b))
    if code:
        raise ewald.EwaldError(code, "request bytes")
    return b.value


def run_stream(server, requests, time_limit=600.0):
    """Drive a request stream: requests = [(t_arrival_s, ctx, pos, n_steps, sigma, seed)].

    Requests are submitted when the wall clock passes their arrival time;
    step() runs whenever work is active or queued.  Returns a dict with the
    per-request results, latencies (ms), total walker-moves and elapsed time.
    """
    order = sorted(range(len(requests)), key=lambda i: requests[i][0])
    ids, done, lat, by_id = {}, {}, {}, {}
    pending = set()
    t0 = time.perf_counter()
    nxt = 0
    moves = sum(np.asarray(r[2]).shape[0] * r[3] for r in requests)
    while len(done) < len(requests):
        now = time.perf_counter() - t0
        if now > time_limit:
            raise TimeoutError("request stream did not finish in %.0f s" % time_limit)
        while nxt < len(order) and requests[order[nxt]][0] <= now:
            t, ctx, pos, steps, sigma, seed = requests[order[nxt]]
            ids[order[nxt]] = server.submit(ctx, pos, steps, sigma, 0.5, seed)
            by_id[ids[order[nxt]]] = order[nxt]
            pending.add(order[nxt])
            nxt += 1
        active, queued = server.step()
        for rid in server.completed():
            i = by_id.get(rid)
            if i is None:
                continue
            r = server.result(rid)
            done[i] = r
            lat[i] = r[2]
            pending.discard(i)
        if not active and not queued and nxt < len(order):
            time.sleep(max(0.0, min(0.001, requests[order[nxt]][0] - (time.perf_counter() - t0))))
    server.drain()
    elapsed = time.perf_counter() - t0
    l = np.array([lat[i] for i in range(len(requests))])
    return {"results": [done[i] for i in range(len(requests))], "latency_ms": l, "moves": moves,
            "elapsed_s": elapsed, "p50_ms": float(np.percentile(l, 50)), "p99_ms": float(np.percentile(l, 99))}
