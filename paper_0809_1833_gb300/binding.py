"""Thin ctypes binding of ``libmpgb.so`` (declared in ``include/mpgb.h``).

Functions keep the C names and only marshal arguments: pointers are passed
as integers (``tensor.data_ptr()`` for device memory), streams as
``torch.cuda.Stream.cuda_stream`` integers.  Every step of the decode runs
in the library's CUDA kernels; there is no Python or CPU fallback, and
``lib()`` raises if the library is missing.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libmpgb.so")

# status codes
MP_OK = 0
MP_PENDING = 1
MP_ERR_INVALID = -1
MP_ERR_NOMEM = -2
MP_ERR_BUSY = -3
MP_ERR_TIMEOUT = -4
MP_ERR_NONFINITE = -5
MP_ERR_CUDA = -6
MP_ERR_UNSUPPORTED = -7
MP_ERR_NOT_FOUND = -8

MP_PREC_FP32, MP_PREC_BF16, MP_PREC_FP8E4M3, MP_PREC_FP64 = 0, 1, 2, 3
MP_LAYOUT_ATOM_MAJOR, MP_LAYOUT_ROW_MAJOR = 0, 1
MP_STOP_CONVERGED, MP_STOP_MAX_ITERS, MP_STOP_ZERO_Y, MP_STOP_RANK = 0, 1, 2, 3

MP_OPT_PLAIN_MODE = 1
MP_OPT_WATCHDOG_NS = 2
MP_OPT_DEBUG_SKIP_ARRIVE = 3
MP_OPT_GRID_CTAS = 4
MP_OPT_BATCH_TILE_N = 5
MP_OPT_PLAIN_PREFETCH = 6
MP_OPT_PLAIN_STAGE_BYTES = 8
MP_OPT_PLAIN_EVICT_FIRST = 9
MP_OPT_BATCH_AUTOTUNE = 10
MP_OPT_PLAIN_GRAM = 11
MP_OPT_PLAIN_L2_KEEP_BYTES = 12
MP_OPT_BATCH_TILE_M = 13
MP_OPT_BATCH_GRAM = 14
MP_OPT_BATCH_PAIR = 15
MP_OPT_BATCH_GRAM_BELOW = 16
MP_Q_BATCH_TILE_N = 10
MP_Q_BATCH_TILE_M = 17
MP_Q_BATCH_GRAM = 19
MP_Q_BATCH_PAIR = 20
MP_Q_BATCH_GRAM_BELOW = 21

MP_Q_PLAIN_MODE = 1
MP_Q_PLAIN_CTAS = 2
MP_Q_PLAIN_THREADS = 3
MP_Q_PLAIN_SMEM = 4
MP_Q_PLAIN_STAGE_ATOMS = 5
MP_Q_PLAIN_STAGES = 6
MP_Q_LD_FP32 = 7
MP_Q_DEVICE_BYTES = 8
MP_Q_KERNEL_LAUNCHES = 9
MP_Q_PLAIN64_MODE = 12
MP_Q_PLAIN64_STAGES = 13
MP_Q_PLAIN64_PIECES = 18
MP_Q_GRAM_BYTES = 14
MP_Q_PLAN_N = 15
MP_Q_PLAN_M = 16


class mp_plan_desc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("M", ctypes.c_int), ("layout", ctypes.c_int),
                ("prec_mask", ctypes.c_uint), ("normalize", ctypes.c_int), ("reserved", ctypes.c_int)]


class mp_stop(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("max_iters", ctypes.c_int), ("reserved", ctypes.c_int)]


class mp_result(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("stop_reason", ctypes.c_int), ("status", ctypes.c_int),
                ("reserved", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("energy_audit_max", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class mp_trace(ctypes.Structure):
    _fields_ = [("atoms", ctypes.c_void_p), ("coefs", ctypes.c_void_p), ("energies", ctypes.c_void_p),
                ("residual", ctypes.c_void_p), ("capacity", ctypes.c_int), ("reserved", ctypes.c_int)]


class mp_trace_f64(ctypes.Structure):
    _fields_ = mp_trace._fields_


class mp_shard_state(ctypes.Structure):
    _fields_ = [("e0", ctypes.c_double), ("e", ctypes.c_double), ("thr2", ctypes.c_double),
                ("audit", ctypes.c_double), ("t", ctypes.c_int), ("T", ctypes.c_int), ("stopped", ctypes.c_int),
                ("stop_reason", ctypes.c_int), ("status", ctypes.c_int), ("reserved", ctypes.c_int)]


class mp_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("rejected", ctypes.c_longlong), ("admitted", ctypes.c_longlong),
                ("completed", ctypes.c_longlong), ("queued", ctypes.c_longlong), ("active", ctypes.c_longlong),
                ("latency_p50_s", ctypes.c_double), ("latency_p99_s", ctypes.c_double),
                ("latency_mean_s", ctypes.c_double), ("latency_max_s", ctypes.c_double),
                ("hbm_bytes", ctypes.c_size_t), ("chunks", ctypes.c_longlong), ("retired", ctypes.c_longlong)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class MpError(RuntimeError):
    def __init__(self, status, where, message):
        super().__init__(f"{where}: {status_name(status)}: {message}")
        self.status = status


_P = ctypes.c_void_p
_I = ctypes.c_int
# name -> (restype, argtypes); the same list is the set of exported symbols
# the header declares.
SIGNATURES = {
    "mp_status_string": (ctypes.c_char_p, [_I]),
    "mp_last_error_message": (ctypes.c_char_p, []),
    "mp_plan_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(mp_plan_desc), _P, _P]),
    "mp_plan_destroy": (_I, [_P]),
    "mp_plan_set_option": (_I, [_P, _I, ctypes.c_longlong]),
    "mp_plan_query": (_I, [_P, _I, ctypes.POINTER(ctypes.c_longlong)]),
    "mp_recover": (_I, [_P, _P, _P, ctypes.POINTER(mp_stop), ctypes.POINTER(mp_trace),
                        ctypes.POINTER(mp_result), _P]),
    "mp_recover_omp": (_I, [_P, _P, _P, ctypes.POINTER(mp_stop), ctypes.POINTER(mp_trace),
                            ctypes.POINTER(mp_result), _P]),
    "mp_plan_create_f64": (_I, [ctypes.POINTER(_P), ctypes.POINTER(mp_plan_desc), _P, _P]),
    "mp_recover_f64": (_I, [_P, _P, _P, ctypes.POINTER(mp_stop), ctypes.POINTER(mp_trace_f64),
                            ctypes.POINTER(mp_result), _P]),
    "mp_plan_last_result": (_I, [_P, ctypes.POINTER(mp_result)]),
    "mp_recover_host": (_I, [_P, _P, _P, ctypes.POINTER(mp_stop), ctypes.POINTER(mp_result)]),
    "mp_recover_batched": (_I, [_P, _I, _P, _P, _I, ctypes.POINTER(mp_stop), _I,
                                ctypes.POINTER(mp_trace), ctypes.POINTER(mp_result), _P]),
    "mp_debug_correlations": (_I, [_P, _I, _P, _I, _P, _P]),
    "mp_debug_time_gemm": (_I, [_P, _I, _I, _I, _I, _I, ctypes.POINTER(ctypes.c_double)]),
    "mp_debug_time_gemm_pair": (_I, [_P, _I, _I, _I, _I, _I, _I, ctypes.POINTER(ctypes.c_double)]),
    "mp_plan_autotune": (_I, [_P, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "mp_plan_autotune_shape": (_I, [_P, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "mp_recover_noalloc": (_I, [_P, _I, _I, _I, _P, _P, ctypes.POINTER(mp_stop), ctypes.POINTER(mp_trace),
                               ctypes.POINTER(mp_result), _P]),
    "mp_shard_record_bytes": (ctypes.c_size_t, [_P]),
    "mp_shard_init": (_I, [_P, _P, _P, _P, ctypes.POINTER(mp_stop), _P, _P]),
    "mp_shard_step_local": (_I, [_P, _I, _P, _P, _P]),
    "mp_shard_step_apply": (_I, [_P, _I, _P, _I, _P, _P, _P, ctypes.POINTER(mp_trace), _P]),
    "mp_server_create": (_I, [ctypes.POINTER(_P), ctypes.c_size_t, _I, _I]),
    "mp_server_add_dictionary": (_I, [_P, _P, _I, ctypes.POINTER(_I)]),
    "mp_server_dictionary_slots": (_I, [_P, _I, ctypes.POINTER(_I)]),
    "mp_server_submit": (_I, [_P, _I, _P, ctypes.POINTER(mp_stop), ctypes.POINTER(ctypes.c_uint64)]),
    "mp_server_poll": (_I, [_P, ctypes.c_uint64, _P, ctypes.POINTER(mp_result)]),
    "mp_server_get_stats": (_I, [_P, ctypes.POINTER(mp_server_stats)]),
    "mp_server_reset_stats": (_I, [_P]),
    "mp_server_destroy": (_I, [_P]),
}

_LIB = None


def lib():
    """Load libmpgb.so (built by ``build.build()``); raises if it is missing."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run __graft_entry__.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def status_name(s):
    return lib().mp_status_string(int(s)).decode()


def last_error():
    return lib().mp_last_error_message().decode()


def check(status, where):
    if status < 0:
        raise MpError(status, where, last_error())
    return status


def _stream(stream):
    if stream is None:
        return None
    return int(getattr(stream, "cuda_stream", stream)) or None


# ---------------------------------------------------------------- wrappers

def mp_plan_create(N, M, psi_ptr, layout=MP_LAYOUT_ATOM_MAJOR, prec_mask=0, normalize=False,
                   stream=None):
    """Returns a plan handle (int); raises MpError on failure."""
    d = mp_plan_desc(int(N), int(M), int(layout), int(prec_mask), 1 if normalize else 0, 0)
    h = ctypes.c_void_p()
    check(lib().mp_plan_create(ctypes.byref(h), ctypes.byref(d), ctypes.c_void_p(int(psi_ptr)),
                               _stream(stream)), "mp_plan_create")
    return h.value


def mp_plan_create_f64(N, M, psi_ptr, layout=MP_LAYOUT_ATOM_MAJOR, prec_mask=1 << MP_PREC_FP64,
                       normalize=False, stream=None):
    """Plan from an FP64 dictionary (device pointer to N*M doubles)."""
    d = mp_plan_desc(int(N), int(M), int(layout), int(prec_mask), 1 if normalize else 0, 0)
    h = ctypes.c_void_p()
    check(lib().mp_plan_create_f64(ctypes.byref(h), ctypes.byref(d), ctypes.c_void_p(int(psi_ptr)),
                                   _stream(stream)), "mp_plan_create_f64")
    return h.value


def mp_plan_destroy(plan):
    return check(lib().mp_plan_destroy(plan), "mp_plan_destroy")


def mp_plan_set_option(plan, option, value):
    return check(lib().mp_plan_set_option(plan, int(option), int(value)), "mp_plan_set_option")


def mp_plan_query(plan, what):
    v = ctypes.c_longlong()
    check(lib().mp_plan_query(plan, int(what), ctypes.byref(v)), "mp_plan_query")
    return v.value


def make_trace(atoms_ptr=0, coefs_ptr=0, energies_ptr=0, capacity=0, residual_ptr=0):
    return mp_trace(atoms_ptr or None, coefs_ptr or None, energies_ptr or None, residual_ptr or None,
                    int(capacity), 0)


def mp_recover(plan, y_ptr, x_ptr, eps, max_iters, trace=None, sync=True, stream=None,
               raise_on_error=True):
    """Decode one signal (device pointers).  With ``sync`` returns
    (status, mp_result); otherwise (status, None) right after enqueueing."""
    st = mp_stop(float(eps), int(max_iters), 0)
    res = mp_result()
    s = lib().mp_recover(plan, ctypes.c_void_p(int(y_ptr)), ctypes.c_void_p(int(x_ptr)), ctypes.byref(st),
                         ctypes.byref(trace) if trace is not None else None,
                         ctypes.byref(res) if sync else None, _stream(stream))
    if raise_on_error:
        check(s, "mp_recover")
    return s, (res if sync else None)


def mp_recover_omp(plan, y_ptr, x_ptr, eps, max_iters, trace=None, sync=True, stream=None,
                   raise_on_error=True):
    """OMP decode of one signal (device pointers); returns as mp_recover."""
    st = mp_stop(float(eps), int(max_iters), 0)
    res = mp_result()
    s = lib().mp_recover_omp(plan, ctypes.c_void_p(int(y_ptr)), ctypes.c_void_p(int(x_ptr)), ctypes.byref(st),
                             ctypes.byref(trace) if trace is not None else None,
                             ctypes.byref(res) if sync else None, _stream(stream))
    if raise_on_error:
        check(s, "mp_recover_omp")
    return s, (res if sync else None)


def make_trace_f64(atoms_ptr=0, coefs_ptr=0, energies_ptr=0, capacity=0, residual_ptr=0):
    return mp_trace_f64(atoms_ptr or None, coefs_ptr or None, energies_ptr or None, residual_ptr or None,
                        int(capacity), 0)


def mp_recover_f64(plan, y_ptr, x_ptr, eps, max_iters, trace=None, sync=True, stream=None,
                   raise_on_error=True):
    """FP64 decode of one signal (device pointers to doubles); returns as mp_recover."""
    st = mp_stop(float(eps), int(max_iters), 0)
    res = mp_result()
    s = lib().mp_recover_f64(plan, ctypes.c_void_p(int(y_ptr)), ctypes.c_void_p(int(x_ptr)), ctypes.byref(st),
                             ctypes.byref(trace) if trace is not None else None,
                             ctypes.byref(res) if sync else None, _stream(stream))
    if raise_on_error:
        check(s, "mp_recover_f64")
    return s, (res if sync else None)


def mp_plan_last_result(plan, raise_on_error=True):
    res = mp_result()
    s = lib().mp_plan_last_result(plan, ctypes.byref(res))
    if raise_on_error:
        check(s, "mp_plan_last_result")
    return s, res


def mp_recover_host(plan, y_host, x_host, eps, max_iters, raise_on_error=True):
    """Host-buffer decode: y_host / x_host are contiguous float32 numpy arrays."""
    st = mp_stop(float(eps), int(max_iters), 0)
    res = mp_result()
    s = lib().mp_recover_host(plan, ctypes.c_void_p(y_host.ctypes.data), ctypes.c_void_p(x_host.ctypes.data),
                              ctypes.byref(st), ctypes.byref(res))
    if raise_on_error:
        check(s, "mp_recover_host")
    return s, res


def mp_recover_batched(plan, prec, Y_ptr, X_ptr, B, stops, trace=None, stream=None, raise_on_error=True):
    """Batched decode; ``stops`` is one (eps, T) pair or a list of B pairs.
    Returns (status, list of mp_result)."""
    if isinstance(stops, tuple):
        stops = [stops]
    arr = (mp_stop * len(stops))(*[mp_stop(float(e), int(t), 0) for e, t in stops])
    res = (mp_result * max(int(B), 1))()
    s = lib().mp_recover_batched(plan, int(prec), ctypes.c_void_p(int(Y_ptr)), ctypes.c_void_p(int(X_ptr)),
                                 int(B), arr, len(stops), ctypes.byref(trace) if trace is not None else None,
                                 res, _stream(stream))
    if raise_on_error:
        check(s, "mp_recover_batched")
    return s, list(res)[:int(B)]


def mp_plan_autotune(plan, prec, B):
    """Returns the (atoms per tile, signals per tile) the autotuner picked."""
    tn, tm = ctypes.c_int(), ctypes.c_int()
    check(lib().mp_plan_autotune(plan, int(prec), int(B), ctypes.byref(tn), ctypes.byref(tm)),
          "mp_plan_autotune")
    return tn.value, tm.value


def mp_plan_autotune_shape(plan, prec, B):
    """Returns (atoms per tile, signals per tile, two-SM tile 0/1) the
    autotuner picked, two-SM tiles included."""
    tn, tm, pr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib().mp_plan_autotune_shape(plan, int(prec), int(B), ctypes.byref(tn), ctypes.byref(tm), ctypes.byref(pr)),
          "mp_plan_autotune_shape")
    return tn.value, tm.value, pr.value


def mp_recover_noalloc(psi_ptr, N, M, ld, y_ptr, x_ptr, stop, result, stream=None, trace=None):
    """Allocation-free decode (include/mpgb_noalloc.h): ``stop`` is an
    mp_stop, ``result`` an mp_result filled in place, ``trace`` an optional
    mp_trace; returns the status."""
    return lib().mp_recover_noalloc(ctypes.c_void_p(int(psi_ptr)), int(N), int(M), int(ld),
                                    ctypes.c_void_p(int(y_ptr)), ctypes.c_void_p(int(x_ptr)), ctypes.byref(stop),
                                    ctypes.byref(trace) if trace is not None else None,
                                    ctypes.byref(result), _stream(stream))


def mp_debug_correlations(plan, prec, R_ptr, B, C_ptr, stream=None):
    """Tensor-core correlations of B residuals (diagnostic)."""
    return check(lib().mp_debug_correlations(plan, int(prec), ctypes.c_void_p(int(R_ptr)), int(B),
                                             ctypes.c_void_p(int(C_ptr)), _stream(stream)),
                 "mp_debug_correlations")


def mp_debug_time_gemm(plan, prec, B, shape=(0, 0), reps=20):
    """Microseconds per launch of the batched correlation GEMM on B
    synthetic rows; shape = (signals per tile, atoms per tile[, two-SM tile
    0/1]), (0, 0) = the shape a batch of B would use."""
    us = ctypes.c_double()
    pair = int(shape[2]) if len(shape) > 2 else 0
    check(lib().mp_debug_time_gemm_pair(plan, int(prec), int(B), int(shape[0]), int(shape[1]), pair, int(reps),
                                        ctypes.byref(us)), "mp_debug_time_gemm")
    return us.value


# ---------------------------------------------------------------- server (include/mpgb_server.h)

def mp_shard_record_bytes(plan):
    return int(lib().mp_shard_record_bytes(plan))


def mp_shard_init(plan, y_ptr, r_ptr, x_ptr, eps, max_iters, state_ptr, stream=None):
    st = mp_stop(float(eps), int(max_iters), 0)
    return check(lib().mp_shard_init(plan, ctypes.c_void_p(int(y_ptr)), ctypes.c_void_p(int(r_ptr)),
                                      ctypes.c_void_p(int(x_ptr)), ctypes.byref(st),
                                      ctypes.c_void_p(int(state_ptr)), _stream(stream)), "mp_shard_init")


def mp_shard_step_local(plan, atom_offset, r_ptr, record_ptr, stream=None):
    return check(lib().mp_shard_step_local(plan, int(atom_offset), ctypes.c_void_p(int(r_ptr)),
                                            ctypes.c_void_p(int(record_ptr)), _stream(stream)),
                 "mp_shard_step_local")


def mp_shard_step_apply(plan, atom_offset, records_ptr, n_records, r_ptr, x_ptr, state_ptr, trace=None,
                        stream=None):
    return check(lib().mp_shard_step_apply(plan, int(atom_offset), ctypes.c_void_p(int(records_ptr)),
                                            int(n_records), ctypes.c_void_p(int(r_ptr)),
                                            ctypes.c_void_p(int(x_ptr)), ctypes.c_void_p(int(state_ptr)),
                                            ctypes.byref(trace) if trace is not None else None,
                                            _stream(stream)), "mp_shard_step_apply")


def mp_server_create(hbm_budget_bytes, max_slots, max_queue):
    h = ctypes.c_void_p()
    check(lib().mp_server_create(ctypes.byref(h), int(hbm_budget_bytes), int(max_slots), int(max_queue)),
          "mp_server_create")
    return h.value


def mp_server_add_dictionary(srv, plan, prec):
    d = ctypes.c_int()
    check(lib().mp_server_add_dictionary(srv, plan, int(prec), ctypes.byref(d)), "mp_server_add_dictionary")
    return d.value


def mp_server_dictionary_slots(srv, dict_id):
    n = ctypes.c_int()
    check(lib().mp_server_dictionary_slots(srv, int(dict_id), ctypes.byref(n)), "mp_server_dictionary_slots")
    return n.value


def mp_server_submit(srv, dict_id, y_host, eps, max_iters):
    """Returns (status, ticket); y_host is a contiguous float32 numpy array."""
    st = mp_stop(float(eps), int(max_iters), 0)
    t = ctypes.c_uint64()
    s = lib().mp_server_submit(srv, int(dict_id), ctypes.c_void_p(y_host.ctypes.data), ctypes.byref(st),
                               ctypes.byref(t))
    return s, t.value


def mp_server_poll(srv, ticket, x_host=None):
    """Returns (status, mp_result or None); fills x_host (float32, M) when done."""
    res = mp_result()
    s = lib().mp_server_poll(srv, ctypes.c_uint64(ticket),
                             ctypes.c_void_p(x_host.ctypes.data) if x_host is not None else None, ctypes.byref(res))
    return s, (res if s == MP_OK else None)


def mp_server_get_stats(srv):
    out = mp_server_stats()
    check(lib().mp_server_get_stats(srv, ctypes.byref(out)), "mp_server_get_stats")
    return out


def mp_server_reset_stats(srv):
    return check(lib().mp_server_reset_stats(srv), "mp_server_reset_stats")


def mp_server_destroy(srv):
    return check(lib().mp_server_destroy(srv), "mp_server_destroy")
