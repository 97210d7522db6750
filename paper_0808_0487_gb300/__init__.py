"""Python binding of libdwt: the multivariate fast discrete Walsh transform over
digital nets on GB300 (sm_103a).

This module only marshals arguments: every step of every call runs in the CUDA
kernels of ``libdwt.so`` behind the C ABI declared in ``include/dwt.h``.  The
functions keep the C names.  Tensors (anything with ``data_ptr()``) or raw
integer addresses may be passed wherever the C call takes a pointer; streams
may be ``None`` (torch's current stream), a ``torch.cuda.Stream`` or an integer
``cudaStream_t``.

There is no fallback: if the library is missing, every call raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdwt.so")

# status codes
DWT_OK = 0
DWT_EINVAL = 1
DWT_ESPAN = 2
DWT_ENOMEM = 3
DWT_ECUDA = 4
DWT_ETIMEOUT = 5
DWT_EBUSY = 6
DWT_EUNSUPPORTED = 7
# dtypes
DWT_F32, DWT_F64, DWT_I32, DWT_C64, DWT_C128 = 0, 1, 2, 3, 4
# algorithms
DWT_ALGO_AUTO, DWT_ALGO_BUTTERFLY, DWT_ALGO_TC_SPLIT_BF16 = 0, 1, 2
# weights
DWT_WEIGHT_NONE, DWT_WEIGHT_INV_SQ_WAVENUMBER = 0, 1
# plan flags
DWT_PLAN_TRANSFORM_ONLY = 1
DWT_PLAN_KEEP_INDEX_MAP = 2
DWT_PLAN_TUNE = 4

_lib = None


class dwt_request(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("m", ctypes.c_int), ("s", ctypes.c_int),
                ("C", ctypes.c_void_p), ("coef", ctypes.c_void_p), ("weight", ctypes.c_int),
                ("threshold", ctypes.c_double), ("c_out", ctypes.c_void_p)]


class dwt_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("s", ctypes.c_int), ("d_trc", ctypes.c_int), ("d_sup", ctypes.c_int),
                ("var_trc", ctypes.c_double * 256), ("var_sup", ctypes.c_double * 256),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_plan", ctypes.c_double),
                ("t_done", ctypes.c_double), ("message", ctypes.c_char * 160)]


class DwtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (_strerror(status), status, msg))
        self.status = status


_VP = ctypes.c_void_p
_LL = ctypes.c_longlong
_I = ctypes.c_int

_SIGS = {
    "dwt_plan_create": (_I, [_I, _I, _I, _VP, ctypes.c_uint, _VP, ctypes.POINTER(_VP)]),
    "dwt_plan_destroy": (_I, [_VP]),
    "dwt_plan_destroy_async": (_I, [_VP, _VP]),
    "dwt_plan_info": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "dwt_plan_passes": (_I, [_VP, _I, _VP, _VP, _VP]),
    "dwt_pass_plan_for": (_I, [_I, _I, _I, _LL, _VP, _VP, _VP]),
    "dwt_plan_tables": (_I, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP)]),
    "dwt_points": (_I, [_VP, _VP, _LL, _VP]),
    "dwt_wavenumber_to_index": (_I, [_VP, _VP, _VP, _LL, _VP]),
    "dwt_index_to_wavenumber": (_I, [_VP, _VP, _VP, _LL, _VP]),
    "dwt_forward": (_I, [_VP, _VP, _VP, _I, _LL, _LL, _I, _I, _I, _VP]),
    "dwt_inverse": (_I, [_VP, _VP, _VP, _I, _LL, _LL, _I, _I, _I, _VP]),
    "dwt_plan_tuned": (_I, [_VP, _VP, _VP, _VP]),
    "dwt_forward_grouped": (_I, [_VP, _I, _I, _I, _VP]),
    "dwt_inverse_grouped": (_I, [_VP, _I, _I, _I, _VP]),
    "dwt_forward_digits": (_I, [_VP, _VP, _VP, _I, _LL, _LL, _I, _I, _I, _I, _VP]),
    "dwt_inverse_digits": (_I, [_VP, _VP, _VP, _I, _LL, _LL, _I, _I, _I, _I, _VP]),
    "dwt_interpolate": (_I, [_VP, _VP, _VP, _VP, _I, _LL, _I, _I, _I, _VP, _VP, ctypes.c_double, _VP]),
    "dwt_interpolate_host": (_I, [_VP, _VP, _VP, _I, _LL, _I, _I, _VP, _VP, ctypes.c_double, _VP]),
    "dwt_selftest_bounded_wait": (_I, [_VP]),
    "dwt_spline_prepare": (_I, [_VP, ctypes.c_double, _VP, _VP]),
    "dwt_spline": (_I, [_VP, _VP, _VP, _I, _LL, _VP, _VP, _VP, ctypes.c_double, _VP]),
    "dwt_spline_values_shifted": (_I, [_VP, _VP, _VP, _I, _VP, _I, _LL, _VP, _VP, _VP]),
    "dwt_spline_eval": (_I, [_VP, _VP, _I, _LL, _VP, _I, _I, _VP, _LL, _VP]),
    "dwt_plan": (_I, [_I, _I, _I, _VP, ctypes.c_uint, _VP, ctypes.POINTER(_VP)]),
    "dwt_effdim": (_I, [_VP, _VP, _I, _LL, _I, _VP, _VP, _VP, _VP, ctypes.c_double, _VP]),
    "dwt_effdim_packed": (_I, [_VP, _VP, _I, _LL, _I, _VP, _VP, ctypes.c_double, _VP]),
    "dwt_effdim_static": (_I, [_VP, _VP, _I, _LL, _I, _VP, _VP, ctypes.c_double, _VP]),
    "dwt_eval_product": (_I, [_VP, _VP, _VP, _I, _LL, _I, _VP]),
    "dwt_eval_exp": (_I, [_VP, _VP, _I, _LL, _I, _VP]),
    "dwt_server_create": (_I, [ctypes.c_size_t, _I, _I, ctypes.POINTER(_VP)]),
    "dwt_server_submit": (_I, [_VP, ctypes.POINTER(dwt_request), ctypes.POINTER(ctypes.c_ulonglong)]),
    "dwt_server_poll": (_I, [_VP, ctypes.c_ulonglong, ctypes.POINTER(dwt_result)]),
    "dwt_server_wait": (_I, [_VP, ctypes.c_ulonglong, ctypes.c_double, ctypes.POINTER(dwt_result)]),
    "dwt_server_stats": (_I, [_VP, ctypes.POINTER(_LL), ctypes.POINTER(ctypes.c_size_t),
                              ctypes.POINTER(ctypes.c_double)]),
    "dwt_server_destroy": (_I, [_VP]),
    "dwt_strerror": (ctypes.c_char_p, [_I]),
    "dwt_last_error": (ctypes.c_char_p, []),
    "dwt_launch_count": (_LL, []),
    "dwt_alloc_count": (_LL, []),
    "dwt_profile_enable": (_I, [_I]),
    "dwt_profile_reset": (_I, []),
    "dwt_profile_query": (_I, [ctypes.c_char_p, ctypes.POINTER(_LL), ctypes.POINTER(ctypes.c_double)]),
}


def lib():
    """The loaded ``libdwt.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise DwtError(DWT_EUNSUPPORTED, "libdwt.so is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _strerror(status):
    try:
        return lib().dwt_strerror(status).decode()
    except Exception:  # library missing while formatting an error
        return "status"


def _ptr(x):
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x)


def _stream(s):
    if s is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def _check(status, allow=()):
    if status != DWT_OK and status not in allow:
        raise DwtError(status, lib().dwt_last_error().decode())
    return status


class Plan:
    """Owner of a ``dwt_plan_t``; ``status`` holds the coset-table status of creation."""

    def __init__(self, handle, p, m, s, status):
        self.handle = handle
        self.p, self.m, self.s = p, m, s
        self.N = p ** m
        self.status = status

    @property
    def _as_parameter_(self):
        return self.handle

    def close(self):
        if self.handle:
            lib().dwt_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dwt_plan(p, m, s, C, flags=0, stream=None):
    """``dwt_plan``: C is a host array uint8 [s][m][m] (numpy)."""
    C = np.ascontiguousarray(C, dtype=np.uint8)
    if C.shape != (s, m, m):
        raise ValueError("C must have shape (s, m, m)")
    h = _VP()
    st = lib().dwt_plan(p, m, s, C.ctypes.data, flags, _stream(stream), ctypes.byref(h))
    _check(st, allow=(DWT_ESPAN, DWT_EUNSUPPORTED))
    return Plan(h.value, p, m, s, st)


def dwt_plan_create(p, m, s, C, flags=0, stream=None):
    """``dwt_plan_create``, the earlier name of ``dwt_plan``."""
    C = np.ascontiguousarray(C, dtype=np.uint8)
    if C.shape != (s, m, m):
        raise ValueError("C must have shape (s, m, m)")
    h = _VP()
    st = lib().dwt_plan_create(p, m, s, C.ctypes.data, flags, _stream(stream), ctypes.byref(h))
    _check(st, allow=(DWT_ESPAN, DWT_EUNSUPPORTED))
    return Plan(h.value, p, m, s, st)


def dwt_plan_destroy(plan):
    plan.close()
    return DWT_OK


def dwt_plan_destroy_async(plan, stream=None):
    st = lib().dwt_plan_destroy_async(plan.handle, _stream(stream))
    plan.handle = None
    return _check(st)


def dwt_plan_info(plan):
    p, m, s, t = _I(), _I(), _I(), _I()
    N = _LL()
    _check(lib().dwt_plan_info(plan.handle, ctypes.byref(p), ctypes.byref(m), ctypes.byref(s), ctypes.byref(N),
                               ctypes.byref(t)))
    return dict(p=p.value, m=m.value, s=s.value, N=N.value, tables_status=t.value)


def dwt_plan_passes(plan, elem_bytes):
    """The digit split of the generic passes for elements of elem_bytes: [(digits, columns), ...]."""
    q = _I()
    d = (_I * 32)()
    w = (_I * 32)()
    _check(lib().dwt_plan_passes(plan.handle, elem_bytes, ctypes.byref(q), d, w))
    return [(d[t], w[t]) for t in range(q.value)]


def dwt_plan_tuned(plan):
    """The measured choices of a DWT_PLAN_TUNE plan: dict(lo_digits, tc, group_bytes); 0 = heuristic."""
    lo = _I()
    tc = _I()
    gb = _LL()
    _check(lib().dwt_plan_tuned(plan.handle, ctypes.byref(lo), ctypes.byref(tc), ctypes.byref(gb)))
    return {"lo_digits": lo.value, "tc": tc.value, "group_bytes": gb.value}


def dwt_pass_plan_for(p, m, elem_bytes, min_tiles=304):
    """The heuristic pass split for (p, m, element size), host only: [(digits, columns), ...]."""
    q = _I()
    d = (_I * 32)()
    w = (_I * 32)()
    _check(lib().dwt_pass_plan_for(p, m, elem_bytes, min_tiles, ctypes.byref(q), d, w))
    return [(d[t], w[t]) for t in range(q.value)]


def dwt_plan_tables(plan):
    """Device addresses (ints) of the plan's W[N] float and cls[N][2] uint8 tables."""
    W, cls = _VP(), _VP()
    _check(lib().dwt_plan_tables(plan.handle, ctypes.byref(W), ctypes.byref(cls)))
    return W.value, cls.value


def dwt_points(plan, Y, ldY=None, stream=None):
    return _check(lib().dwt_points(plan.handle, _ptr(Y), ldY or plan.N, _stream(stream)))


def dwt_wavenumber_to_index(plan, k, H, cnt, stream=None):
    return _check(lib().dwt_wavenumber_to_index(plan.handle, _ptr(k), _ptr(H), cnt, _stream(stream)))


def dwt_index_to_wavenumber(plan, H, k, cnt, stream=None):
    return _check(lib().dwt_index_to_wavenumber(plan.handle, _ptr(H), _ptr(k), cnt, _stream(stream)))


def dwt_forward(plan, inp, out, batch, ld_in, ld_out, in_t, out_t, algo=DWT_ALGO_AUTO, stream=None):
    return _check(lib().dwt_forward(plan.handle, _ptr(inp), _ptr(out), batch, ld_in, ld_out, in_t, out_t, algo,
                                    _stream(stream)))


def dwt_inverse(plan, inp, out, batch, ld_in, ld_out, in_t, out_t, algo=DWT_ALGO_AUTO, stream=None):
    return _check(lib().dwt_inverse(plan.handle, _ptr(inp), _ptr(out), batch, ld_in, ld_out, in_t, out_t, algo,
                                    _stream(stream)))


class _Job(ctypes.Structure):
    """struct dwt_job of include/dwt.h."""
    _fields_ = [("plan", _VP), ("in_", _VP), ("out", _VP), ("batch", _I), ("ld_in", _LL), ("ld_out", _LL)]


def _jobs(jobs):
    arr = (_Job * len(jobs))()
    for i, (plan, inp, out, batch, ld_in, ld_out) in enumerate(jobs):
        arr[i] = _Job(plan.handle, _ptr(inp), _ptr(out), batch, ld_in, ld_out)
    return arr


def dwt_forward_grouped(jobs, in_t, out_t, stream=None):
    """jobs: list of (plan, in, out, batch, ld_in, ld_out); see dwt_forward_grouped in include/dwt.h."""
    arr = _jobs(jobs)
    return _check(lib().dwt_forward_grouped(ctypes.cast(arr, _VP), len(jobs), in_t, out_t, _stream(stream)))


def dwt_inverse_grouped(jobs, in_t, out_t, stream=None):
    arr = _jobs(jobs)
    return _check(lib().dwt_inverse_grouped(ctypes.cast(arr, _VP), len(jobs), in_t, out_t, _stream(stream)))


def dwt_forward_digits(plan, inp, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, stream=None):
    return _check(lib().dwt_forward_digits(plan.handle, _ptr(inp), _ptr(out), batch, ld_in, ld_out, in_t, out_t, d0, nd,
                                           _stream(stream)))


def dwt_inverse_digits(plan, inp, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, stream=None):
    return _check(lib().dwt_inverse_digits(plan.handle, _ptr(inp), _ptr(out), batch, ld_in, ld_out, in_t, out_t, d0, nd,
                                           _stream(stream)))


def dwt_interpolate(plan, f, c, coef, batch, ld, f_t, weight, algo=DWT_ALGO_AUTO, var=None, dim=None,
                    threshold=0.99, stream=None):
    return _check(lib().dwt_interpolate(plan.handle, _ptr(f), _ptr(c), _ptr(coef), batch, ld, f_t, weight, algo,
                                        _ptr(var), _ptr(dim), threshold, _stream(stream)))


def dwt_interpolate_host(plan, f, c, batch, ld, f_t, weight, var=None, dim=None, threshold=0.99, stream=None):
    """dwt_interpolate on host buffers (f, c, var, dim host-resident; page-locked ones overlap copies)."""
    return _check(lib().dwt_interpolate_host(plan.handle, _ptr(f), _ptr(c), batch, ld, f_t, weight, _ptr(var),
                                             _ptr(dim), threshold, _stream(stream)))


def dwt_selftest_bounded_wait(stream=None):
    """Run the bounded-wait self-test; returns the status (DWT_ETIMEOUT expected) without raising."""
    return lib().dwt_selftest_bounded_wait(_stream(stream))


def dwt_spline_prepare(plan, alpha, gamma, stream=None):
    """Kernel-spline tables for (alpha, gamma[s]) (Sec. 3.1, Sec. 4); gamma is a host sequence."""
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    return _check(lib().dwt_spline_prepare(plan.handle, float(alpha), g.ctypes.data, _stream(stream)))


def dwt_spline(plan, f, c, batch, ld, var_trc=None, var_sup=None, dim=None, threshold=0.99, stream=None):
    """Spline coefficients c_n of f (FP64) and the ANOVA variances of the spline."""
    return _check(lib().dwt_spline(plan.handle, _ptr(f), _ptr(c), batch, ld, _ptr(var_trc), _ptr(var_sup),
                                   _ptr(dim), threshold, _stream(stream)))


def dwt_spline_values_shifted(plan, c, delta, M, values, batch, ld, f_shift=None, sse=None, stream=None):
    """Spline values at the net shifted by delta (host uint32 [s], M digits); optional hold-out error."""
    d = np.ascontiguousarray(delta, dtype=np.uint32)
    return _check(lib().dwt_spline_values_shifted(plan.handle, _ptr(c), d.ctypes.data, int(M), _ptr(values), batch, ld,
                                                  _ptr(f_shift), _ptr(sse), _stream(stream)))


def dwt_spline_eval(plan, c, batch, ld, X, Q, M, values, ldv=None, stream=None):
    """Spline values at Q arbitrary points X (device uint32 [Q][s], M digits) into values [batch][ldv]."""
    return _check(lib().dwt_spline_eval(plan.handle, _ptr(c), batch, ld, _ptr(X), int(Q), int(M), _ptr(values),
                                        Q if ldv is None else ldv, _stream(stream)))


def dwt_effdim(plan, coef, batch, ld, t, var_trc=None, var_sup=None, d_trc=None, d_sup=None, threshold=0.99,
               stream=None):
    return _check(lib().dwt_effdim(plan.handle, _ptr(coef), batch, ld, t, _ptr(var_trc), _ptr(var_sup), _ptr(d_trc),
                                   _ptr(d_sup), threshold, _stream(stream)))


def dwt_effdim_packed(plan, coef, batch, ld, t, var=None, dim=None, threshold=0.99, stream=None):
    return _check(lib().dwt_effdim_packed(plan.handle, _ptr(coef), batch, ld, t, _ptr(var), _ptr(dim), threshold,
                                   _stream(stream)))


def dwt_effdim_static(plan, coef, batch, ld, t, var=None, dim=None, threshold=0.99, stream=None):
    """dwt_effdim_packed without any device allocation (fixed in-library scratch; see include/dwt.h)."""
    return _check(lib().dwt_effdim_static(plan.handle, _ptr(coef), batch, ld, t, _ptr(var), _ptr(dim), threshold,
                                          _stream(stream)))


def dwt_eval_product(plan, coef, f, batch, ld, t, stream=None):
    return _check(lib().dwt_eval_product(plan.handle, _ptr(coef), _ptr(f), batch, ld, t, _stream(stream)))


def dwt_eval_exp(plan, f, batch, ld, t, stream=None):
    return _check(lib().dwt_eval_exp(plan.handle, _ptr(f), batch, ld, t, _stream(stream)))


def dwt_strerror(status):
    return lib().dwt_strerror(status).decode()


def dwt_last_error():
    return lib().dwt_last_error().decode()


def dwt_launch_count():
    return lib().dwt_launch_count()


def dwt_alloc_count():
    return lib().dwt_alloc_count()


def dwt_profile_enable(on=True):
    return _check(lib().dwt_profile_enable(1 if on else 0))


def dwt_profile_reset():
    return _check(lib().dwt_profile_reset())


def dwt_profile_query(name):
    n = _LL()
    ms = ctypes.c_double()
    _check(lib().dwt_profile_query(name.encode(), ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


# ---- serving ------------------------------------------------------------------
class Server:
    """Owner of a ``dwt_server_t`` (continuous-batching engine, see include/dwt.h)."""

    def __init__(self, handle):
        self.handle = handle
        self._keep = {}

    def close(self):
        if self.handle:
            lib().dwt_server_destroy(self.handle)
            self.handle = None
        self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dwt_server_create(hbm_budget_bytes=0, slots=8, max_queue=1 << 16):
    h = _VP()
    _check(lib().dwt_server_create(hbm_budget_bytes, slots, max_queue, ctypes.byref(h)))
    return Server(h.value)


def dwt_server_submit(server, p, m, s, C, coef, weight=DWT_WEIGHT_INV_SQ_WAVENUMBER, threshold=0.99, c_out=None):
    """Queue one request; returns its ticket.  C and coef are copied by the call;
    c_out (a host array) must stay alive until the request is done."""
    C = np.ascontiguousarray(C, dtype=np.uint8)
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    req = dwt_request(p, m, s, C.ctypes.data, coef.ctypes.data, weight, threshold, _ptr(c_out))
    t = ctypes.c_ulonglong()
    _check(lib().dwt_server_submit(server.handle, ctypes.byref(req), ctypes.byref(t)))
    if c_out is not None:
        server._keep[t.value] = c_out
    return t.value


def _result(r):
    s = r.s
    return dict(status=r.status, d_trc=r.d_trc, d_sup=r.d_sup, var_trc=np.array(r.var_trc[:s + 1]),
                var_sup=np.array(r.var_sup[:s + 1]), t_submit=r.t_submit, t_admit=r.t_admit, t_plan=r.t_plan,
                t_done=r.t_done, message=r.message.decode(errors="replace"))


def dwt_server_poll(server, ticket):
    """The result dict when done, else None."""
    r = dwt_result()
    st = lib().dwt_server_poll(server.handle, ticket, ctypes.byref(r))
    if st == DWT_EBUSY:
        return None
    _check(st)
    server._keep.pop(ticket, None)
    return _result(r)


def dwt_server_wait(server, ticket, timeout_s=600.0):
    r = dwt_result()
    _check(lib().dwt_server_wait(server.handle, ticket, timeout_s, ctypes.byref(r)))
    server._keep.pop(ticket, None)
    return _result(r)


def dwt_server_stats(server):
    q = _LL()
    b = ctypes.c_size_t()
    t = ctypes.c_double()
    _check(lib().dwt_server_stats(server.handle, ctypes.byref(q), ctypes.byref(b), ctypes.byref(t)))
    return dict(queued=q.value, bytes_in_use=b.value, now=t.value)


def dwt_server_destroy(server):
    server.close()
    return DWT_OK
