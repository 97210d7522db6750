"""CPU oracle for the multivariate discrete Walsh transform over digital nets.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  It is a plain, slow, FP64 restatement of the paper (Liu, Dick and
Hickernell, "A Multivariate Fast Discrete Walsh Transform with an Application
to Function Interpolation") in ``oracle.c``, wrapped here with numpy.  It
shares no code with the GPU library.

Every wrapper names the paper passage its C function follows.  Arrays:
generating matrices ``C`` are uint8 ``[s][m][m]`` (``C[j][i][c]``: row ``i``
gives the point digit ``y_{i+1}``, column ``c`` multiplies the index digit
``n_c``); net points are uint32 ``Y[s][N]`` with ``x = Y / p**m``; data and
coefficients are in natural ``n`` / ``H`` order.

Parity status: every function here is pinned by a test in
``tests/test_oracle_*.py`` against something other than itself.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_u8p = ctypes.POINTER(ctypes.c_uint8)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f32p = ctypes.POINTER(ctypes.c_float)
_f64p = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_net_points.argtypes = [ctypes.c_int] * 3 + [_u8p, _u32p]
        L.orc_net_x.argtypes = [ctypes.c_int] * 3 + [_u32p, _f64p]
        L.orc_k_to_h.argtypes = [ctypes.c_int] * 3 + [_u8p, _u32p, ctypes.c_int, _u32p]
        L.orc_dwt_direct.argtypes = [ctypes.c_int, ctypes.c_int, _f64p, _f64p, _u32p, ctypes.c_long, _f64p, _f64p]
        L.orc_dwt_walsh_def.argtypes = [ctypes.c_int] * 3 + [_u32p, _f64p, _f64p, _u32p, ctypes.c_long, _f64p, _f64p]
        L.orc_fwt.argtypes = [ctypes.c_int, ctypes.c_int, _f64p, _f64p]
        L.orc_fiwt.argtypes = [ctypes.c_int, ctypes.c_int, _f64p, _f64p]
        L.orc_fwt_i64.argtypes = [ctypes.c_int, _i64p]
        L.orc_fiwt_i64.argtypes = [ctypes.c_int, _i64p]
        L.orc_weight_class.argtypes = [ctypes.c_int, _u32p, ctypes.c_long, _f32p, _f64p, _u8p]
        L.orc_rank.argtypes = [ctypes.c_int] * 3 + [_u8p]
        L.orc_coset_leaders_bruteforce.argtypes = [ctypes.c_int] * 3 + [_u8p, _u32p]
        L.orc_coset_leaders_dp.argtypes = [ctypes.c_int] * 3 + [_u8p, _u8p, _u32p, _f32p, _f64p, _u8p,
                                                                _u32p, ctypes.c_long, _u32p]
        L.orc_effdim_threshold.argtypes = [ctypes.c_int, _f64p, _f64p, ctypes.c_double, _ip, _ip]
        L.orc_effdim.argtypes = [ctypes.c_int, ctypes.c_long, _f64p, _f64p, _u8p, ctypes.c_double,
                                 _f64p, _f64p, _ip, _ip]
        L.orc_eval_product.argtypes = [ctypes.c_int] * 3 + [_u32p, _f64p, _f64p]
        L.orc_eval_exp.argtypes = [ctypes.c_int] * 3 + [_u32p, _f64p]
        L.orc_kprime.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint32]
        L.orc_kprime.restype = ctypes.c_double
        L.orc_rprime.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_uint32]
        L.orc_rprime.restype = ctypes.c_double
        L.orc_kernel_data.argtypes = [ctypes.c_int] * 3 + [_u32p, ctypes.c_double, _f64p, _f64p, _f64p, _f64p]
        L.orc_spline_eval.argtypes = [ctypes.c_int] * 3 + [_u32p, _f64p, _u32p, ctypes.c_int, ctypes.c_int,
                                                            ctypes.c_double, _f64p, _f64p]
        L.orc_spline_eval.restype = None
        L.orc_kernel_shift_data.argtypes = [ctypes.c_int] * 3 + [_u32p, _u32p, ctypes.c_int, ctypes.c_double, _f64p,
                                                                  _f64p]
        _lib = L
    return _lib


def _p(a, t):
    if a is None:
        return None
    return a.ctypes.data_as(t)


def _C(C):
    C = np.ascontiguousarray(C, dtype=np.uint8)
    assert C.ndim == 3 and C.shape[1] == C.shape[2]
    return C


# --- Def. 1.1 ---------------------------------------------------------------
def net_points(p, m, C):
    """Integer net points ``Y[s][N]`` with ``x_{j,n} = Y / p**m`` (Def. 1.1, eq. defy)."""
    C = _C(C)
    s = C.shape[0]
    Y = np.empty((s, p ** m), dtype=np.uint32)
    lib().orc_net_points(p, m, s, _p(C, _u8p), _p(Y, _u32p))
    return Y


def net_x(p, m, Y):
    """``x_{j,n} = Y_{j,n} / p**m`` in double (Def. 1.1)."""
    Y = np.ascontiguousarray(Y, dtype=np.uint32)
    x = np.empty(Y.shape, dtype=np.float64)
    lib().orc_net_x(p, m, Y.shape[0], _p(Y, _u32p), _p(x, _f64p))
    return x


# --- Sec. 2.1 ---------------------------------------------------------------
def k_to_h(p, m, C, k):
    """Coset index ``H`` of wavenumber vectors ``k[cnt][s]``: ``C . k`` (Sec. 2.1)."""
    C = _C(C)
    k = np.ascontiguousarray(np.atleast_2d(k), dtype=np.uint32)
    H = np.empty(k.shape[0], dtype=np.uint32)
    lib().orc_k_to_h(p, m, C.shape[0], _p(C, _u8p), _p(k, _u32p), k.shape[0], _p(H, _u32p))
    return H


def rank(p, m, C):
    """Rank over F_p of the rows of C_1..C_s (all cosets nonempty iff rank == m)."""
    C = _C(C)
    return lib().orc_rank(p, m, C.shape[0], _p(C, _u8p))


def coset_leaders_bruteforce(p, m, C):
    """K(C) by enumeration in (nu, lexicographic) order (Sec. 2.1). Returns (status, kmap[N][s])."""
    C = _C(C)
    s = C.shape[0]
    kmap = np.zeros((p ** m, s), dtype=np.uint32)
    st = lib().orc_coset_leaders_bruteforce(p, m, s, _p(C, _u8p), _p(kmap, _u32p))
    return st, kmap


def coset_leaders_dp(p, m, C, want_kmap=False, Hsel=None, want_W64=True):
    """K(C) by the coordinate dynamic programme (Sec. 2.1).

    Returns a dict with ``status``, ``numin[N]`` (least nu per coset), ``W32[N]``,
    ``W64[N]`` (optional), ``cls[N][2]`` and optionally ``kmap[N][s]`` and
    ``ksel[len(Hsel)][s]``.
    """
    C = _C(C)
    s = C.shape[0]
    N = p ** m
    numin = np.empty(N, dtype=np.uint8)
    W32 = np.empty(N, dtype=np.float32)
    W64 = np.empty(N, dtype=np.float64) if want_W64 else None
    cls = np.empty((N, 2), dtype=np.uint8)
    kmap = np.empty((N, s), dtype=np.uint32) if want_kmap else None
    if Hsel is not None:
        Hsel = np.ascontiguousarray(Hsel, dtype=np.uint32)
        ksel = np.empty((len(Hsel), s), dtype=np.uint32)
        nsel = len(Hsel)
    else:
        ksel = None
        nsel = 0
    st = lib().orc_coset_leaders_dp(p, m, s, _p(C, _u8p), _p(numin, _u8p), _p(kmap, _u32p),
                                    _p(W32, _f32p), _p(W64, _f64p), _p(cls, _u8p),
                                    _p(Hsel, _u32p), nsel, _p(ksel, _u32p))
    return dict(status=st, numin=numin, W32=W32, W64=W64, cls=cls, kmap=kmap, ksel=ksel)


def weight_class(k):
    """Exact weight ``prod_j (1+k_j)^-2`` (FP32 and FP64) and class (max supp, |supp|) of ``k[cnt][s]``."""
    k = np.ascontiguousarray(np.atleast_2d(k), dtype=np.uint32)
    cnt, s = k.shape
    W32 = np.empty(cnt, dtype=np.float32)
    W64 = np.empty(cnt, dtype=np.float64)
    cls = np.empty((cnt, 2), dtype=np.uint8)
    st = lib().orc_weight_class(s, _p(k, _u32p), cnt, _p(W32, _f32p), _p(W64, _f64p), _p(cls, _u8p))
    if st:
        raise OverflowError("weight denominator exceeds 64 bits")
    return W32, W64, cls


# --- Sec. 2.2 / 3.3 ---------------------------------------------------------
def _split(f):
    f = np.asarray(f)
    re = np.ascontiguousarray(f.real, dtype=np.float64).copy()
    im = np.ascontiguousarray(f.imag if np.iscomplexobj(f) else np.zeros_like(re), dtype=np.float64).copy()
    return re, im


def dwt_direct(p, m, f, H=None):
    """O(N) per output: ``f~(H) = p^-m sum_n f_n omega^{-n.h}`` (eq. dwalshcoeff, Sec. 2.2)."""
    re, im = _split(f)
    if H is not None:
        H = np.ascontiguousarray(H, dtype=np.uint32)
        n = len(H)
    else:
        n = p ** m
    ore = np.empty(n)
    oim = np.empty(n)
    lib().orc_dwt_direct(p, m, _p(re, _f64p), _p(im, _f64p), _p(H, _u32p), n if H is not None else 0,
                         _p(ore, _f64p), _p(oim, _f64p))
    return ore + 1j * oim


def dwt_walsh_def(p, m, Y, f, k):
    """``f~(k) = p^-m sum_n f(x_n) conj(wal_k(x_n))`` from Def. 1.2/1.3 directly."""
    Y = np.ascontiguousarray(Y, dtype=np.uint32)
    re, im = _split(f)
    k = np.ascontiguousarray(np.atleast_2d(k), dtype=np.uint32)
    ore = np.empty(k.shape[0])
    oim = np.empty(k.shape[0])
    lib().orc_dwt_walsh_def(p, m, Y.shape[0], _p(Y, _u32p), _p(re, _f64p), _p(im, _f64p),
                            _p(k, _u32p), k.shape[0], _p(ore, _f64p), _p(oim, _f64p))
    return ore + 1j * oim


def fwt(p, m, f):
    """Algorithm 1 (FWT) in FP64, including the factor p^-m. Complex result."""
    re, im = _split(f)
    lib().orc_fwt(p, m, _p(re, _f64p), _p(im, _f64p))
    return re + 1j * im


def fiwt(p, m, c):
    """Algorithm 2 (FIWT) in FP64, no factor. Complex result."""
    re, im = _split(c)
    lib().orc_fiwt(p, m, _p(re, _f64p), _p(im, _f64p))
    return re + 1j * im


def fwt_i64(m, v):
    """Algorithm 1 for p = 2 in exact int64, unscaled: G^{(m)}."""
    v = np.ascontiguousarray(v, dtype=np.int64).copy()
    lib().orc_fwt_i64(m, _p(v, _i64p))
    return v


def fiwt_i64(m, v):
    """Algorithm 2 for p = 2 in exact int64: D^{(m)}."""
    v = np.ascontiguousarray(v, dtype=np.int64).copy()
    lib().orc_fiwt_i64(m, _p(v, _i64p))
    return v


# --- Sec. 4 -----------------------------------------------------------------
def effdim_threshold(var_trc, var_sup, thr=0.99):
    """Least d with cumulative variance >= thr * total, for trc and sup (Sec. 4)."""
    vt = np.ascontiguousarray(var_trc, dtype=np.float64)
    vs = np.ascontiguousarray(var_sup, dtype=np.float64)
    dt = ctypes.c_int()
    ds = ctypes.c_int()
    lib().orc_effdim_threshold(len(vt) - 1, _p(vt, _f64p), _p(vs, _f64p), thr, ctypes.byref(dt), ctypes.byref(ds))
    return dt.value, ds.value


def effdim(g, cls, s, thr=0.99):
    """Truncation/superposition class variances of ``sum_H g(H) wal_k(H)`` and the effective dimensions."""
    re, im = _split(g)
    cls = np.ascontiguousarray(cls, dtype=np.uint8)
    vt = np.empty(s + 1)
    vs = np.empty(s + 1)
    dt = ctypes.c_int()
    ds = ctypes.c_int()
    lib().orc_effdim(s, len(re), _p(re, _f64p), _p(im, _f64p), _p(cls, _u8p), thr,
                     _p(vt, _f64p), _p(vs, _f64p), ctypes.byref(dt), ctypes.byref(ds))
    return vt, vs, dt.value, ds.value


def interpolate(p, m, f, W, cls, s, thr=0.99):
    """Forward (Alg. 1), per-coefficient weight ``g = W f~`` (the spectral step of
    eq. splinecoef with the weight supplied by the caller), inverse (Alg. 2), and the
    effective dimensions of ``g``.  Returns ``(c, g, var_trc, var_sup, d_trc, d_sup)``."""
    ft = fwt(p, m, f)
    g = ft * np.asarray(W, dtype=np.float64)
    c = fiwt(p, m, g)
    vt, vs, dt, ds = effdim(g, cls, s, thr)
    return c, g, vt, vs, dt, ds


# --- the kernel spline (Sec. 3.1) and its ANOVA variances (Sec. 4) ---------------
def kprime(p, m, alpha, Y):
    """K'(x, 0) at x = Y / p^m (short form of Sec. 4)."""
    return lib().orc_kprime(p, m, alpha, int(Y))


def rprime(p, m, alpha, Y):
    """R'(x, 0) at x = Y / p^m (short form of Sec. 4)."""
    return lib().orc_rprime(p, m, alpha, int(Y))


def kernel_data(p, m, Y, alpha, gamma):
    """(K[N], R[s][N], E[s][N]): the kernel data K(x_n, 0), the truncated products
    R_d(x_n, 0), d = 1..s, and the degree-j parts E_j(x_n, 0) = sum_{|u|=j} gamma_u^2 R_u."""
    Y = np.ascontiguousarray(Y, dtype=np.uint32)
    s, N = Y.shape
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    K = np.empty(N)
    R = np.empty((s, N))
    E = np.empty((s, N))
    lib().orc_kernel_data(p, m, s, _p(Y, _u32p), alpha, _p(gamma, _f64p), _p(K, _f64p), _p(R, _f64p), _p(E, _f64p))
    return K, R, E


def spline(p, m, Y, f, alpha, gamma, thr=0.99):
    """The kernel spline of f on the net and the variances of its ANOVA effects.

    K~ = DWT of the kernel data; c~ = f~ / (p^m K~) (eq. splinecoef); c = FIWT(c~)
    (Algorithm 2); sigma^2_trc(d) = p^{2m} sum_H |c~|^2 (R~_d - [H = 0]) and
    sigma^2_sup(d) = p^{2m} sum_H |c~|^2 sum_{j <= d} E~_j, d = 0..s (eq. sig2sfu
    summed over u, the constant effect u = {} left out), then d_trc, d_sup.
    Returns a dict with Ktil, W (= 1 / (p^m K~)), ctil, c, var_trc, var_sup, d_trc, d_sup."""
    N = p ** m
    s = Y.shape[0]
    K, R, E = kernel_data(p, m, Y, alpha, gamma)
    Kt = fwt(p, m, K)
    W = 1.0 / (N * Kt.real)
    ft = fwt(p, m, f)
    ct = ft * W
    c = fiwt(p, m, ct)
    a = np.abs(ct) ** 2
    vt = np.zeros(s + 1)
    vs = np.zeros(s + 1)
    for d in range(1, s + 1):
        Rt = fwt(p, m, R[d - 1]).real
        Rt[0] -= 1.0
        vt[d] = N * N * float(np.dot(a, Rt))
        vs[d] = vs[d - 1] + N * N * float(np.dot(a, fwt(p, m, E[d - 1]).real))
    dt, ds = effdim_threshold(vt, vs, thr)
    return dict(Ktil=Kt, W=W, ctil=ct, c=c, var_trc=vt, var_sup=vs, d_trc=dt, d_sup=ds)


def spline_values_shifted(p, m, Y, c, delta, M, alpha, gamma):
    """Values of the spline Sf(x) = sum_v c_v K(x (-) x_v, 0) at the shifted points
    x_n (+) delta, n = 0..N-1, delta_j = delta[j] / p^M (M >= m digits).  As a
    function of n this is a convolution over the net: its DWT is
    p^m c~(H) k~(H), k~ the DWT of the shifted kernel data K(x_w (+) delta, 0);
    FIWT (Algorithm 2) gives the values."""
    Y = np.ascontiguousarray(Y, dtype=np.uint32)
    s, N = Y.shape
    D = np.ascontiguousarray(delta, dtype=np.uint32)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    Kd = np.empty(N)
    lib().orc_kernel_shift_data(p, m, s, _p(Y, _u32p), _p(D, _u32p), M, alpha, _p(g, _f64p), _p(Kd, _f64p))
    kt = fwt(p, m, Kd)
    ct = fwt(p, m, c)
    return fiwt(p, m, N * ct * kt)


def spline_eval(p, m, Y, c, X, M, alpha, gamma):
    """The spline Sf(x) = sum_n c_n K(x (-) x_n, 0) at arbitrary points x_q
    (Sec. 3.1): X[q][j] the M-digit numerators (x_{q,j} = X[q][j] / p^M, M >= m),
    c the real spline coefficients on the net; direct sum over the net with the
    short form of K' on M digits, O(N s) per point."""
    Y = np.ascontiguousarray(Y, dtype=np.uint32)
    s, N = Y.shape
    X = np.ascontiguousarray(X, dtype=np.uint32).reshape(-1, s)
    c = np.ascontiguousarray(np.real(c), dtype=np.float64)
    g = np.ascontiguousarray(gamma, dtype=np.float64)
    out = np.empty(X.shape[0])
    lib().orc_spline_eval(p, m, s, _p(Y, _u32p), _p(c, _f64p), _p(X, _u32p), X.shape[0], M, alpha, _p(g, _f64p),
                          _p(out, _f64p))
    return out


# --- synthetic test functions ------------------------------------------------
def eval_product(p, m, Y, c):
    """``f_n = prod_j (1 + c_j (x_{j,n} - 1/2))`` in FP64."""
    Y = np.ascontiguousarray(Y, dtype=np.uint32)
    c = np.ascontiguousarray(c, dtype=np.float64)
    f = np.empty(Y.shape[1])
    lib().orc_eval_product(p, m, Y.shape[0], _p(Y, _u32p), _p(c, _f64p), _p(f, _f64p))
    return f


def eval_exp(p, m, Y):
    """``f_n = exp(sum_j x_{j,n} / j^2)`` in FP64."""
    Y = np.ascontiguousarray(Y, dtype=np.uint32)
    f = np.empty(Y.shape[1])
    lib().orc_eval_exp(p, m, Y.shape[0], _p(Y, _u32p), _p(f, _f64p))
    return f
