"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module holds none of the transform's arithmetic: it draws random numbers
(SplitMix64) and turns them into generating matrices, test-function
parameters and integer data.  Net points, Walsh coefficients and everything
else are computed separately by the oracle and by the GPU library.

PRNG: SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: output i of
stream ``seed`` is ``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)`` with the
published 64-bit finaliser.  Uniform doubles take the top 53 bits; integers in
a range are drawn by rejection, so they are exactly uniform.

Workload shapes follow the paper's experiments (p = 2 nets with m = 12 and
m = 14 digits) scaled to GPU sizes; the paper's Sobol matrices are replaced by
seeded random upper-triangular generating matrices (unit diagonal for p = 2,
diagonal uniform in 1..p-1 otherwise).
"""
import numpy as np

MASTER_SEED = 0x08080487
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream purposes
P_MATRICES = 1
P_COEFFS = 2
P_INTS = 3
P_SAMPLE = 4
P_SERVE = 5
P_VALUES = 6


def _mix(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed, count, offset=0):
    """Outputs ``offset .. offset+count-1`` of the SplitMix64 stream ``seed`` (uint64 array)."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + i * _GAMMA
    return _mix(z)


def stream_seed(config, purpose, index=0):
    """Seed of the stream for (config id, purpose, index), derived from the master seed."""
    key = (int(MASTER_SEED) ^ (int(config) << 48) ^ (int(purpose) << 40) ^ int(index)) & 0xFFFFFFFFFFFFFFFF
    return int(_mix(np.uint64(key)))


def uniform(seed, count, offset=0):
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def integers(seed, count, lo, hi):
    """Exactly uniform integers in [lo, hi] by rejection sampling."""
    R = hi - lo + 1
    limit = (1 << 64) - ((1 << 64) % R)
    out = np.empty(count, dtype=np.int64)
    filled = 0
    offset = 0
    while filled < count:
        want = count - filled
        draw = want + want // 64 + 16
        z = splitmix64(seed, draw, offset)
        offset += draw
        if limit < (1 << 64):
            z = z[z < np.uint64(limit)]
        z = z[:want]
        out[filled:filled + len(z)] = (z % np.uint64(R)).astype(np.int64) + lo
        filled += len(z)
    return out


def upper_triangular_matrices(p, m, s, seed):
    """``C[s][m][m]`` uint8: zero below the diagonal, uniform F_p above it, and a
    diagonal of ones (p = 2) or uniform in 1..p-1 (p > 2): nonsingular."""
    C = np.zeros((s, m, m), dtype=np.uint8)
    iu = np.triu_indices(m, 1)
    nup = len(iu[0])
    above = integers(seed, s * nup, 0, p - 1).reshape(s, nup)
    diag = np.ones((s, m), dtype=np.int64) if p == 2 else \
        integers(stream_seed(0, P_MATRICES, seed & 0xFFFFFF), s * m, 1, p - 1).reshape(s, m)
    for j in range(s):
        C[j][iu] = above[j]
        C[j][np.arange(m), np.arange(m)] = diag[j]
    return C


def reversed_identity(m):
    """J with ones at [i][m-1-i]: the net coordinate x_n = n / p^m."""
    return np.fliplr(np.eye(m, dtype=np.uint8)).copy()


# --------------------------------------------------------------------------
# Named workloads.  Each returns a dict of plain arrays and sizes.

def workload_pr1():
    """p=2, s=4, m=12 (N=4096): C_1 = J, C_2..C_4 random upper-triangular with
    unit diagonal; f(x) = prod_j (1 + (x_j - 1/2)/j) in FP64; one function."""
    p, m, s = 2, 12, 4
    C = np.empty((s, m, m), dtype=np.uint8)
    C[0] = reversed_identity(m)
    C[1:] = upper_triangular_matrices(p, m, s - 1, stream_seed(0, P_MATRICES))
    coef = 1.0 / np.arange(1, s + 1, dtype=np.float64)
    return dict(name="pr1_p2_m12_s4", p=p, m=m, s=s, C=C, coef=coef[None, :], batch=1)


def workload_p2_m20(batch_f32=32, batch_i32=32):
    """p=2, s=16, m=20: 32 FP32 product functions with c_j ~ U(0,1) and
    32 int32 arrays with values uniform in {-1000..1000}."""
    p, m, s = 2, 20, 16
    C = upper_triangular_matrices(p, m, s, stream_seed(2, P_MATRICES))
    coef = uniform(stream_seed(2, P_COEFFS), batch_f32 * s).reshape(batch_f32, s)
    return dict(name="p2_m20_s16", p=p, m=m, s=s, C=C, coef=coef, batch=batch_f32,
                batch_i32=batch_i32, int_seed=stream_seed(2, P_INTS))


def int_values(seed, batch, N, lo=-1000, hi=1000):
    """``batch`` int32 arrays of length N, uniform in [lo, hi]."""
    return integers(seed, batch * N, lo, hi).astype(np.int32).reshape(batch, N)


def workload_p3_m13():
    """p=3, s=8, m=13 (N=1,594,323): random nonsingular upper-triangular
    matrices over F_3; f(x) = exp(sum_j x_j / j^2), real FP32 in."""
    p, m, s = 3, 13, 8
    C = upper_triangular_matrices(p, m, s, stream_seed(3, P_MATRICES))
    return dict(name="p3_m13_s8", p=p, m=m, s=s, C=C, batch=1)


def workload_p2_m24(batch=32):
    """p=2, s=32, m=24 (N=16,777,216): batch of FP32 product functions
    f(x) = prod_j (1 + (x_j - 1/2)/j^2); weight prod_j (1+k_j)^-2."""
    p, m, s = 2, 24, 32
    C = upper_triangular_matrices(p, m, s, stream_seed(4, P_MATRICES))
    coef = np.tile(1.0 / np.arange(1, s + 1, dtype=np.float64) ** 2, (batch, 1))
    return dict(name="p2_m24_s32_b%d" % batch, p=p, m=m, s=s, C=C, coef=coef, batch=batch)


def small_net(p, m, s, index=0, config=9):
    """A seeded random upper-triangular net for small tests."""
    return upper_triangular_matrices(p, m, s, stream_seed(config, P_MATRICES, index))


def dense_matrices(p, m, s, index=0, config=10):
    """Seeded dense random matrices over F_p (may be singular): for index-map tests."""
    v = integers(stream_seed(config, P_MATRICES, index), s * m * m, 0, p - 1)
    return v.astype(np.uint8).reshape(s, m, m)


def sample_indices(count, N, index=0, config=11):
    """``count`` distinct-ish sample positions in [0, N) (always includes 0 and N-1)."""
    v = integers(stream_seed(config, P_SAMPLE, index), count, 0, N - 1).astype(np.uint32)
    v[0] = 0
    if count > 1:
        v[-1] = N - 1
    return v


def serving_requests(count, config=5, first=0):
    """The serving mix: p uniform in {2, 3, 5}; log2 N uniform in [10, 22], m = round(log_p N)
    clamped to 10..22 (p=2), 7..13 (p=3), 5..9 (p=5); s uniform in 2..64; each request has its
    own seeded upper-triangular net (seed = request id) and product-function coefficients
    c_j ~ U(0,1).  Returns a list of dicts (p, m, s, C, coef)."""
    out = []
    lim = {2: (10, 22), 3: (7, 13), 5: (5, 9)}
    for r in range(first, first + count):
        u = uniform(stream_seed(config, P_SERVE, r), 3)
        p = (2, 3, 5)[min(2, int(u[0] * 3))]
        log2n = 10.0 + 12.0 * u[1]
        m = int(round(log2n / np.log2(p)))
        m = max(lim[p][0], min(lim[p][1], m))
        s = 2 + min(62, int(u[2] * 63))
        C = upper_triangular_matrices(p, m, s, stream_seed(config, P_MATRICES, r))
        coef = uniform(stream_seed(config, P_COEFFS, r), s)
        out.append(dict(id=r, p=p, m=m, s=s, C=C, coef=coef))
    return out


def poisson_arrivals(count, rate, config=5):
    """Arrival times (seconds) of a Poisson process of the given rate."""
    u = uniform(stream_seed(config, P_SERVE, 1 << 30), count)
    return np.cumsum(-np.log1p(-u) / rate)
