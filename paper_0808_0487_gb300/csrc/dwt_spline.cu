// dwt_spline.cu -- the kernel spline of Sec. 3.1 and the variances of its
// ANOVA effects (Sec. 4), in FP64.
//
// The reproducing kernel K(x, y) = prod_j (1 + gamma_j K'(x_j (-) y_j, 0)) has
// Walsh coefficients supported on all wavenumbers, and its data at the net
// points aliases them onto the cosets: K~(H) = DWT of (K(x_n, 0))_n.  The
// interpolation conditions f(x_n) = sum_v c_v K(x_n (-) x_v, 0) are diagonal
// in the Walsh basis (eq. splinecoef): c~(H) = f~(H) / (p^m K~(H)), and
// c = FIWT(c~) (Algorithm 2).  With R'(x, 0) = int K'(t, x) K'(t, 0) dt and
// R_d = prod_{j <= d} (1 + gamma_j^2 R'), eq. sig2sfu summed over the nonempty
// u within 1..d gives
//     sigma^2_trc(d) = p^{2m} sum_H |c~(H)|^2 (R~_d(H) - [H = 0]),
// and over |u| = j the degree-j part E_j = sum_{|u| = j} gamma_u^2 R_u of
// R_s = prod_j (1 + gamma_j^2 R'), built point by point with the recurrence
// of elementary symmetric polynomials, gives
//     sigma^2_sup(d) = p^{2m} sum_H |c~(H)|^2 sum_{j <= d} E~_j(H).
// The constant effect (u = {}, the squared mean) is not a variance and is
// left out; the K' and R' values come from their short forms (Sec. 4).
//
// dwt_spline_prepare builds, once per (alpha, gamma), the kernel data at the
// net points, its 1 + 2s DWTs, and keeps W_K = 1 / (p^m K~) and the 2s
// variance tables (real parts: the kernels are real and symmetric, so their
// DWTs are real up to rounding).  dwt_spline then transforms each function,
// multiplies by W_K, transforms back, and contracts |c~|^2 with the tables in
// a fixed summation order.
#include <math.h>

#include <algorithm>
#include <vector>

#include "dwt_internal.cuh"

namespace dwt {

namespace {

constexpr int kSplineMaxS = 64;
constexpr int kDotTile = 4096;   // labels per block of the variance contraction

// kernel data at point n: K, R_1..R_s, E_1..E_s (rows of `out`, ld N)
__global__ void k_spline_data(const uint32_t* __restrict__ Y, long long N, int s, int p, int m,
                              const double* __restrict__ kp, const double* __restrict__ rp,
                              const double* __restrict__ gam, double* out) {
    double e[kSplineMaxS + 1];
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        double kv = 1.0, rv = 1.0;
        e[0] = 1.0;
        for (int q = 1; q <= s; ++q) e[q] = 0.0;
        for (int j = 0; j < s; ++j) {
            uint32_t y = Y[(long long)j * N + n];
            int i = 0;   // position of the first nonzero base-p digit of x = y / p^m
            if (y) {
                int t = 0;
                while (y >= (uint32_t)p) {
                    y /= (uint32_t)p;
                    ++t;
                }
                i = m - t;
            }
            kv *= 1.0 + gam[j] * kp[i];
            const double a = gam[j] * gam[j] * rp[i];
            rv *= 1.0 + a;
            out[(long long)(1 + j) * N + n] = rv;
            for (int q = j + 1; q >= 1; --q) e[q] += a * e[q - 1];
        }
        out[n] = kv;
        for (int q = 1; q <= s; ++q) out[(long long)(s + q) * N + n] = e[q];
    }
}

// real parts of the 1 + 2s transforms (interleaved complex when cplx) ->
// W_K = 1 / (N Re K~) and the tables, with R~_d(0) - 1
__global__ void k_spline_tables(const double* __restrict__ tr, int cplx, long long N, int s, double* W,
                                double* tab) {
    const long long total = (long long)(1 + 2 * s) * N;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        const long long row = x / N, H = x - row * N;
        const double v = cplx ? tr[2 * x] : tr[x];
        if (row == 0) {
            W[H] = 1.0 / ((double)N * v);
        } else {
            tab[x - N] = (row <= s && H == 0) ? v - 1.0 : v;
        }
    }
}

// c~ = f~ W_K in place ([batch][N], real or interleaved complex)
__global__ void k_spline_scale(double* ft, int cplx, long long N, long long total, const double* __restrict__ W) {
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        const double w = W[x % N];
        if (cplx) {
            ft[2 * x] *= w;
            ft[2 * x + 1] *= w;
        } else {
            ft[x] *= w;
        }
    }
}

// partial sums of |c~(H)|^2 T_t(H) over one tile of labels, for all 2s tables:
// part[(b * 2s + t) * ntile + tile]; per thread in label order, then a fixed
// tree.  Consecutive blocks take the same tile for consecutive functions, so a
// tile's table rows come from HBM once and from L2 for the other functions.
__global__ void __launch_bounds__(256) k_spline_dots(const double* __restrict__ ct, int cplx, long long N, int nt,
                                                     const double* __restrict__ tab, double* part, long long ntile,
                                                     long long tile0) {
    __shared__ double red[256];
    const long long tile = tile0 + blockIdx.y, b = blockIdx.x;
    const long long h0 = tile * kDotTile;
    const int t = threadIdx.x;
    constexpr int PER = kDotTile / 256;
    double a[PER];
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const long long H = h0 + t + 256 * q;
        double v = 0.0;
        if (H < N) {
            const long long x = b * N + H;
            v = cplx ? ct[2 * x] * ct[2 * x] + ct[2 * x + 1] * ct[2 * x + 1] : ct[x] * ct[x];
        }
        a[q] = v;
    }
    for (int tb = 0; tb < nt; ++tb) {
        const double* T = tab + (long long)tb * N;
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < PER; ++q) {
            const long long H = h0 + t + 256 * q;
            if (H < N) acc += a[q] * T[H];
        }
        red[t] = acc;
        __syncthreads();
        for (int w = 128; w > 0; w >>= 1) {
            if (t < w) red[t] += red[t + w];
            __syncthreads();
        }
        if (t == 0) part[(b * nt + tb) * ntile + tile] = red[0];
        __syncthreads();
    }
}

// sums over tiles in tile order, then the cumulative variances and dimensions
// (least d with variance >= thr * total, 0 when the total is 0)
__global__ void k_spline_finalize(const double* __restrict__ part, long long ntile, int s, int batch, double N2,
                                  double thr, double* var_trc, double* var_sup, int* dim) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    const int nt = 2 * s;
    double vt[kSplineMaxS + 1], vs[kSplineMaxS + 1];
    vt[0] = vs[0] = 0.0;
    for (int d = 1; d <= s; ++d) {
        double x = 0.0, y = 0.0;
        const double* pr = part + ((long long)b * nt + (d - 1)) * ntile;
        const double* pe = part + ((long long)b * nt + (s + d - 1)) * ntile;
        for (long long i = 0; i < ntile; ++i) {
            x += pr[i];
            y += pe[i];
        }
        vt[d] = N2 * x;
        vs[d] = vs[d - 1] + N2 * y;
    }
    for (int d = 0; d <= s; ++d) {
        if (var_trc) var_trc[(long long)b * (s + 1) + d] = vt[d];
        if (var_sup) var_sup[(long long)b * (s + 1) + d] = vs[d];
    }
    if (dim) {
        const double tot = vt[s];
        int dt = 0, ds = 0;
        if (tot > 0.0) {
            dt = ds = s;
            for (int d = s; d >= 0; --d) {
                if (vt[d] >= thr * tot) dt = d;
                if (vs[d] >= thr * tot) ds = d;
            }
        }
        dim[2 * b] = dt;
        dim[2 * b + 1] = ds;
    }
}

// kernel data at the shifted points: Kd[w] = prod_j (1 + gamma_j K'(x_{j,w} (+) delta_j, 0)),
// x_{j,w} with m digits, delta_j = D[j] / p^M with M digits; kpM[i] = K' for a first
// nonzero digit at position i of M (kpM[0] = 1)
__global__ void k_spline_shift_data(const uint32_t* __restrict__ Y, long long N, int s, int p, int m, int M,
                                    const uint32_t* __restrict__ D, const double* __restrict__ kpM,
                                    const double* __restrict__ gam, double* Kd) {
    unsigned long long up = 1;
    for (int i = m; i < M; ++i) up *= (unsigned long long)p;
    for (long long w = blockIdx.x * (long long)blockDim.x + threadIdx.x; w < N; w += (long long)gridDim.x * blockDim.x) {
        double kv = 1.0;
        for (int j = 0; j < s; ++j) {
            unsigned long long a = (unsigned long long)Y[(long long)j * N + w] * up, b = D[j], y;
            if (p == 2) {
                y = a ^ b;
            } else {
                y = 0;
                unsigned long long pw = 1;
                for (int c = 0; c < M; ++c) {
                    y += ((a % p + b % p) % p) * pw;
                    a /= p;
                    b /= p;
                    pw *= p;
                }
            }
            int i = 0;
            if (y) {
                int t = 0;
                while (y >= (unsigned long long)p) {
                    y /= p;
                    ++t;
                }
                i = M - t;
            }
            kv *= 1.0 + gam[j] * kpM[i];
        }
        Kd[w] = kv;
    }
}

// g~ = N c~ k~ in place in c~ (real, or interleaved complex with k~ complex)
__global__ void k_spline_conv(double* ct, const double* __restrict__ kt, int cplx, long long N, long long total) {
    const double n = (double)N;
    for (long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x; x < total;
         x += (long long)gridDim.x * blockDim.x) {
        const long long H = x % N;
        if (cplx) {
            const double ar = ct[2 * x], ai = ct[2 * x + 1], br = kt[2 * H], bi = kt[2 * H + 1];
            ct[2 * x] = n * (ar * br - ai * bi);
            ct[2 * x + 1] = n * (ar * bi + ai * br);
        } else {
            ct[x] *= n * kt[H];
        }
    }
}

// per-block partial sums of (f - Re v)^2 over a tile of points; part[b * ntile + tile]
__global__ void __launch_bounds__(256) k_spline_sse(const double* __restrict__ f, const double* __restrict__ v,
                                                    int cplx, long long N, long long ld, double* part,
                                                    long long ntile) {
    __shared__ double red[256];
    const long long tile = blockIdx.x, b = blockIdx.y;
    double acc = 0.0;
    for (int q = 0; q < kDotTile / 256; ++q) {
        const long long n = tile * kDotTile + threadIdx.x + 256 * q;
        if (n < N) {
            const long long x = b * ld + n;
            const double d = f[x] - (cplx ? v[2 * x] : v[x]);
            acc += d * d;
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[b * ntile + tile] = red[0];
}

__global__ void k_spline_sse_final(const double* __restrict__ part, long long ntile, int batch, double* sse) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= batch) return;
    double x = 0.0;
    for (long long i = 0; i < ntile; ++i) x += part[(long long)b * ntile + i];
    sse[b] = x;
}

// ---- the spline at arbitrary points (Sec. 3.1) ----------------------------
// K(x (-) x_n, 0) = prod_j (1 + gamma_j K'(x_j (-) x_{j,n}, 0)), and K' depends
// only on the position i of the first nonzero digit of the difference: the
// first digit (of m) where x_j and the net point differ, or, when the top m
// digits agree, the first nonzero digit of x_j below them (0 if none).  With
// the base-p digits packed BP bits each (1, 2, 3, 4, 5 bits for p = 2, 3, 5 / 7,
// 11 / 13, 17 .. 31), the first differing digit is the highest set bit of an XOR.
constexpr int kEvalQB = 128;   // points per block, one per thread
constexpr int kEvalFB = 8;     // functions per block

__host__ __device__ inline int eval_bits(int p) { return p == 2 ? 1 : p == 3 ? 2 : p <= 7 ? 3 : p <= 15 ? 4 : 5; }

__device__ __forceinline__ unsigned long long pack_digits(uint32_t v, int p, int m, int bp) {
    unsigned long long r = 0;
    for (int k = 0; k < m; ++k) {
        r |= (unsigned long long)(v % (uint32_t)p) << (bp * k);
        v /= (uint32_t)p;
    }
    return r;
}

// packed top-m digits of the net points, [s][N]
__global__ void k_eval_pack(const uint32_t* __restrict__ Y, long long total, int p, int m,
                            unsigned long long* __restrict__ PY) {
    const int bp = eval_bits(p);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x)
        PY[e] = p == 2 ? (unsigned long long)Y[e] : pack_digits(Y[e], p, m, bp);
}

// Partial sums over one chunk of the net (blockIdx.z) for kEvalQB points
// (blockIdx.x) and kEvalFB functions (blockIdx.y):
//   part[z][f][q] = sum_{n in chunk} Re c[f][n] prod_j T[j][i_j(q, n)],
// T[j][i] = 1 + gamma_j K'(i) (i = 0 .. M).  The net points and coefficients
// of the chunk pass through shared memory in tiles of TN; each thread keeps
// its point's packed digits and tail positions in shared memory too.
template <int P>
__global__ void __launch_bounds__(kEvalQB) k_spline_eval(const unsigned long long* __restrict__ PY, long long N,
                                                          const double* __restrict__ c, long long ldc, int cstride,
                                                          int batch, const uint32_t* __restrict__ X, int Q, int s,
                                                          int m, int M, const double* __restrict__ Tg,
                                                          long long chunk, int TN, double* __restrict__ part) {
    constexpr int p = P;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int M1 = M + 1;
    double* T = reinterpret_cast<double*>(smraw);                                   // [s][M+1]
    unsigned long long* PX = reinterpret_cast<unsigned long long*>(T + (size_t)s * M1);   // [s][QB]
    unsigned long long* PYs = PX + (size_t)s * kEvalQB;                             // [s][TN]
    double* cs = reinterpret_cast<double*>(PYs + (size_t)s * TN);                   // [FB][TN]
    unsigned char* tl = reinterpret_cast<unsigned char*>(cs + (size_t)kEvalFB * TN);   // [s][QB]
    const int t = threadIdx.x;
    const int q = blockIdx.x * kEvalQB + t;
    const int f0 = blockIdx.y * kEvalFB;
    const int nf = min(kEvalFB, batch - f0);
    constexpr int bp = P == 2 ? 1 : P == 3 ? 2 : P <= 7 ? 3 : P <= 15 ? 4 : 5;   // eval_bits(P)
    for (int e = t; e < s * M1; e += blockDim.x) T[e] = Tg[e];
    {
        uint32_t up = 1;
        for (int k = 0; k < M - m; ++k) up *= (uint32_t)p;
        for (int j = 0; j < s; ++j) {
            const uint32_t x = q < Q ? X[(long long)q * s + j] : 0u;
            const uint32_t top = up > 1 ? x / up : x, tail = up > 1 ? x % up : 0u;
            PX[j * kEvalQB + t] = p == 2 ? (unsigned long long)top : pack_digits(top, p, m, bp);
            int tp = 0;   // first nonzero digit of the tail, as a position in 1..M
            if (tail) {
                int e = 0;
                for (uint32_t v = tail; v >= (uint32_t)p; v /= (uint32_t)p) ++e;
                tp = M - e;
            }
            tl[j * kEvalQB + t] = (unsigned char)tp;
        }
    }
    double acc[kEvalFB];
#pragma unroll
    for (int f = 0; f < kEvalFB; ++f) acc[f] = 0.0;
    const long long n0 = blockIdx.z * chunk, n1 = min(N, n0 + chunk);
    for (long long nb = n0; nb < n1; nb += TN) {
        const int tn = (int)min((long long)TN, n1 - nb);
        __syncthreads();   // the previous tile is consumed (and the tables above are written)
        for (int e = t; e < s * TN; e += blockDim.x) {
            const int j = e / TN, u = e - j * TN;
            PYs[e] = u < tn ? PY[(long long)j * N + nb + u] : 0ull;
        }
        for (int e = t; e < kEvalFB * TN; e += blockDim.x) {
            const int f = e / TN, u = e - f * TN;
            cs[e] = (f < nf && u < tn) ? c[(long long)(f0 + f) * ldc + (nb + u) * cstride] : 0.0;
        }
        __syncthreads();
        for (int u = 0; u < tn; ++u) {
            // two partial products (even and odd coordinates) keep two
            // multiplication chains in flight
            double pr0 = 1.0, pr1 = 1.0;
            int j = 0;
            for (; j + 1 < s; j += 2) {
                const unsigned long long d0 = PX[j * kEvalQB + t] ^ PYs[j * TN + u];
                const unsigned long long d1 = PX[(j + 1) * kEvalQB + t] ^ PYs[(j + 1) * TN + u];
                const int i0 = d0 ? m - (63 - __clzll((long long)d0)) / bp : (int)tl[j * kEvalQB + t];
                const int i1 = d1 ? m - (63 - __clzll((long long)d1)) / bp : (int)tl[(j + 1) * kEvalQB + t];
                pr0 *= T[j * M1 + i0];
                pr1 *= T[(j + 1) * M1 + i1];
            }
            if (j < s) {
                const unsigned long long d0 = PX[j * kEvalQB + t] ^ PYs[j * TN + u];
                const int i0 = d0 ? m - (63 - __clzll((long long)d0)) / bp : (int)tl[j * kEvalQB + t];
                pr0 *= T[j * M1 + i0];
            }
            const double prod = pr0 * pr1;
#pragma unroll
            for (int f = 0; f < kEvalFB; ++f) acc[f] = fma(cs[f * TN + u], prod, acc[f]);
        }
    }
    if (q < Q) {
        for (int f = 0; f < nf; ++f) part[((long long)blockIdx.z * batch + f0 + f) * Q + q] = acc[f];
    }
}

// values[f][q] = sum over the chunks in order
__global__ void k_spline_eval_reduce(const double* __restrict__ part, int nch, int batch, int Q,
                                     double* __restrict__ values, long long ldv) {
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= (long long)batch * Q) return;
    const long long f = e / Q, q = e - f * Q;
    double a = 0.0;
    for (int z = 0; z < nch; ++z) a += part[(long long)z * batch * Q + e];
    values[f * ldv + q] = a;
}

unsigned grid_sp(long long n) { return (unsigned)std::max(1ll, std::min((n + 255) / 256, 8ll * 152)); }

}  // namespace

void spline_free(dwt_plan_s* P, cudaStream_t st, bool sync) {
    if (sync) {
        cudaFree(P->d_splW);
        cudaFree(P->d_splT);
    } else {
        dfree(P->d_splW, st);
        dfree(P->d_splT, st);
    }
    P->d_splW = nullptr;
    P->d_splT = nullptr;
}

int run_spline_prepare(dwt_plan_s* P, double alpha, const double* gamma, cudaStream_t st) {
    const long long N = P->N;
    const int s = P->s, p = P->p, m = P->m;
    if (s > kSplineMaxS) {
        set_error("the kernel spline supports s <= %d", kSplineMaxS);
        return DWT_EUNSUPPORTED;
    }
    // K'(x, 0) and R'(x, 0) by the position i (1..m) of the first nonzero digit; i = 0 for x = 0
    std::vector<double> hv(3 * (m + 1) + s);
    const double pa = std::pow((double)p, alpha), p2a = std::pow((double)p, 2.0 * alpha);
    const double rc = (pa - p) * (pa - p) / ((p - 1.0) * (p2a - p));
    for (int i = 0; i <= m; ++i) {
        hv[i] = i == 0 ? 1.0 : 1.0 - std::pow((double)p, i * (1.0 - alpha)) * (pa - 1.0) / (p - 1.0);
        hv[m + 1 + i] = i == 0 ? rc : rc * (1.0 - std::pow((double)p, i * (1.0 - 2.0 * alpha)) * (p2a - 1.0) / (p - 1.0));
    }
    for (int j = 0; j < s; ++j) hv[2 * (m + 1) + j] = gamma[j];
    const int rows = 1 + 2 * s;
    const bool cplx = p != 2;
    uint32_t* Y = nullptr;
    double *dv = nullptr, *data = nullptr, *tr = nullptr;
    auto cleanup = [&]() {
        dfree(Y, st);
        dfree(dv, st);
        dfree(data, st);
        if (tr != data) dfree(tr, st);
    };
    if (dmalloc((void**)&Y, (size_t)s * N * 4, st) || dmalloc((void**)&dv, hv.size() * 8, st) ||
        dmalloc((void**)&data, (size_t)rows * N * 8, st)) {
        cleanup();
        return DWT_ENOMEM;
    }
    tr = data;
    if (cplx && dmalloc((void**)&tr, (size_t)rows * N * 16, st)) {
        tr = data;
        cleanup();
        return DWT_ENOMEM;
    }
    DWT_CK(cudaMemcpyAsync(dv, hv.data(), hv.size() * 8, cudaMemcpyHostToDevice, st));
    int rc2 = run_points(P, Y, N, st);
    if (rc2) { cleanup(); return rc2; }
    {
        LaunchScope ls("spline_data", st);
        k_spline_data<<<grid_sp(N), 128, 0, st>>>(Y, N, s, p, m, dv, dv + m + 1, dv + 2 * (m + 1), data);
    }
    DWT_CK_LAUNCH("k_spline_data");
    rc2 = run_transform(P, data, tr, rows, N, N, DWT_F64, cplx ? DWT_C128 : DWT_F64, -1, st);
    if (rc2) { cleanup(); return rc2; }
    spline_free(P, st, false);
    P->spl_alpha = alpha;
    P->spl_gamma.assign(gamma, gamma + s);
    if (dmalloc((void**)&P->d_splW, (size_t)N * 8, st) || dmalloc((void**)&P->d_splT, (size_t)2 * s * N * 8, st)) {
        spline_free(P, st, false);
        cleanup();
        return DWT_ENOMEM;
    }
    {
        LaunchScope ls("spline_tables", st);
        k_spline_tables<<<grid_sp((long long)rows * N), 256, 0, st>>>(tr, cplx ? 1 : 0, N, s, P->d_splW, P->d_splT);
    }
    DWT_CK_LAUNCH("k_spline_tables");
    cleanup();
    return DWT_OK;
}

int run_spline_shifted(dwt_plan_s* P, const void* c, const uint32_t* delta, int M, void* values, int batch,
                       long long ld, const double* f_shift, double* sse, cudaStream_t st) {
    if (!P->d_splW) {
        set_error("dwt_spline_values_shifted: no kernel tables (call dwt_spline_prepare first)");
        return DWT_EINVAL;
    }
    const long long N = P->N;
    const int s = P->s, p = P->p, m = P->m;
    if (M < m || (double)M * std::log2((double)p) > 32.0) {
        set_error("dwt_spline_values_shifted: need m <= M and p^M <= 2^32");
        return DWT_EINVAL;
    }
    const bool cplx = p != 2;
    const size_t eb = cplx ? 16 : 8;
    // K'(y, 0) on M digits by the first nonzero digit, and the kernel weights
    const double alpha = P->spl_alpha;
    const double pa = std::pow((double)p, alpha);
    std::vector<double> hv((size_t)M + 1 + s);
    for (int i = 0; i <= M; ++i)
        hv[i] = i == 0 ? 1.0 : 1.0 - std::pow((double)p, i * (1.0 - alpha)) * (pa - 1.0) / (p - 1.0);
    for (int j = 0; j < s; ++j) hv[M + 1 + j] = P->spl_gamma[j];
    uint32_t *Y = nullptr, *dD = nullptr;
    double *dv = nullptr, *kd = nullptr, *kt = nullptr, *ct = nullptr, *part = nullptr;
    auto cleanup = [&]() {
        dfree(Y, st); dfree(dD, st); dfree(dv, st); dfree(kd, st); dfree(kt, st); dfree(ct, st); dfree(part, st);
    };
    const long long ntile = (N + kDotTile - 1) / kDotTile;
    if (dmalloc((void**)&Y, (size_t)s * N * 4, st) || dmalloc((void**)&dD, (size_t)s * 4, st) ||
        dmalloc((void**)&dv, hv.size() * 8, st) || dmalloc((void**)&kd, (size_t)N * 8, st) ||
        dmalloc((void**)&kt, (size_t)N * eb, st) || dmalloc((void**)&ct, (size_t)batch * N * eb, st) ||
        (sse && f_shift && dmalloc((void**)&part, (size_t)batch * ntile * 8, st))) {
        cleanup();
        return DWT_ENOMEM;
    }
    DWT_CK(cudaMemcpyAsync(dv, hv.data(), hv.size() * 8, cudaMemcpyHostToDevice, st));
    DWT_CK(cudaMemcpyAsync(dD, delta, (size_t)s * 4, cudaMemcpyHostToDevice, st));
    int rc = run_points(P, Y, N, st);
    if (rc) { cleanup(); return rc; }
    {
        LaunchScope ls("spline_shift_data", st);
        k_spline_shift_data<<<grid_sp(N), 128, 0, st>>>(Y, N, s, p, m, M, dD, dv, dv + M + 1, kd);
    }
    DWT_CK_LAUNCH("k_spline_shift_data");
    const dwt_dtype ct_t = cplx ? DWT_C128 : DWT_F64;
    if ((rc = run_transform(P, kd, kt, 1, N, N, DWT_F64, ct_t, -1, st)) ||
        (rc = run_transform(P, c, ct, batch, ld, N, ct_t, ct_t, -1, st))) {
        cleanup();
        return rc;
    }
    {
        LaunchScope ls("spline_conv", st);
        k_spline_conv<<<grid_sp((long long)batch * N), 256, 0, st>>>(ct, kt, cplx ? 1 : 0, N, (long long)batch * N);
    }
    DWT_CK_LAUNCH("k_spline_conv");
    if ((rc = run_transform(P, ct, values, batch, N, ld, ct_t, ct_t, +1, st))) {
        cleanup();
        return rc;
    }
    if (sse && f_shift) {
        for (int b0 = 0; b0 < batch; b0 += 65535) {
            const int nb = std::min(65535, batch - b0);
            LaunchScope ls("spline_sse", st);
            k_spline_sse<<<dim3((unsigned)ntile, (unsigned)nb), 256, 0, st>>>(
                f_shift + (size_t)b0 * ld, reinterpret_cast<const double*>(values) + (size_t)b0 * ld * (eb / 8),
                cplx ? 1 : 0, N, ld, part + (size_t)b0 * ntile, ntile);
        }
        LaunchScope ls("spline_sse", st);
        k_spline_sse_final<<<(batch + 127) / 128, 128, 0, st>>>(part, ntile, batch, sse);
    }
    DWT_CK_LAUNCH("k_spline_sse");
    cleanup();
    return DWT_OK;
}

int run_spline_eval(dwt_plan_s* P, const void* c, int batch, long long ld, const uint32_t* X, int Q, int M,
                    double* values, long long ldv, cudaStream_t st) {
    if (!P->d_splW) {
        set_error("dwt_spline_eval: no kernel (call dwt_spline_prepare first)");
        return DWT_EINVAL;
    }
    const long long N = P->N;
    const int s = P->s, p = P->p, m = P->m;
    if (M < m || (double)M * std::log2((double)p) > 32.0) {
        set_error("dwt_spline_eval: need m <= M and p^M <= 2^32");
        return DWT_EINVAL;
    }
    if (Q == 0) return DWT_OK;
    // T[j][i] = 1 + gamma_j K'(i) on M digits
    const double alpha = P->spl_alpha;
    const double pa = std::pow((double)p, alpha);
    std::vector<double> hT((size_t)s * (M + 1));
    for (int j = 0; j < s; ++j)
        for (int i = 0; i <= M; ++i) {
            const double kp = i == 0 ? 1.0 : 1.0 - std::pow((double)p, i * (1.0 - alpha)) * (pa - 1.0) / (p - 1.0);
            hT[(size_t)j * (M + 1) + i] = 1.0 + P->spl_gamma[j] * kp;
        }
    // tiles of the net: TN points, within the shared-memory budget
    const int TN = s > 32 ? 64 : 128;
    const size_t smem = (size_t)s * (M + 1) * 8 + (size_t)s * kEvalQB * 8 + (size_t)s * TN * 8 +
                        (size_t)kEvalFB * TN * 8 + (size_t)s * kEvalQB;
    int dev = 0, sms = 0;
    DWT_CK(cudaGetDevice(&dev));
    DWT_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int qb = (Q + kEvalQB - 1) / kEvalQB, fb = (batch + kEvalFB - 1) / kEvalFB;
    const long long ntn = (N + TN - 1) / TN;
    long long nch = std::max(1ll, std::min(ntn, (4ll * sms + (long long)qb * fb - 1) / ((long long)qb * fb)));
    nch = std::min(nch, 65535ll);
    const long long chunk = (ntn + nch - 1) / nch * TN;
    nch = (N + chunk - 1) / chunk;
    if (fb > 65535 || qb > (1 << 30)) {
        set_error("dwt_spline_eval: too many functions in one call");
        return DWT_EINVAL;
    }
    uint32_t* Y = nullptr;
    unsigned long long* PY = nullptr;
    double *dT = nullptr, *part = nullptr;
    auto cleanup = [&]() { dfree(Y, st); dfree(PY, st); dfree(dT, st); dfree(part, st); };
    if (dmalloc((void**)&Y, (size_t)s * N * 4, st) || dmalloc((void**)&PY, (size_t)s * N * 8, st) ||
        dmalloc((void**)&dT, hT.size() * 8, st) || dmalloc((void**)&part, (size_t)nch * batch * Q * 8, st)) {
        cleanup();
        return DWT_ENOMEM;
    }
    DWT_CK(cudaMemcpyAsync(dT, hT.data(), hT.size() * 8, cudaMemcpyHostToDevice, st));
    int rc = run_points(P, Y, N, st);
    if (rc) { cleanup(); return rc; }
    {
        LaunchScope ls("spline_eval_pack", st);
        k_eval_pack<<<grid_sp((long long)s * N), 256, 0, st>>>(Y, (long long)s * N, p, m, PY);
    }
    DWT_CK_LAUNCH("k_eval_pack");
    {
        auto kern = k_spline_eval<2>;
        switch (p) {
            case 3: kern = k_spline_eval<3>; break;
            case 5: kern = k_spline_eval<5>; break;
            case 7: kern = k_spline_eval<7>; break;
            case 11: kern = k_spline_eval<11>; break;
            case 13: kern = k_spline_eval<13>; break;
            case 17: kern = k_spline_eval<17>; break;
            case 19: kern = k_spline_eval<19>; break;
            case 23: kern = k_spline_eval<23>; break;
            case 29: kern = k_spline_eval<29>; break;
            case 31: kern = k_spline_eval<31>; break;
            default: break;
        }
        if ((rc = smem_limit_max(kern))) { cleanup(); return rc; }
        LaunchScope ls("spline_eval", st);
        kern<<<dim3((unsigned)qb, (unsigned)fb, (unsigned)nch), kEvalQB, smem, st>>>(
            PY, N, reinterpret_cast<const double*>(c), (p == 2 ? 1 : 2) * ld, p == 2 ? 1 : 2, batch, X, Q, s, m, M,
            dT, chunk, TN, part);
    }
    DWT_CK_LAUNCH("k_spline_eval");
    {
        LaunchScope ls("spline_eval_reduce", st);
        const long long tot = (long long)batch * Q;
        k_spline_eval_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(part, (int)nch, batch, Q, values, ldv);
    }
    DWT_CK_LAUNCH("k_spline_eval_reduce");
    cleanup();
    return DWT_OK;
}

int run_spline(dwt_plan_s* P, const double* f, void* c, int batch, long long ld, double* var_trc, double* var_sup,
               int* dim, double thr, cudaStream_t st) {
    if (!P->d_splW) {
        set_error("dwt_spline: no kernel tables (call dwt_spline_prepare first)");
        return DWT_EINVAL;
    }
    const long long N = P->N;
    const int s = P->s;
    const bool cplx = P->p != 2;
    const size_t eb = cplx ? 16 : 8;
    double* ft = nullptr;
    double* part = nullptr;
    const long long ntile = (N + kDotTile - 1) / kDotTile;
    const bool want_var = var_trc || var_sup || dim;
    if (dmalloc((void**)&ft, (size_t)batch * N * eb, st) ||
        (want_var && dmalloc((void**)&part, (size_t)batch * 2 * s * ntile * 8, st))) {
        dfree(ft, st);
        return DWT_ENOMEM;
    }
    auto cleanup = [&]() {
        dfree(ft, st);
        dfree(part, st);
    };
    int rc = run_transform(P, f, ft, batch, ld, N, DWT_F64, cplx ? DWT_C128 : DWT_F64, -1, st);
    if (rc) { cleanup(); return rc; }
    {
        LaunchScope ls("spline_scale", st);
        k_spline_scale<<<grid_sp((long long)batch * N), 256, 0, st>>>(ft, cplx ? 1 : 0, N, (long long)batch * N,
                                                                     P->d_splW);
    }
    DWT_CK_LAUNCH("k_spline_scale");
    if (want_var) {
        for (int b0 = 0; b0 < batch; b0 += 65535) {
            const int nb = std::min(65535, batch - b0);
            for (long long t0 = 0; t0 < ntile; t0 += 65535) {
                LaunchScope ls("spline_dots", st);
                k_spline_dots<<<dim3((unsigned)nb, (unsigned)std::min(65535ll, ntile - t0)), 256, 0, st>>>(
                    ft + (size_t)b0 * N * (eb / 8), cplx ? 1 : 0, N, 2 * s, P->d_splT, part + (size_t)b0 * 2 * s * ntile,
                    ntile, t0);
            }
        }
        DWT_CK_LAUNCH("k_spline_dots");
    }
    if (c) {
        rc = run_transform(P, ft, c, batch, N, ld, cplx ? DWT_C128 : DWT_F64, cplx ? DWT_C128 : DWT_F64, +1, st);
        if (rc) { cleanup(); return rc; }
    }
    if (want_var) {
        LaunchScope ls("spline_finalize", st);
        k_spline_finalize<<<(batch + 127) / 128, 128, 0, st>>>(part, ntile, s, batch, (double)N * (double)N, thr,
                                                               var_trc, var_sup, dim);
    }
    DWT_CK_LAUNCH("k_spline_finalize");
    cleanup();
    return DWT_OK;
}

}  // namespace dwt
