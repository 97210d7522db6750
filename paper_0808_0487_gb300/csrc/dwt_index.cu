// dwt_index.cu -- integer F_p kernels: net points (Def. 1.1), the wavenumber
// -> coset label map C . k (Sec. 2.1), the coset representatives K(C) with
// their weight and class tables (Sec. 2.1), and the synthetic test functions.
//
// Coset representatives.  For coordinate j let T_j[h] be the least
// nu(k_j)+...+nu(k_s) over wavenumbers of coordinates j..s whose label is h
// (T_{s+1} = 0 at h = 0, "infinite" elsewhere).  With R_{j,i} the label of row
// i of C_j, a k_j with nu(k_j) = d has its top nonzero digit at d-1 and free
// digits below, so with M_0 = T_{j+1}, M_{i+1}[h] = min_a M_i[h (-) a R_{j,i}]:
//     T_j[h] = min(T_{j+1}[h], min_d (d + min_{a != 0} M_{d-1}[h (-) a R_{j,d-1}])).
// The backward sweep runs one kernel per (j, i) over all h and also records
// D_j[h], the smallest optimal nu(k_j) (0 when k_j = 0 is optimal).  The
// representative of every coset is then read forward, coordinate by
// coordinate, taking the smallest integer k_j that keeps the least total:
// k_j = 0 if D_j = 0, else top digit and lower digits chosen smallest-first
// from the M arrays of that coordinate (rebuilt per coordinate).  That is the
// least-nu representative with the lexicographic tie-break of Sec. 2.1.
// Values are bytes; 255 stands for "unreachable or >= 255" and never lies on
// an optimal path whose total is below 255.
#include <algorithm>
#include <vector>

#include "dwt_internal.cuh"

namespace dwt {

static const uint8_t kInf = 255;

// h (-) a * r digitwise over F_p (labels as integers in base p)
template <int P>
__device__ __forceinline__ uint32_t dsub(uint32_t h, uint32_t r, int a, int m) {
    if constexpr (P == 2) {
        return a ? (h ^ r) : h;
    } else {
        uint32_t out = 0, pw = 1;
        for (int c = 0; c < m; ++c) {
            const int hc = (int)(h % P), rc = (int)(r % P);
            h /= P;
            r /= P;
            const int v = ((hc - a * rc) % P + P) % P;
            out += (uint32_t)v * pw;
            pw *= P;
        }
        return out;
    }
}

// ---------------------------------------------------------------------------
// net points: Y[j][n] = sum_i y_{j,n,i+1} p^{m-1-i}, y_{j,n} = C_j n
template <int P>
__global__ void k_points(const uint8_t* __restrict__ C, const uint32_t* __restrict__ col, int m, long long N,
                         uint32_t* Y, long long ldY) {
    const int j = blockIdx.y;
    __shared__ uint8_t Cj[32 * 32];
    __shared__ uint32_t colj[32];
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) Cj[t] = C[(size_t)j * m * m + t];
    for (int t = threadIdx.x; t < m; t += blockDim.x) colj[t] = col[(size_t)j * m + t];
    __syncthreads();
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        uint32_t Yv = 0;
        if constexpr (P == 2) {
            uint32_t v = (uint32_t)n;
            while (v) {
                const int c = __ffs(v) - 1;
                Yv ^= colj[c];
                v &= v - 1;
            }
        } else {
            int nd[32];
            uint32_t v = (uint32_t)n;
            for (int c = 0; c < m; ++c) {
                nd[c] = (int)(v % P);
                v /= P;
            }
            for (int i = 0; i < m; ++i) {
                int acc = 0;
                for (int c = 0; c < m; ++c) acc += Cj[i * m + c] * nd[c];
                Yv = Yv * P + (uint32_t)(acc % P);
            }
        }
        Y[(long long)j * ldY + n] = Yv;
    }
}

// H = C . k, k given as [cnt][s]
template <int P>
__global__ void k_k_to_h(const uint8_t* __restrict__ C, const uint32_t* __restrict__ R, int m, int s,
                         const uint32_t* __restrict__ k, uint32_t* H, long long cnt) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < cnt; t += (long long)gridDim.x * blockDim.x) {
        const uint32_t* kv = k + t * s;
        if constexpr (P == 2) {
            uint32_t h = 0;
            for (int j = 0; j < s; ++j) {
                uint32_t v = kv[j];
                for (int i = 0; i < m && v; ++i, v >>= 1)
                    if (v & 1) h ^= R[j * m + i];
            }
            H[t] = h;
        } else {
            uint32_t out = 0, pw = 1;
            for (int c = 0; c < m; ++c) {
                int acc = 0;
                for (int j = 0; j < s; ++j) {
                    uint32_t v = kv[j];
                    for (int i = 0; i < m && v; ++i) {
                        acc += (int)(v % P) * C[((size_t)j * m + i) * m + c];
                        v /= P;
                    }
                }
                out += (uint32_t)(acc % P) * pw;
                pw *= P;
            }
            H[t] = out;
        }
    }
}

// ---------------------------------------------------------------------------
// backward sweep, one (j, i): candidate nu(k_j) = i + 1
template <int P>
__global__ void k_dp_step(const uint8_t* __restrict__ Mcur, uint8_t* __restrict__ Mnext, uint8_t* Tj, uint8_t* Dj,
                          uint32_t r, int i, int m, long long N) {
    for (long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x; h < N; h += (long long)gridDim.x * blockDim.x) {
        unsigned e = kInf;
#pragma unroll
        for (int a = 1; a < P; ++a) {
            const unsigned v = Mcur[dsub<P>((uint32_t)h, r, a, m)];
            e = v < e ? v : e;
        }
        const unsigned cur = Mcur[h];
        Mnext[h] = (uint8_t)(e < cur ? e : cur);
        unsigned cand = e == kInf ? kInf : e + (unsigned)(i + 1);
        if (cand > kInf) cand = kInf;
        if (cand < Tj[h]) {
            Tj[h] = (uint8_t)cand;
            Dj[h] = (uint8_t)(i + 1);
        }
    }
}

// M_i from M_{i-1} for the reconstruction of one coordinate
template <int P>
__global__ void k_dp_prefix(const uint8_t* __restrict__ Mp, uint8_t* __restrict__ Mi, uint32_t r, int m, long long N) {
    for (long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x; h < N; h += (long long)gridDim.x * blockDim.x) {
        unsigned v = Mp[h];
#pragma unroll
        for (int a = 1; a < P; ++a) {
            const unsigned w = Mp[dsub<P>((uint32_t)h, r, a, m)];
            v = w < v ? w : v;
        }
        Mi[h] = (uint8_t)v;
    }
}

__global__ void k_max_byte(const uint8_t* __restrict__ a, long long N, unsigned* out) {
    unsigned mx = 0;
    for (long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x; h < N; h += (long long)gridDim.x * blockDim.x)
        mx = max(mx, (unsigned)a[h]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

struct Mptrs {
    const uint8_t* M[32];
};

// read k_j of every coset label (list) from the tables of coordinate j
template <int P>
__device__ __forceinline__ uint32_t recon_one(uint32_t& g, const uint8_t* Tj, const uint8_t* Dj, const Mptrs& Mp,
                                              const uint32_t* __restrict__ Rj, int m) {
    const unsigned tau = Tj[g];
    const int d = Dj[g];
    if (d == 0) return 0;
    uint32_t k = 0, pw = 1;
    for (int i = 0; i < d - 1; ++i) pw *= P;
    for (int i = d - 1; i >= 0; --i, pw /= P) {
        const uint8_t* Mi = Mp.M[i];
        for (int a = (i == d - 1) ? 1 : 0; a < P; ++a) {
            const uint32_t cand = dsub<P>(g, Rj[i], a, m);
            if ((unsigned)Mi[cand] + (unsigned)d == tau) {
                g = cand;
                k += (uint32_t)a * pw;
                break;
            }
        }
    }
    return k;
}

template <int P>
__global__ void k_recon_all(uint32_t* G, unsigned long long* Pden, uint8_t* cls, int* overflow, const uint8_t* Tj,
                            const uint8_t* Dj, Mptrs Mp, const uint32_t* Rj, int j, int m, long long N) {
    for (long long H = blockIdx.x * (long long)blockDim.x + threadIdx.x; H < N; H += (long long)gridDim.x * blockDim.x) {
        uint32_t g = G[H];
        const uint32_t k = recon_one<P>(g, Tj, Dj, Mp, Rj, m);
        G[H] = g;
        if (k) {
            const unsigned long long q = (unsigned long long)k + 1ull;
            const unsigned long long q2 = q * q;   // k < 2^31 so q^2 < 2^62... checked below for the product
            const unsigned long long pd = Pden[H];
            if (__umul64hi(pd, q2) != 0ull) *overflow = 1;
            Pden[H] = pd * q2;
            cls[2 * H] = (uint8_t)(j + 1);
            cls[2 * H + 1] = (uint8_t)(cls[2 * H + 1] + 1);
        }
    }
}

template <int P>
__global__ void k_recon_list(uint32_t* G, uint32_t* kout, int s, const uint8_t* Tj, const uint8_t* Dj, Mptrs Mp,
                             const uint32_t* Rj, int j, int m, long long cnt) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < cnt; t += (long long)gridDim.x * blockDim.x) {
        uint32_t g = G[t];
        kout[t * s + j] = recon_one<P>(g, Tj, Dj, Mp, Rj, m);
        G[t] = g;
    }
}

__global__ void k_init_recon(uint32_t* G, unsigned long long* Pden, uint8_t* cls, long long N) {
    for (long long H = blockIdx.x * (long long)blockDim.x + threadIdx.x; H < N; H += (long long)gridDim.x * blockDim.x) {
        G[H] = (uint32_t)H;
        Pden[H] = 1ull;
        cls[2 * H] = 0;
        cls[2 * H + 1] = 0;
    }
}

__global__ void k_copy_list(const uint32_t* __restrict__ a, uint32_t* b, long long cnt) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < cnt; t += (long long)gridDim.x * blockDim.x)
        b[t] = a[t];
}

// W = RN_f32(1 / RN_f32(P)) from the exact denominator
__global__ void k_weights(const unsigned long long* __restrict__ Pden, float* W, long long N) {
    for (long long H = blockIdx.x * (long long)blockDim.x + threadIdx.x; H < N; H += (long long)gridDim.x * blockDim.x)
        W[H] = __fdiv_rn(1.0f, __ull2float_rn(Pden[H]));
}

__global__ void k_init_T(uint8_t* Ts, long long N) {
    for (long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x; h < N; h += (long long)gridDim.x * blockDim.x)
        Ts[h] = h == 0 ? 0 : kInf;
}

// ---------------------------------------------------------------------------
static unsigned grid_for(long long n, int threads = 256) {
    long long b = (n + threads - 1) / threads;
    return (unsigned)std::min<long long>(std::max<long long>(b, 1), 152ll * 64);
}

// rank of the s*m rows over F_p (host, exact)
static int host_rank(const dwt_plan_s* P) {
    const int p = P->p, m = P->m, rows = P->s * m;
    std::vector<int> A(P->C.begin(), P->C.end());
    auto inv = [p](int a) {
        int r = 1;
        for (int e = 0; e < p - 2; ++e) r = r * a % p;
        return r;
    };
    int rank = 0;
    for (int c = 0; c < m && rank < rows; ++c) {
        int piv = -1;
        for (int r = rank; r < rows; ++r)
            if (A[(size_t)r * m + c]) { piv = r; break; }
        if (piv < 0) continue;
        for (int t = 0; t < m; ++t) std::swap(A[(size_t)rank * m + t], A[(size_t)piv * m + t]);
        const int iv = inv(A[(size_t)rank * m + c]);
        for (int t = 0; t < m; ++t) A[(size_t)rank * m + t] = A[(size_t)rank * m + t] * iv % p;
        for (int r = 0; r < rows; ++r) {
            if (r == rank || !A[(size_t)r * m + c]) continue;
            const int f = A[(size_t)r * m + c];
            for (int t = 0; t < m; ++t)
                A[(size_t)r * m + t] = ((A[(size_t)r * m + t] - f * A[(size_t)rank * m + t]) % p + p) % p;
        }
        ++rank;
    }
    return rank;
}

struct DpBuffers {
    uint8_t* T = nullptr;     // [(s+1)][N]
    uint8_t* D = nullptr;     // [s][N]
    uint8_t* M = nullptr;     // [m][N]  (M_0 aliases T_{j+1}, slots 1..m-1 used)
    uint8_t* M2 = nullptr;    // [2][N] ping-pong for the backward sweep
    void free_all(cudaStream_t st) {
        dfree(T, st); dfree(D, st); dfree(M, st); dfree(M2, st);
        T = D = M = M2 = nullptr;
    }
};

template <int P>
static int coset_tables_p(dwt_plan_s* Pl, cudaStream_t st) {
    const long long N = Pl->N;
    const int m = Pl->m, s = Pl->s;
    if (host_rank(Pl) < m) {
        set_error("rows of C_1..C_s span a space of dimension < m");
        return DWT_ESPAN;
    }
    const std::vector<uint32_t>& R = Pl->R_host;
    DpBuffers b;
    auto oom = [&]() {
        b.free_all(st);
        return DWT_ENOMEM;
    };
    if (dmalloc((void**)&b.T, (size_t)(s + 1) * N, st)) return oom();
    if (dmalloc((void**)&b.D, (size_t)s * N, st)) return oom();
    if (dmalloc((void**)&b.M, (size_t)m * N, st)) return oom();
    if (dmalloc((void**)&b.M2, (size_t)2 * N, st)) return oom();
    const unsigned gN = grid_for(N);
    // backward sweep
    {
        LaunchScope ls("dp_init", st);
        k_init_T<<<gN, 256, 0, st>>>(b.T + (size_t)s * N, N);
    }
    for (int j = s - 1; j >= 0; --j) {
        uint8_t* Tj = b.T + (size_t)j * N;
        const uint8_t* Tn = b.T + (size_t)(j + 1) * N;
        uint8_t* Dj = b.D + (size_t)j * N;
        DWT_CK(cudaMemcpyAsync(Tj, Tn, N, cudaMemcpyDeviceToDevice, st));
        DWT_CK(cudaMemsetAsync(Dj, 0, N, st));
        const uint8_t* cur = Tn;
        for (int i = 0; i < m; ++i) {
            uint8_t* nxt = b.M2 + (size_t)(i & 1) * N;
            {
                LaunchScope ls("dp_step", st);
                k_dp_step<P><<<gN, 256, 0, st>>>(cur, nxt, Tj, Dj, R[(size_t)j * m + i], i, m, N);
            }
            cur = nxt;
        }
    }
    DWT_CK_LAUNCH("coset backward sweep");
    // saturation check on T_1
    unsigned* d_flag = nullptr;
    if (dmalloc((void**)&d_flag, 2 * sizeof(unsigned), st)) return oom();
    DWT_CK(cudaMemsetAsync(d_flag, 0, 2 * sizeof(unsigned), st));
    {
        LaunchScope ls("dp_check", st);
        k_max_byte<<<gN, 256, 0, st>>>(b.T, N, d_flag);
    }
    unsigned mx = 0;
    DWT_CK(cudaMemcpyAsync(&mx, d_flag, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    DWT_CK(cudaStreamSynchronize(st));
    if (mx >= kInf) {
        dfree(d_flag, st);
        b.free_all(st);
        set_error("a least nu over some coset reaches 255");
        return DWT_EUNSUPPORTED;
    }
    // forward reconstruction over all labels
    uint32_t* G = nullptr;
    unsigned long long* Pden = nullptr;
    if (dmalloc((void**)&G, (size_t)N * 4, st) || dmalloc((void**)&Pden, (size_t)N * 8, st) ||
        dmalloc((void**)&Pl->d_W, (size_t)N * 4, st) || dmalloc((void**)&Pl->d_cls, (size_t)N * 2, st)) {
        dfree(G, st);
        dfree(Pden, st);
        dfree(d_flag, st);
        return oom();
    }
    uint32_t* d_R = Pl->d_R;
    {
        LaunchScope ls("dp_init", st);
        k_init_recon<<<gN, 256, 0, st>>>(G, Pden, Pl->d_cls, N);
    }
    int* d_over = (int*)(d_flag + 1);
    for (int j = 0; j < s; ++j) {
        Mptrs mp;
        mp.M[0] = b.T + (size_t)(j + 1) * N;
        for (int i = 1; i < m; ++i) {
            uint8_t* Mi = b.M + (size_t)i * N;
            {
                LaunchScope ls("dp_prefix", st);
                k_dp_prefix<P><<<gN, 256, 0, st>>>(mp.M[i - 1], Mi, R[(size_t)j * m + i - 1], m, N);
            }
            mp.M[i] = Mi;
        }
        {
            LaunchScope ls("dp_recon", st);
            k_recon_all<P><<<gN, 256, 0, st>>>(G, Pden, Pl->d_cls, d_over, b.T + (size_t)j * N, b.D + (size_t)j * N, mp,
                                               d_R + (size_t)j * m, j, m, N);
        }
    }
    {
        LaunchScope ls("dp_weights", st);
        k_weights<<<gN, 256, 0, st>>>(Pden, Pl->d_W, N);
    }
    DWT_CK_LAUNCH("coset reconstruction");
    int over = 0;
    DWT_CK(cudaMemcpyAsync(&over, d_over, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWT_CK(cudaStreamSynchronize(st));
    dfree(G, st);
    dfree(Pden, st);
    dfree(d_flag, st);
    if (Pl->flags & DWT_PLAN_KEEP_INDEX_MAP) {
        Pl->d_T = b.T;
        Pl->d_D = b.D;
        b.T = b.D = nullptr;
    }
    b.free_all(st);
    if (over) {
        set_error("a weight denominator prod (1+k_j)^2 exceeds 64 bits");
        return DWT_EUNSUPPORTED;
    }
    return DWT_OK;
}

// ---------------------------------------------------------------------------
// The whole coset programme in one CTA, for small nets (N <= 2^16): the same
// steps as above, separated by __syncthreads() instead of kernel launches, with
// the working arrays of the backward sweep in shared memory (three N-byte
// buffers).  A plan build is then a single launch on one SM, so many small
// plans (the serving mix) build side by side.
struct SmallDp {
    long long N;
    int m, s;
    const uint32_t* R;       // [s][m]
    uint8_t* T;              // [(s+1)][N]
    uint8_t* D;              // [s][N]
    uint8_t* M;              // [m][N] prefix minima of one coordinate (slot 0 unused)
    uint32_t* G;             // [N]
    unsigned long long* Pden;
    uint8_t* cls;            // [N][2]
    float* W;                // [N]
    unsigned* flags;         // [0] max least-nu, [1] denominator overflow
};

template <int P>
__global__ void __launch_bounds__(1024, 1) k_dp_small(SmallDp a) {
    extern __shared__ uint8_t sbuf[];
    const long long N = a.N;
    const int m = a.m, s = a.s, t = threadIdx.x, nt = blockDim.x;
    uint8_t* bx = sbuf;            // three rotating N-byte buffers
    uint8_t* by = sbuf + N;
    uint8_t* bz = sbuf + 2 * N;
    // T_s
    for (long long h = t; h < N; h += nt) {
        const uint8_t v = h == 0 ? 0 : kInf;
        by[h] = v;
        a.T[(long long)s * N + h] = v;
    }
    __syncthreads();
    uint8_t* Tn = by;   // T_{j+1}
    for (int j = s - 1; j >= 0; --j) {
        uint8_t* Tj = bx;
        uint8_t* Ma = bz;
        uint8_t* Mb = Tn;             // free once both copies are made
        uint8_t* Dj = a.D + (long long)j * N;
        for (long long h = t; h < N; h += nt) {
            Tj[h] = Tn[h];
            Ma[h] = Tn[h];
            Dj[h] = 0;
        }
        __syncthreads();
        for (int i = 0; i < m; ++i) {
            const uint32_t r = a.R[j * m + i];
            for (long long h = t; h < N; h += nt) {
                unsigned e = kInf;
#pragma unroll
                for (int q = 1; q < P; ++q) {
                    const unsigned v = Ma[dsub<P>((uint32_t)h, r, q, m)];
                    e = v < e ? v : e;
                }
                const unsigned cur = Ma[h];
                Mb[h] = (uint8_t)(e < cur ? e : cur);
                unsigned cand = e == kInf ? kInf : e + (unsigned)(i + 1);
                if (cand > kInf) cand = kInf;
                if (cand < Tj[h]) {
                    Tj[h] = (uint8_t)cand;
                    Dj[h] = (uint8_t)(i + 1);
                }
            }
            __syncthreads();
            uint8_t* tmp = Ma;
            Ma = Mb;
            Mb = tmp;
        }
        for (long long h = t; h < N; h += nt) a.T[(long long)j * N + h] = Tj[h];
        // rotate: T_j becomes T_{j+1} of the next coordinate
        Tn = Tj;
        bx = Ma;   // the two buffers not holding T_j
        bz = Mb;
        __syncthreads();
    }
    // saturation check on T_0
    {
        unsigned mx = 0;
        for (long long h = t; h < N; h += nt) mx = max(mx, (unsigned)a.T[h]);
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((t & 31) == 0) atomicMax(a.flags, mx);
    }
    __syncthreads();
    if (*(volatile unsigned*)a.flags >= kInf) return;
    // forward reconstruction over all labels
    for (long long H = t; H < N; H += nt) {
        a.G[H] = (uint32_t)H;
        a.Pden[H] = 1ull;
        a.cls[2 * H] = 0;
        a.cls[2 * H + 1] = 0;
    }
    __syncthreads();
    for (int j = 0; j < s; ++j) {
        Mptrs mp;
        mp.M[0] = a.T + (long long)(j + 1) * N;
        for (int i = 1; i < m; ++i) {
            const uint8_t* Mp = mp.M[i - 1];
            uint8_t* Mi = a.M + (long long)i * N;
            const uint32_t r = a.R[j * m + i - 1];
            for (long long h = t; h < N; h += nt) {
                unsigned v = Mp[h];
#pragma unroll
                for (int q = 1; q < P; ++q) {
                    const unsigned w = Mp[dsub<P>((uint32_t)h, r, q, m)];
                    v = w < v ? w : v;
                }
                Mi[h] = (uint8_t)v;
            }
            mp.M[i] = Mi;
            __syncthreads();
        }
        const uint8_t* Tj = a.T + (long long)j * N;
        const uint8_t* Dj = a.D + (long long)j * N;
        const uint32_t* Rj = a.R + (long long)j * m;
        for (long long H = t; H < N; H += nt) {
            uint32_t g = a.G[H];
            const uint32_t k = recon_one<P>(g, Tj, Dj, mp, Rj, m);
            a.G[H] = g;
            if (k) {
                const unsigned long long q = (unsigned long long)k + 1ull, q2 = q * q;
                const unsigned long long pd = a.Pden[H];
                if (__umul64hi(pd, q2) != 0ull) atomicExch(a.flags + 1, 1u);
                a.Pden[H] = pd * q2;
                a.cls[2 * H] = (uint8_t)(j + 1);
                a.cls[2 * H + 1] = (uint8_t)(a.cls[2 * H + 1] + 1);
            }
        }
        __syncthreads();
    }
    for (long long H = t; H < N; H += nt) a.W[H] = __fdiv_rn(1.0f, __ull2float_rn(a.Pden[H]));
}

static const long long kSmallDpMax = 1ll << 16;

template <int P>
static int coset_tables_small(dwt_plan_s* Pl, cudaStream_t st) {
    const long long N = Pl->N;
    const int m = Pl->m, s = Pl->s;
    if (host_rank(Pl) < m) {
        set_error("rows of C_1..C_s span a space of dimension < m");
        return DWT_ESPAN;
    }
    SmallDp a{};
    a.N = N;
    a.m = m;
    a.s = s;
    a.R = Pl->d_R;
    uint8_t *T = nullptr, *D = nullptr, *M = nullptr;
    uint32_t* G = nullptr;
    unsigned long long* Pden = nullptr;
    unsigned* flags = nullptr;
    auto cleanup = [&]() {
        dfree(T, st); dfree(D, st); dfree(M, st); dfree(G, st); dfree(Pden, st); dfree(flags, st);
    };
    if (dmalloc((void**)&T, (size_t)(s + 1) * N, st) || dmalloc((void**)&D, (size_t)s * N, st) ||
        dmalloc((void**)&M, (size_t)m * N, st) || dmalloc((void**)&G, (size_t)N * 4, st) ||
        dmalloc((void**)&Pden, (size_t)N * 8, st) || dmalloc((void**)&flags, 8, st) ||
        dmalloc((void**)&Pl->d_W, (size_t)N * 4, st) || dmalloc((void**)&Pl->d_cls, (size_t)N * 2, st)) {
        cleanup();
        return DWT_ENOMEM;
    }
    DWT_CK(cudaMemsetAsync(flags, 0, 8, st));
    a.T = T; a.D = D; a.M = M; a.G = G; a.Pden = Pden; a.cls = Pl->d_cls; a.W = Pl->d_W; a.flags = flags;
    auto kern = k_dp_small<P>;
    int rc = smem_limit_max(kern);
    if (rc) { cleanup(); return rc; }
    {
        LaunchScope ls("dp_small", st);
        kern<<<1, 1024, (size_t)3 * N, st>>>(a);
    }
    DWT_CK_LAUNCH("k_dp_small");
    unsigned hf[2] = {0, 0};
    DWT_CK(cudaMemcpyAsync(hf, flags, 8, cudaMemcpyDeviceToHost, st));
    DWT_CK(cudaStreamSynchronize(st));
    if (hf[0] >= kInf) {
        cleanup();
        set_error("a least nu over some coset reaches 255");
        return DWT_EUNSUPPORTED;
    }
    if (Pl->flags & DWT_PLAN_KEEP_INDEX_MAP) {
        Pl->d_T = T;
        Pl->d_D = D;
        T = D = nullptr;
    }
    cleanup();
    if (hf[1]) {
        set_error("a weight denominator prod (1+k_j)^2 exceeds 64 bits");
        return DWT_EUNSUPPORTED;
    }
    return DWT_OK;
}

int coset_tables_tree2(dwt_plan_s* Pl, cudaStream_t st, bool* used);
int coset_tables_treep(dwt_plan_s* Pl, cudaStream_t st, bool* used);

int build_coset_tables(dwt_plan_s* Pl, cudaStream_t st) {
    // the min-tree form (O(s N)) when every coordinate's rows are a basis; the
    // per-digit programme otherwise, and when the index maps are kept
    if (!(Pl->flags & DWT_PLAN_KEEP_INDEX_MAP)) {
        // the tree form runs only when every C_j is nonsingular, so its rows
        // already span F_p^m and the rank test below is not needed for it
        bool used = false;
        const int rc = Pl->p == 2 ? coset_tables_tree2(Pl, st, &used) : coset_tables_treep(Pl, st, &used);
        if (used || rc) return rc;
        if (host_rank(Pl) < Pl->m) {
            set_error("rows of C_1..C_s span a space of dimension < m");
            return DWT_ESPAN;
        }
    }
    const bool small = Pl->N <= kSmallDpMax;
    switch (Pl->p) {
        case 2: return small ? coset_tables_small<2>(Pl, st) : coset_tables_p<2>(Pl, st);
        case 3: return small ? coset_tables_small<3>(Pl, st) : coset_tables_p<3>(Pl, st);
        case 5: return small ? coset_tables_small<5>(Pl, st) : coset_tables_p<5>(Pl, st);
        case 7: return small ? coset_tables_small<7>(Pl, st) : coset_tables_p<7>(Pl, st);
        case 11: return small ? coset_tables_small<11>(Pl, st) : coset_tables_p<11>(Pl, st);
        case 13: return small ? coset_tables_small<13>(Pl, st) : coset_tables_p<13>(Pl, st);
        case 17: return small ? coset_tables_small<17>(Pl, st) : coset_tables_p<17>(Pl, st);
        case 19: return small ? coset_tables_small<19>(Pl, st) : coset_tables_p<19>(Pl, st);
        case 23: return small ? coset_tables_small<23>(Pl, st) : coset_tables_p<23>(Pl, st);
        case 29: return small ? coset_tables_small<29>(Pl, st) : coset_tables_p<29>(Pl, st);
        case 31: return small ? coset_tables_small<31>(Pl, st) : coset_tables_p<31>(Pl, st);
        default: return DWT_EUNSUPPORTED;
    }
}

template <int P>
static int h_to_k_p(dwt_plan_s* Pl, const uint32_t* H, uint32_t* k, long long cnt, cudaStream_t st) {
    const long long N = Pl->N;
    const int m = Pl->m, s = Pl->s;
    const std::vector<uint32_t>& R = Pl->R_host;
    int rc = ensure_workspace(Pl, (size_t)m * N + (size_t)cnt * 4 + 256, st);
    if (rc) return rc;
    uint8_t* M = (uint8_t*)Pl->d_ws;
    uint32_t* G = (uint32_t*)((uint8_t*)Pl->d_ws + (((size_t)m * N + 255) & ~(size_t)255));
    {
        LaunchScope ls("h2k_copy", st);
        k_copy_list<<<grid_for(cnt), 256, 0, st>>>(H, G, cnt);
    }
    for (int j = 0; j < s; ++j) {
        Mptrs mp;
        mp.M[0] = Pl->d_T + (size_t)(j + 1) * N;
        for (int i = 1; i < m; ++i) {
            uint8_t* Mi = M + (size_t)i * N;
            {
                LaunchScope ls("dp_prefix", st);
                k_dp_prefix<P><<<grid_for(N), 256, 0, st>>>(mp.M[i - 1], Mi, R[(size_t)j * m + i - 1], m, N);
            }
            mp.M[i] = Mi;
        }
        LaunchScope ls("h2k_recon", st);
        k_recon_list<P><<<grid_for(cnt), 256, 0, st>>>(G, k, s, Pl->d_T + (size_t)j * N, Pl->d_D + (size_t)j * N, mp,
                                                        Pl->d_R + (size_t)j * m, j, m, cnt);
    }
    DWT_CK_LAUNCH("index_to_wavenumber");
    return DWT_OK;
}

int run_h_to_k(dwt_plan_s* Pl, const uint32_t* H, uint32_t* k, long long cnt, cudaStream_t st) {
    switch (Pl->p) {
        case 2: return h_to_k_p<2>(Pl, H, k, cnt, st);
        case 3: return h_to_k_p<3>(Pl, H, k, cnt, st);
        case 5: return h_to_k_p<5>(Pl, H, k, cnt, st);
        case 7: return h_to_k_p<7>(Pl, H, k, cnt, st);
        case 11: return h_to_k_p<11>(Pl, H, k, cnt, st);
        case 13: return h_to_k_p<13>(Pl, H, k, cnt, st);
        case 17: return h_to_k_p<17>(Pl, H, k, cnt, st);
        case 19: return h_to_k_p<19>(Pl, H, k, cnt, st);
        case 23: return h_to_k_p<23>(Pl, H, k, cnt, st);
        case 29: return h_to_k_p<29>(Pl, H, k, cnt, st);
        case 31: return h_to_k_p<31>(Pl, H, k, cnt, st);
        default: return DWT_EUNSUPPORTED;
    }
}

int run_points(dwt_plan_s* Pl, uint32_t* Y, long long ldY, cudaStream_t st) {
    dim3 grid(std::min<unsigned>(grid_for(Pl->N), 4096), (unsigned)Pl->s);
    {
        LaunchScope ls("points", st);
        switch (Pl->p) {
            case 2: k_points<2><<<grid, 256, 0, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->N, Y, ldY); break;
            case 3: k_points<3><<<grid, 256, 0, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->N, Y, ldY); break;
            case 5: k_points<5><<<grid, 256, 0, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->N, Y, ldY); break;
            case 7: k_points<7><<<grid, 256, 0, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->N, Y, ldY); break;
            case 11: k_points<11><<<grid, 256, 0, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->N, Y, ldY); break;
            case 13: k_points<13><<<grid, 256, 0, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->N, Y, ldY); break;
            case 17: k_points<17><<<grid, 256, 0, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->N, Y, ldY); break;
            case 19: k_points<19><<<grid, 256, 0, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->N, Y, ldY); break;
            case 23: k_points<23><<<grid, 256, 0, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->N, Y, ldY); break;
            case 29: k_points<29><<<grid, 256, 0, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->N, Y, ldY); break;
            case 31: k_points<31><<<grid, 256, 0, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->N, Y, ldY); break;
        }
    }
    DWT_CK_LAUNCH("k_points");
    return DWT_OK;
}

int run_k_to_h(dwt_plan_s* Pl, const uint32_t* k, uint32_t* H, long long cnt, cudaStream_t st) {
    const unsigned g = grid_for(cnt);
    {
        LaunchScope ls("k_to_h", st);
        switch (Pl->p) {
            case 2: k_k_to_h<2><<<g, 256, 0, st>>>(Pl->d_C, Pl->d_R, Pl->m, Pl->s, k, H, cnt); break;
            case 3: k_k_to_h<3><<<g, 256, 0, st>>>(Pl->d_C, Pl->d_R, Pl->m, Pl->s, k, H, cnt); break;
            case 5: k_k_to_h<5><<<g, 256, 0, st>>>(Pl->d_C, Pl->d_R, Pl->m, Pl->s, k, H, cnt); break;
            case 7: k_k_to_h<7><<<g, 256, 0, st>>>(Pl->d_C, Pl->d_R, Pl->m, Pl->s, k, H, cnt); break;
            case 11: k_k_to_h<11><<<g, 256, 0, st>>>(Pl->d_C, Pl->d_R, Pl->m, Pl->s, k, H, cnt); break;
            case 13: k_k_to_h<13><<<g, 256, 0, st>>>(Pl->d_C, Pl->d_R, Pl->m, Pl->s, k, H, cnt); break;
            case 17: k_k_to_h<17><<<g, 256, 0, st>>>(Pl->d_C, Pl->d_R, Pl->m, Pl->s, k, H, cnt); break;
            case 19: k_k_to_h<19><<<g, 256, 0, st>>>(Pl->d_C, Pl->d_R, Pl->m, Pl->s, k, H, cnt); break;
            case 23: k_k_to_h<23><<<g, 256, 0, st>>>(Pl->d_C, Pl->d_R, Pl->m, Pl->s, k, H, cnt); break;
            case 29: k_k_to_h<29><<<g, 256, 0, st>>>(Pl->d_C, Pl->d_R, Pl->m, Pl->s, k, H, cnt); break;
            case 31: k_k_to_h<31><<<g, 256, 0, st>>>(Pl->d_C, Pl->d_R, Pl->m, Pl->s, k, H, cnt); break;
        }
    }
    DWT_CK_LAUNCH("k_k_to_h");
    return DWT_OK;
}

// ---------------------------------------------------------------------------
// synthetic test functions at the net points
template <int P>
__device__ __forceinline__ uint32_t point_Y(const uint8_t* Cj, const uint32_t* colj, int m, uint32_t n) {
    uint32_t Yv = 0;
    if constexpr (P == 2) {
        while (n) {
            const int c = __ffs(n) - 1;
            Yv ^= colj[c];
            n &= n - 1;
        }
    } else {
        int nd[32];
        for (int c = 0; c < m; ++c) {
            nd[c] = (int)(n % P);
            n /= P;
        }
        for (int i = 0; i < m; ++i) {
            int acc = 0;
            for (int c = 0; c < m; ++c) acc += Cj[i * m + c] * nd[c];
            Yv = Yv * P + (uint32_t)(acc % P);
        }
    }
    return Yv;
}

// f_b(x_n) = prod_j (1 + coef[b][j] (x_{j,n} - 1/2)); one thread per n, all b
template <int P, typename T>
__global__ void k_eval_product(const uint8_t* __restrict__ C, const uint32_t* __restrict__ col, int m, int s,
                               long long N, const double* __restrict__ coef, int batch, T* f, long long ld) {
    extern __shared__ double sh[];   // coef [batch][s]
    double* cf = sh;
    for (int t = threadIdx.x; t < batch * s; t += blockDim.x) cf[t] = coef[t];
    __syncthreads();
    const T inv = (T)1.0 / (T)(double)N;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        for (int b = 0; b < batch; ++b) {
            T v = (T)1;
            for (int j = 0; j < s; ++j) {
                const uint32_t Y = point_Y<P>(C + (size_t)j * m * m, col + (size_t)j * m, m, (uint32_t)n);
                const T x = (T)Y * inv;
                v *= (T)1 + (T)cf[b * s + j] * (x - (T)0.5);
            }
            f[(long long)b * ld + n] = v;
        }
    }
}

template <int P, typename T>
__global__ void k_eval_exp(const uint8_t* __restrict__ C, const uint32_t* __restrict__ col, int m, int s, long long N,
                           int batch, T* f, long long ld) {
    const T inv = (T)1.0 / (T)(double)N;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N; n += (long long)gridDim.x * blockDim.x) {
        T a = (T)0;
        for (int j = 0; j < s; ++j) {
            const uint32_t Y = point_Y<P>(C + (size_t)j * m * m, col + (size_t)j * m, m, (uint32_t)n);
            a += ((T)Y * inv) / (T)((j + 1) * (j + 1));
        }
        const T v = exp(a);
        for (int b = 0; b < batch; ++b) f[(long long)b * ld + n] = v;
    }
}

template <int P, typename T>
static int eval_product_t(dwt_plan_s* Pl, const double* coef, T* f, int batch, long long ld, cudaStream_t st) {
    const size_t smem = (size_t)batch * Pl->s * sizeof(double);
    if (smem > 200 * 1024) {
        set_error("batch * s too large for dwt_eval_product");
        return DWT_EUNSUPPORTED;
    }
    auto kern = k_eval_product<P, T>;
    if (int rc = smem_limit_max(kern)) return rc;
    {
        LaunchScope ls("eval_product", st);
        kern<<<grid_for(Pl->N), 256, smem, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->s, Pl->N, coef, batch, f, ld);
    }
    DWT_CK_LAUNCH("k_eval_product");
    return DWT_OK;
}

int run_eval_product(dwt_plan_s* Pl, const double* coef, void* f, int batch, long long ld, dwt_dtype t,
                     cudaStream_t st) {
#define DWT_EVP(PP)                                                                       \
    case PP:                                                                              \
        return t == DWT_F32 ? eval_product_t<PP, float>(Pl, coef, (float*)f, batch, ld, st) \
                            : eval_product_t<PP, double>(Pl, coef, (double*)f, batch, ld, st);
    switch (Pl->p) {
        DWT_EVP(2)
        DWT_EVP(3)
        DWT_EVP(5)
        DWT_EVP(7)
    }
#undef DWT_EVP
    return DWT_EUNSUPPORTED;
}

int run_eval_exp(dwt_plan_s* Pl, void* f, int batch, long long ld, dwt_dtype t, cudaStream_t st) {
    {
        LaunchScope ls("eval_exp", st);
        const unsigned g = grid_for(Pl->N);
#define DWT_EVE(PP)                                                                                           \
    case PP:                                                                                                  \
        if (t == DWT_F32)                                                                                     \
            k_eval_exp<PP, float><<<g, 256, 0, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->s, Pl->N, batch, (float*)f, ld); \
        else                                                                                                  \
            k_eval_exp<PP, double><<<g, 256, 0, st>>>(Pl->d_C, Pl->d_col, Pl->m, Pl->s, Pl->N, batch, (double*)f, ld); \
        break;
        switch (Pl->p) {
            DWT_EVE(2)
            DWT_EVE(3)
            DWT_EVE(5)
            DWT_EVE(7)
        }
#undef DWT_EVE
    }
    DWT_CK_LAUNCH("k_eval_exp");
    return DWT_OK;
}

}  // namespace dwt
