// dwt_treep.cu -- the min-tree form of the coset tables (see dwt_tree.cu) for
// p = 3, 5, 7.  In the basis r_0 .. r_{m-1} of coordinate j's rows a label has
// base-p coordinates U; the prefix minima M_i are the nodes U div p^i of the
// p-ary min-tree over T'[U] = T_{j+1}[h(U)], and the candidate with
// nu(k_j) = d is d + the least of the p - 1 siblings of node U div p^(d-1):
//     T_j = min(T'[U], A_0[U]),
//     A_i[V] = min(i+1 + min_{V' sibling of V} S_i[V'], A_{i+1}[V div p]).
// The representative is read forward as in the per-digit programme: top digit
// a >= 1 then lower digits a >= 0, smallest first, each tested as
// S_i[U' div p^i] + d = tau with U' = U minus a p^i digit-wise.
//
// Linear maps over F_p (labels <-> coordinates, coordinate j -> j+1) are
// applied with tables over groups of base-p digits whose entries are vectors
// of 4-bit digits in a 64-bit word; two such vectors add digit-wise mod p
// without carries (each digit sum is at most 2p - 2 < 16), with the reduction
// done on all digits at once.  Nets outside m <= 16 and the shared-memory
// limits of the coarse tree (p = 3: m <= 16, p = 5: m <= 11, p = 7: m <= 8),
// or with dependent rows, use the per-digit programme.
#include <algorithm>
#include <vector>

#include "dwt_internal.cuh"

namespace dwt {

namespace {

constexpr int kThreadsP = 512;
constexpr uint8_t kInfP = 255;
constexpr int kMaxGroups = 6;
constexpr unsigned long long kOnes = 0x1111111111111111ull;

template <int P> struct TreeShape;
template <> struct TreeShape<3> { static constexpr int LB = 8, TS = 6561, G = 5, PG = 243; };
template <> struct TreeShape<5> { static constexpr int LB = 5, TS = 3125, G = 3, PG = 125; };
template <> struct TreeShape<7> { static constexpr int LB = 4, TS = 2401, G = 2, PG = 49; };

// a linear map: table[g][x] = image of the digit group g with value x, as packed digits
struct MapP {
    unsigned long long t[kMaxGroups][256];
};

template <int P>
__host__ __device__ __forceinline__ unsigned long long padd(unsigned long long a, unsigned long long b) {
    const unsigned long long s = a + b;
    const unsigned long long ge = ((s + (unsigned long long)(8 - P) * kOnes) >> 3) & kOnes;
    return s - (unsigned long long)P * ge;
}

// packed digits -> label
template <int P>
__host__ __device__ __forceinline__ uint32_t unpack(unsigned long long v, int m) {
    uint32_t h = 0;
    for (int c = m - 1; c >= 0; --c) h = h * P + (uint32_t)((v >> (4 * c)) & 15u);
    return h;
}

template <int P>
__device__ __forceinline__ uint32_t applyP(const unsigned long long (*t)[256], uint32_t x, int ng, int m) {
    unsigned long long v = 0;
    for (int g = 0; g < ng; ++g) {
        const uint32_t q = x / TreeShape<P>::PG;
        v = padd<P>(v, t[g][x - q * TreeShape<P>::PG]);
        x = q;
    }
    return unpack<P>(v, m);
}

template <int P>
__device__ __forceinline__ void load_mapP(unsigned long long (*sm)[256], const MapP* g, int ng) {
    for (int i = threadIdx.x; i < ng * 256; i += blockDim.x) sm[i >> 8][i & 255] = g->t[i >> 8][i & 255];
}

// level i of a p-ary tree over n leaves starts at sum_{l < i} n / p^l
template <int P>
__host__ __device__ __forceinline__ long long loffP(long long n, long long n_i) {
    return (n - n_i) * P / (P - 1);   // n_i = n / p^i
}

__device__ __forceinline__ unsigned sat_addP(unsigned v, unsigned d) {
    if (v >= kInfP) return kInfP;
    const unsigned c = v + d;
    return c > kInfP ? kInfP : c;
}

template <int P>
__global__ void __launch_bounds__(kThreadsP) k_treep_up(const uint8_t* __restrict__ Tprev, const MapP* __restrict__ Q,
                                                        uint8_t* lev, long long N, int m, int ng) {
    using SH = TreeShape<P>;
    __shared__ unsigned long long q[kMaxGroups][256];
    __shared__ uint8_t sl[2 * SH::TS];
    const long long base = (long long)blockIdx.x * SH::TS;
    if (Tprev) load_mapP<P>(q, Q, ng);
    __syncthreads();
    for (int e = threadIdx.x; e < SH::TS; e += blockDim.x) {
        const uint32_t U = (uint32_t)(base + e);
        const uint8_t v = Tprev ? Tprev[applyP<P>(q, U, ng, m)] : (U == 0 ? 0 : kInfP);
        sl[e] = v;
        lev[base + e] = v;
    }
    __syncthreads();
    int n = SH::TS;
    long long nN = N;
    for (int i = 1; i <= SH::LB; ++i) {
        const int np = n / P;
        const long long nNp = nN / P;
        const uint8_t* src = sl + loffP<P>(SH::TS, n);
        uint8_t* dst = sl + loffP<P>(SH::TS, np);
        for (int v = threadIdx.x; v < np; v += blockDim.x) {
            unsigned x = src[P * v];
#pragma unroll
            for (int c = 1; c < P; ++c) x = min(x, (unsigned)src[P * v + c]);
            dst[v] = (uint8_t)x;
            lev[loffP<P>(N, nNp) + base / (N / nNp) + v] = (uint8_t)x;
        }
        __syncthreads();
        n = np;
        nN = nNp;
    }
}

// the least of the p - 1 siblings of node v (children of v's parent other than v)
template <int P>
__device__ __forceinline__ unsigned sib_min(const uint8_t* S, long long v) {
    const long long b = v - v % P;
    unsigned x = kInfP;
#pragma unroll
    for (int c = 0; c < P; ++c)
        if (b + c != v) x = min(x, (unsigned)S[b + c]);
    return x;
}

template <int P>
__global__ void __launch_bounds__(1024) k_treep_coarse(uint8_t* lev, uint16_t* Aout, long long N, int m, int want_a) {
    using SH = TreeShape<P>;
    extern __shared__ __align__(16) unsigned char sm[];
    const int nLB = (int)(N / SH::TS);
    uint8_t* sl = sm;
    uint16_t* A0 = reinterpret_cast<uint16_t*>(sm + ((2 * nLB + 15) & ~15));
    uint16_t* A1 = A0 + nLB;
    const int top = m - SH::LB;
    const long long offLB = loffP<P>(N, nLB);
    for (int v = threadIdx.x; v < nLB; v += blockDim.x) sl[v] = lev[offLB + v];
    __syncthreads();
    int n = nLB;
    for (int i = 1; i <= top; ++i) {
        const int np = n / P;
        const uint8_t* src = sl + loffP<P>(nLB, n);
        uint8_t* dst = sl + loffP<P>(nLB, np);
        for (int v = threadIdx.x; v < np; v += blockDim.x) {
            unsigned x = src[P * v];
#pragma unroll
            for (int c = 1; c < P; ++c) x = min(x, (unsigned)src[P * v + c]);
            dst[v] = (uint8_t)x;
            lev[loffP<P>(N, np) + v] = (uint8_t)x;
        }
        __syncthreads();
        n = np;
    }
    if (!want_a) return;
    uint16_t* cur = A0;
    uint16_t* nxt = A1;
    if (threadIdx.x == 0) cur[0] = kInfP;
    __syncthreads();
    n = 1;   // nodes at level i + 1
    for (int i = m - 1; i >= SH::LB; --i) {
        const int ni = n * P;
        const uint8_t* S = sl + loffP<P>(nLB, ni);
        for (int v = threadIdx.x; v < ni; v += blockDim.x) {
            const uint16_t par = cur[v / P];
            const unsigned c = sat_addP(sib_min<P>(S, v), (unsigned)(i + 1));
            nxt[v] = c <= (unsigned)(par & 255) ? (uint16_t)(c | ((unsigned)(i + 1) << 8)) : par;
        }
        __syncthreads();
        uint16_t* tmp = cur;
        cur = nxt;
        nxt = tmp;
        n = ni;
    }
    for (int v = threadIdx.x; v < nLB; v += blockDim.x) Aout[v] = cur[v];
}

template <int P>
__global__ void __launch_bounds__(kThreadsP) k_treep_down(const uint8_t* __restrict__ lev,
                                                          const uint16_t* __restrict__ Acoarse, uint8_t* TU, uint8_t* DU,
                                                          long long N) {
    using SH = TreeShape<P>;
    __shared__ uint8_t sl[2 * SH::TS];
    __shared__ uint16_t a0[SH::TS], a1[SH::TS];
    const long long base = (long long)blockIdx.x * SH::TS;
    {
        int n = SH::TS;
        long long nN = N;
        for (int i = 0; i < SH::LB; ++i) {
            for (int v = threadIdx.x; v < n; v += blockDim.x)
                sl[loffP<P>(SH::TS, n) + v] = lev[loffP<P>(N, nN) + base / (N / nN) + v];
            n /= P;
            nN /= P;
        }
    }
    if (threadIdx.x == 0) a0[0] = Acoarse[blockIdx.x];
    __syncthreads();
    uint16_t* cur = a0;
    uint16_t* nxt = a1;
    int n = 1;
    for (int i = SH::LB - 1; i >= 0; --i) {
        const int ni = n * P;
        const uint8_t* S = sl + loffP<P>(SH::TS, ni);
        for (int v = threadIdx.x; v < ni; v += blockDim.x) {
            const uint16_t par = cur[v / P];
            const unsigned c = sat_addP(sib_min<P>(S, v), (unsigned)(i + 1));
            nxt[v] = c <= (unsigned)(par & 255) ? (uint16_t)(c | ((unsigned)(i + 1) << 8)) : par;
        }
        __syncthreads();
        uint16_t* tmp = cur;
        cur = nxt;
        nxt = tmp;
        n = ni;
    }
    for (int e = threadIdx.x; e < SH::TS; e += blockDim.x) {
        const unsigned t = sl[e], a = cur[e];
        const bool keep = t <= (a & 255);
        TU[base + e] = keep ? (uint8_t)t : (uint8_t)(a & 255);
        DU[base + e] = keep ? 0 : (uint8_t)(a >> 8);
    }
}

template <int P>
__global__ void __launch_bounds__(kThreadsP) k_treep_recon(uint32_t* G, unsigned long long* Pden, uint8_t* cls,
                                                           int* overflow, const uint8_t* __restrict__ TU,
                                                           const uint8_t* __restrict__ DU,
                                                           const uint8_t* __restrict__ lev,
                                                           const MapP* __restrict__ Ij, const MapP* __restrict__ Fj,
                                                           int j, int m, int ng, long long N) {
    __shared__ unsigned long long inv[kMaxGroups][256];
    __shared__ unsigned long long fwd[kMaxGroups][256];
    __shared__ long long off[32];
    __shared__ uint32_t pw[32];
    load_mapP<P>(inv, Ij, ng);
    load_mapP<P>(fwd, Fj, ng);
    if (threadIdx.x == 0) {
        long long n = N;
        uint32_t w = 1;
        for (int i = 0; i <= m; ++i) {
            off[i] = loffP<P>(N, n);
            pw[i] = w;
            n /= P;
            w *= P;
        }
    }
    __syncthreads();
    for (long long H = blockIdx.x * (long long)blockDim.x + threadIdx.x; H < N; H += (long long)gridDim.x * blockDim.x) {
        const uint32_t g = G[H];
        uint32_t U = applyP<P>(inv, g, ng, m);
        const int tau = TU[U], d = DU[U];
        if (!d) continue;
        uint32_t k = 0;
        for (int i = d - 1; i >= 0; --i) {
            const uint32_t u = (U / pw[i]) % P;
            int a = i == d - 1 ? 1 : 0;
            uint32_t Un = U;
            for (; a < P; ++a) {
                const uint32_t un = (u + P - (uint32_t)a) % P;
                Un = U - u * pw[i] + un * pw[i];
                if ((int)lev[off[i] + Un / pw[i]] + d == tau) break;
            }
            if (a == P) a = P - 1;   // unreachable for a consistent table
            U = Un;
            k += (uint32_t)a * pw[i];
        }
        G[H] = applyP<P>(fwd, U, ng, m);
        const unsigned long long q = (unsigned long long)k + 1ull, q2 = q * q;
        const unsigned long long pd = Pden[H];
        if (__umul64hi(pd, q2) != 0ull) *overflow = 1;
        Pden[H] = pd * q2;
        cls[2 * H] = (uint8_t)(j + 1);
        cls[2 * H + 1] = (uint8_t)(cls[2 * H + 1] + 1);
    }
}

// The whole construction for a net of N = p^m <= one tile in one CTA (see the
// p = 2 form): maps, levels and the previous coordinate's table in shared
// memory, the reading state of labels H = t + 1024 q in registers.
template <int P>
__global__ void __launch_bounds__(1024, 1) k_treep_one(const MapP* __restrict__ Imaps, const MapP* __restrict__ Fmaps,
                                                       const MapP* __restrict__ Qmaps, int m, int s, int ng,
                                                       uint8_t* TU, uint8_t* DU, uint8_t* cls, float* W,
                                                       unsigned* flags) {
    using SH = TreeShape<P>;
    constexpr int QN = (SH::TS + 1023) / 1024;
    extern __shared__ __align__(16) unsigned char sm[];
    unsigned long long (*mq)[256] = reinterpret_cast<unsigned long long (*)[256]>(sm);
    unsigned long long (*mi)[256] = reinterpret_cast<unsigned long long (*)[256]>(sm + sizeof(MapP));
    unsigned long long (*mf)[256] = reinterpret_cast<unsigned long long (*)[256]>(sm + 2 * sizeof(MapP));
    long long* off = reinterpret_cast<long long*>(sm + 3 * sizeof(MapP));          // [32]
    uint32_t* pw = reinterpret_cast<uint32_t*>(off + 32);                          // [32]
    int N = 1;
    for (int i = 0; i < m; ++i) N *= P;
    uint16_t* A0 = reinterpret_cast<uint16_t*>(pw + 32);
    uint16_t* A1 = A0 + N;
    uint8_t* lv = reinterpret_cast<uint8_t*>(A1 + N);
    uint8_t* Tp = lv + 2 * N;
    const int t = threadIdx.x;
    if (t == 0) {
        long long n = N;
        uint32_t w = 1;
        for (int i = 0; i <= m; ++i) {
            off[i] = loffP<P>(N, n);
            pw[i] = w;
            n /= P;
            w *= P;
        }
    }
    auto load = [&](unsigned long long (*dst)[256], const MapP* src) {
        for (int i = t; i < ng * 256; i += blockDim.x) dst[i >> 8][i & 255] = src->t[i >> 8][i & 255];
    };
    auto build_levels = [&](int j) {
        for (int U = t; U < N; U += blockDim.x)
            lv[U] = j == s - 1 ? (U == 0 ? 0 : kInfP) : Tp[applyP<P>(mq, (uint32_t)U, ng, m)];
        __syncthreads();
        for (int i = 1; i <= m; ++i) {
            const int np = N / (int)pw[i];
            const uint8_t* src = lv + off[i - 1];
            uint8_t* dst = lv + off[i];
            for (int v = t; v < np; v += blockDim.x) {
                unsigned x = src[P * v];
#pragma unroll
                for (int c = 1; c < P; ++c) x = min(x, (unsigned)src[P * v + c]);
                dst[v] = (uint8_t)x;
            }
            __syncthreads();
        }
    };
    for (int j = s - 1; j >= 0; --j) {
        if (j < s - 1) load(mq, Qmaps + j);
        __syncthreads();
        build_levels(j);
        uint16_t* cur = A0;
        uint16_t* nxt = A1;
        if (t == 0) cur[0] = kInfP;
        __syncthreads();
        int n = 1;
        for (int i = m - 1; i >= 0; --i) {
            const int ni = n * P;
            const uint8_t* S = lv + off[i];
            for (int v = t; v < ni; v += blockDim.x) {
                const uint16_t par = cur[v / P];
                const unsigned c = sat_addP(sib_min<P>(S, v), (unsigned)(i + 1));
                nxt[v] = c <= (unsigned)(par & 255) ? (uint16_t)(c | ((unsigned)(i + 1) << 8)) : par;
            }
            __syncthreads();
            uint16_t* tmp = cur;
            cur = nxt;
            nxt = tmp;
            n = ni;
        }
        for (int U = t; U < N; U += blockDim.x) {
            const unsigned tv = lv[U], a = cur[U];
            const bool keep = tv <= (a & 255);
            const uint8_t val = keep ? (uint8_t)tv : (uint8_t)(a & 255);
            TU[(size_t)j * N + U] = val;
            DU[(size_t)j * N + U] = keep ? 0 : (uint8_t)(a >> 8);
            Tp[U] = val;
        }
        __syncthreads();
    }
    {
        unsigned mx = 0;
        for (int U = t; U < N; U += blockDim.x) mx = max(mx, (unsigned)Tp[U]);
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((t & 31) == 0) atomicMax(flags, mx);
        __syncthreads();
        if (*(volatile unsigned*)flags >= kInfP) return;
    }
    uint32_t g[QN];
    unsigned long long pd[QN];
    uint8_t ct[QN], cs[QN];
#pragma unroll
    for (int q = 0; q < QN; ++q) {
        g[q] = (uint32_t)(t + 1024 * q);
        pd[q] = 1ull;
        ct[q] = cs[q] = 0;
    }
    bool over = false;
    for (int j = 0; j < s; ++j) {
        __syncthreads();
        load(mi, Imaps + j);
        load(mf, Fmaps + j);
        if (j < s - 1) {
            load(mq, Qmaps + j);
            for (int U = t; U < N; U += blockDim.x) Tp[U] = TU[(size_t)(j + 1) * N + U];
        }
        __syncthreads();
        build_levels(j);
#pragma unroll
        for (int q = 0; q < QN; ++q) {
            if (t + 1024 * q >= N) continue;
            uint32_t U = applyP<P>(mi, g[q], ng, m);
            const int tau = TU[(size_t)j * N + U], d = DU[(size_t)j * N + U];
            if (!d) continue;
            uint32_t k = 0;
            for (int i = d - 1; i >= 0; --i) {
                const uint32_t u = (U / pw[i]) % P;
                int a = i == d - 1 ? 1 : 0;
                uint32_t Un = U;
                for (; a < P; ++a) {
                    Un = U - u * pw[i] + ((u + P - (uint32_t)a) % P) * pw[i];
                    if ((int)lv[off[i] + Un / pw[i]] + d == tau) break;
                }
                if (a == P) a = P - 1;   // unreachable for a consistent table
                U = Un;
                k += (uint32_t)a * pw[i];
            }
            g[q] = applyP<P>(mf, U, ng, m);
            const unsigned long long qq = (unsigned long long)k + 1ull, q2 = qq * qq;
            if (__umul64hi(pd[q], q2) != 0ull) over = true;
            pd[q] *= q2;
            ct[q] = (uint8_t)(j + 1);
            ++cs[q];
        }
    }
#pragma unroll
    for (int q = 0; q < QN; ++q) {
        const int H = t + 1024 * q;
        if (H >= N) continue;
        W[H] = __fdiv_rn(1.0f, __ull2float_rn(pd[q]));
        cls[2 * H] = ct[q];
        cls[2 * H + 1] = cs[q];
    }
    if (over) atomicExch(flags + 1, 1u);
}

__global__ void k_treep_max(const uint8_t* __restrict__ a, long long N, unsigned* out) {
    unsigned mx = 0;
    for (long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x; h < N; h += (long long)gridDim.x * blockDim.x)
        mx = max(mx, (unsigned)a[h]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

__global__ void k_treep_init(uint32_t* G, unsigned long long* Pden, uint8_t* cls, long long N) {
    for (long long H = blockIdx.x * (long long)blockDim.x + threadIdx.x; H < N; H += (long long)gridDim.x * blockDim.x) {
        G[H] = (uint32_t)H;
        Pden[H] = 1ull;
        cls[2 * H] = 0;
        cls[2 * H + 1] = 0;
    }
}

__global__ void k_treep_weights(const unsigned long long* __restrict__ Pden, float* W, long long N) {
    for (long long H = blockIdx.x * (long long)blockDim.x + threadIdx.x; H < N; H += (long long)gridDim.x * blockDim.x)
        W[H] = __fdiv_rn(1.0f, __ull2float_rn(Pden[H]));
}

int inv_mod_p(int a, int p) {
    for (int x = 1; x < p; ++x)
        if (a * x % p == 1) return x;
    return 0;
}

// columns c[i] (digit vectors, digit a of c[i] = row a) of an m x m matrix over
// F_p -> columns of its inverse (digit vectors); false if singular
bool gfp_inverse(const std::vector<std::vector<int>>& c, int m, int p, std::vector<std::vector<int>>& ci) {
    std::vector<std::vector<int>> A(m, std::vector<int>(2 * m, 0));
    for (int a = 0; a < m; ++a) {
        for (int i = 0; i < m; ++i) A[a][i] = c[i][a];
        A[a][m + a] = 1;
    }
    for (int col = 0; col < m; ++col) {
        int piv = -1;
        for (int a = col; a < m; ++a)
            if (A[a][col]) { piv = a; break; }
        if (piv < 0) return false;
        std::swap(A[col], A[piv]);
        const int iv = inv_mod_p(A[col][col], p);
        for (int t = 0; t < 2 * m; ++t) A[col][t] = A[col][t] * iv % p;
        for (int a = 0; a < m; ++a) {
            if (a == col || !A[a][col]) continue;
            const int f = A[a][col];
            for (int t = 0; t < 2 * m; ++t) A[a][t] = ((A[a][t] - f * A[col][t]) % p + p) % p;
        }
    }
    ci.assign(m, std::vector<int>(m, 0));
    for (int a = 0; a < m; ++a)
        for (int i = 0; i < m; ++i) ci[a][i] = A[i][m + a];   // column a of B^{-1}: entry i
    return true;
}

std::vector<int> digits_of(uint32_t h, int p, int m) {
    std::vector<int> d(m);
    for (int c = 0; c < m; ++c) {
        d[c] = (int)(h % (uint32_t)p);
        h /= (uint32_t)p;
    }
    return d;
}

unsigned long long pack(const std::vector<int>& d) {
    unsigned long long v = 0;
    for (size_t c = 0; c < d.size(); ++c) v |= (unsigned long long)d[c] << (4 * c);
    return v;
}

// table of the linear map with image columns cols (digit vectors)
template <int P>
void make_mapP(const std::vector<std::vector<int>>& cols, int m, MapP& M) {
    using SH = TreeShape<P>;
    const int ng = (m + SH::G - 1) / SH::G;
    // packed multiples a * column i, a = 0 .. p-1
    std::vector<unsigned long long> mult((size_t)m * P, 0ull);
    for (int i = 0; i < m; ++i) {
        const unsigned long long c = pack(cols[i]);
        for (int a = 1; a < P; ++a) mult[(size_t)i * P + a] = padd<P>(mult[(size_t)i * P + a - 1], c);
    }
    for (int g = 0; g < kMaxGroups; ++g)
        for (int x = 0; x < 256; ++x) {
            unsigned long long v = 0;
            if (g < ng && x < SH::PG) {
                int y = x;
                for (int l = 0; l < SH::G; ++l) {
                    const int dgt = y % P, i = g * SH::G + l;
                    y /= P;
                    if (dgt && i < m) v = padd<P>(v, mult[(size_t)i * P + dgt]);
                }
            }
            M.t[g][x] = v;
        }
}

template <int P>
unsigned long long host_applyP(const MapP& M, uint32_t x, int ng) {
    unsigned long long v = 0;
    for (int g = 0; g < ng; ++g) {
        v = padd<P>(v, M.t[g][x % TreeShape<P>::PG]);
        x /= TreeShape<P>::PG;
    }
    return v;
}

unsigned grid_np(long long n) { return (unsigned)std::max(1ll, std::min((n + 255) / 256, 8ll * 152)); }

template <int P>
int treep_one(dwt_plan_s* Pl, const std::vector<MapP>& Imap, const std::vector<MapP>& Fmap,
              const std::vector<MapP>& Qmap, int ng, cudaStream_t st) {
    const long long N = Pl->N;
    const int m = Pl->m, s = Pl->s;
    uint8_t *TU = nullptr, *DU = nullptr;
    MapP* dmaps = nullptr;
    unsigned* flags = nullptr;
    auto cleanup = [&]() {
        dfree(TU, st); dfree(DU, st); dfree(dmaps, st); dfree(flags, st);
    };
    if (dmalloc((void**)&TU, (size_t)s * N, st) || dmalloc((void**)&DU, (size_t)s * N, st) ||
        dmalloc((void**)&dmaps, sizeof(MapP) * 3 * s, st) || dmalloc((void**)&flags, 8, st) ||
        dmalloc((void**)&Pl->d_W, (size_t)N * 4, st) || dmalloc((void**)&Pl->d_cls, (size_t)N * 2, st)) {
        cleanup();
        return DWT_ENOMEM;
    }
    std::vector<MapP> hm(3 * s);
    for (int j = 0; j < s; ++j) {
        hm[j] = Imap[j];
        hm[s + j] = Fmap[j];
        hm[2 * s + j] = Qmap[j];
    }
    DWT_CK(cudaMemcpyAsync(dmaps, hm.data(), sizeof(MapP) * 3 * s, cudaMemcpyHostToDevice, st));
    DWT_CK(cudaMemsetAsync(flags, 0, 8, st));
    const size_t smem = 3 * sizeof(MapP) + 32 * 8 + 32 * 4 + (size_t)4 * N + 2 * N + N;
    int rc = smem_limit_max(k_treep_one<P>);
    if (rc) { cleanup(); return rc; }
    {
        LaunchScope ls("tree_one", st);
        k_treep_one<P><<<1, 1024, smem, st>>>(dmaps, dmaps + s, dmaps + 2 * s, m, s, ng, TU, DU, Pl->d_cls, Pl->d_W,
                                              flags);
    }
    DWT_CK_LAUNCH("k_treep_one");
    unsigned hf[2] = {0, 0};
    DWT_CK(cudaMemcpyAsync(hf, flags, 8, cudaMemcpyDeviceToHost, st));
    DWT_CK(cudaStreamSynchronize(st));
    cleanup();
    if (hf[0] >= kInfP) {
        set_error("a least nu over some coset reaches 255");
        return DWT_EUNSUPPORTED;
    }
    if (hf[1]) {
        set_error("a weight denominator prod (1+k_j)^2 exceeds 64 bits");
        return DWT_EUNSUPPORTED;
    }
    return DWT_OK;
}

template <int P>
int treep(dwt_plan_s* Pl, cudaStream_t st, bool* used) {
    using SH = TreeShape<P>;
    const long long N = Pl->N;
    const int m = Pl->m, s = Pl->s;
    *used = false;
    if (m > 16 || m < 1) return DWT_OK;
    const long long nLB = N / SH::TS;
    if (nLB > 16384) return DWT_OK;
    const int ng = (m + SH::G - 1) / SH::G;
    if (ng > kMaxGroups) return DWT_OK;
    const std::vector<uint32_t>& R = Pl->R_host;
    std::vector<MapP> Imap(s), Fmap(s), Qmap(s);
    std::vector<std::vector<std::vector<int>>> rows(s), invc(s);
    for (int j = 0; j < s; ++j) {
        rows[j].resize(m);
        for (int i = 0; i < m; ++i) rows[j][i] = digits_of(R[(size_t)j * m + i], P, m);
        if (!gfp_inverse(rows[j], m, P, invc[j])) return DWT_OK;
        make_mapP<P>(invc[j], m, Imap[j]);
        make_mapP<P>(rows[j], m, Fmap[j]);
    }
    for (int j = 0; j + 1 < s; ++j) {
        std::vector<std::vector<int>> qc(m);
        for (int i = 0; i < m; ++i) {
            // image of e_i under I_{j+1} o F_j, as a digit vector
            const uint32_t h = unpack<P>(pack(rows[j][i]), m);
            qc[i] = digits_of(unpack<P>(host_applyP<P>(Imap[j + 1], h, ng), m), P, m);
        }
        make_mapP<P>(qc, m, Qmap[j]);
    }
    *used = true;
    if (m <= SH::LB) return treep_one<P>(Pl, Imap, Fmap, Qmap, ng, st);
    uint8_t *TU = nullptr, *DU = nullptr, *lev = nullptr;
    uint16_t* Ac = nullptr;
    MapP* dmaps = nullptr;
    uint32_t* G = nullptr;
    unsigned long long* Pden = nullptr;
    unsigned* flags = nullptr;
    auto cleanup = [&]() {
        dfree(TU, st); dfree(DU, st); dfree(lev, st); dfree(Ac, st); dfree(dmaps, st);
        dfree(G, st); dfree(Pden, st); dfree(flags, st);
    };
    if (dmalloc((void**)&TU, (size_t)s * N, st) || dmalloc((void**)&DU, (size_t)s * N, st) ||
        dmalloc((void**)&lev, (size_t)2 * N, st) || dmalloc((void**)&Ac, (size_t)2 * nLB, st) ||
        dmalloc((void**)&dmaps, sizeof(MapP) * 3 * s, st) || dmalloc((void**)&flags, 8, st)) {
        cleanup();
        return DWT_ENOMEM;
    }
    std::vector<MapP> hm(3 * s);
    for (int j = 0; j < s; ++j) {
        hm[j] = Imap[j];
        hm[s + j] = Fmap[j];
        hm[2 * s + j] = Qmap[j];
    }
    DWT_CK(cudaMemcpyAsync(dmaps, hm.data(), sizeof(MapP) * 3 * s, cudaMemcpyHostToDevice, st));
    DWT_CK(cudaMemsetAsync(flags, 0, 8, st));
    const MapP* dI = dmaps;
    const MapP* dF = dmaps + s;
    const MapP* dQ = dmaps + 2 * s;
    const size_t coarse_smem = (size_t)((2 * nLB + 15) & ~15ll) + (size_t)4 * nLB;
    {
        int rc = smem_limit_max(k_treep_coarse<P>);
        if (rc) { cleanup(); return rc; }
    }
    const unsigned tiles = (unsigned)nLB;
    for (int j = s - 1; j >= 0; --j) {
        const uint8_t* Tn = j + 1 < s ? TU + (size_t)(j + 1) * N : nullptr;
        {
            LaunchScope ls("tree_up", st);
            k_treep_up<P><<<tiles, kThreadsP, 0, st>>>(Tn, Tn ? dQ + j : nullptr, lev, N, m, ng);
        }
        {
            LaunchScope ls("tree_coarse", st);
            k_treep_coarse<P><<<1, 1024, coarse_smem, st>>>(lev, Ac, N, m, 1);
        }
        {
            LaunchScope ls("tree_down", st);
            k_treep_down<P><<<tiles, kThreadsP, 0, st>>>(lev, Ac, TU + (size_t)j * N, DU + (size_t)j * N, N);
        }
    }
    DWT_CK_LAUNCH("coset tree backward sweep");
    {
        LaunchScope ls("tree_check", st);
        k_treep_max<<<grid_np(N), 256, 0, st>>>(TU, N, flags);
    }
    unsigned mx = 0;
    DWT_CK(cudaMemcpyAsync(&mx, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    DWT_CK(cudaStreamSynchronize(st));
    if (mx >= kInfP) {
        cleanup();
        set_error("a least nu over some coset reaches 255");
        return DWT_EUNSUPPORTED;
    }
    if (dmalloc((void**)&G, (size_t)N * 4, st) || dmalloc((void**)&Pden, (size_t)N * 8, st) ||
        dmalloc((void**)&Pl->d_W, (size_t)N * 4, st) || dmalloc((void**)&Pl->d_cls, (size_t)N * 2, st)) {
        cleanup();
        return DWT_ENOMEM;
    }
    {
        LaunchScope ls("tree_init", st);
        k_treep_init<<<grid_np(N), 256, 0, st>>>(G, Pden, Pl->d_cls, N);
    }
    int* over = reinterpret_cast<int*>(flags + 1);
    for (int j = 0; j < s; ++j) {
        const uint8_t* Tn = j + 1 < s ? TU + (size_t)(j + 1) * N : nullptr;
        {
            LaunchScope ls("tree_up", st);
            k_treep_up<P><<<tiles, kThreadsP, 0, st>>>(Tn, Tn ? dQ + j : nullptr, lev, N, m, ng);
        }
        if (m > SH::LB) {
            LaunchScope ls("tree_coarse", st);
            k_treep_coarse<P><<<1, 1024, coarse_smem, st>>>(lev, Ac, N, m, 0);
        }
        {
            LaunchScope ls("tree_recon", st);
            k_treep_recon<P><<<grid_np(N), kThreadsP, 0, st>>>(G, Pden, Pl->d_cls, over, TU + (size_t)j * N,
                                                               DU + (size_t)j * N, lev, dI + j, dF + j, j, m, ng, N);
        }
    }
    {
        LaunchScope ls("tree_weights", st);
        k_treep_weights<<<grid_np(N), 256, 0, st>>>(Pden, Pl->d_W, N);
    }
    DWT_CK_LAUNCH("coset tree reconstruction");
    int ov = 0;
    DWT_CK(cudaMemcpyAsync(&ov, over, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWT_CK(cudaStreamSynchronize(st));
    cleanup();
    if (ov) {
        set_error("a weight denominator prod (1+k_j)^2 exceeds 64 bits");
        return DWT_EUNSUPPORTED;
    }
    return DWT_OK;
}

}  // namespace

// Tables W, cls of a p = 3, 5, 7 plan by the tree form; *used = false (nothing
// allocated or launched) when the net is outside its limits.
int coset_tables_treep(dwt_plan_s* Pl, cudaStream_t st, bool* used) {
    switch (Pl->p) {
        case 3: return treep<3>(Pl, st, used);
        case 5: return treep<5>(Pl, st, used);
        case 7: return treep<7>(Pl, st, used);
        default: *used = false; return DWT_OK;
    }
}

}  // namespace dwt
