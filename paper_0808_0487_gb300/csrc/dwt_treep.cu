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
// done on all digits at once.  A net of at most one small tile runs in one
// CTA, larger ones in the tiled form below.  Nets outside m <= 16 and the shared-memory
// limits of the coarse tree (p = 3: m <= 16, p = 5: m <= 11, p = 7: m <= 8),
// or with dependent rows, use the per-digit programme.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dwt_grid.cuh"
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

constexpr int cpow_i(int b, int e) { return e == 0 ? 1 : b * cpow_i(b, e - 1); }

// the smaller tiles of the tiled form for nets of fewer than 64 full tiles:
// 3^5, 5^3, 7^2 labels, one CTA of NT threads each
template <int P> struct SmallTile;
template <> struct SmallTile<3> { static constexpr int LB = 5, NT = 256; };
template <> struct SmallTile<5> { static constexpr int LB = 3, NT = 128; };
template <> struct SmallTile<7> { static constexpr int LB = 2, NT = 64; };

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

// the least of the p - 1 siblings of node v (children of v's parent other than v)
template <int P>
__device__ __forceinline__ unsigned sib_min(const uint8_t* S, uint32_t v) {
    const uint32_t b = v - v % P;
    unsigned x = kInfP;
#pragma unroll
    for (int c = 0; c < P; ++c)
        if (b + c != v) x = min(x, (unsigned)S[b + c]);
    return x;
}

// ---------------------------------------------------------------------------
// The tiled form for nets of more than one tile.  Tiles of p^LB labels, one
// CTA each: 3^8, 5^5, 7^4 labels (512 threads), or for nets of fewer than 64
// such tiles the smaller 3^5, 5^3, 7^2 (SmallTile), so that more CTAs share a
// coordinate; the levels 0 .. LB of every tile in a global array laid out
// level after level over all N labels; the levels above, built from the tile
// minima (level LB) in every CTA's shared memory.
//
// Backward sweep, one cooperative launch with two grid-wide waits per
// coordinate j = s-2 .. 0 (T_{s-1} and k_{s-1} have a closed form):
//   up    leaves T'[U] = T_{j+1}[Q_j(U)] of every tile and the tile's levels;
//   wait
//   down  the coarse tree, A from the tile root to the leaves, T_j =
//         min(T', A_0) and the digit vector k_j(U) of the representative
//         (top digit a >= 1 at position d-1, then the lower digits, each the
//         smallest a whose node keeps S_i + d = T_j), which depends on U
//         alone; T_j replaces T_{j+1} in place, k_j goes to K[j][U];
//   wait  (T_j complete before coordinate j-1 gathers from it).
// Forward reading, one ordinary launch: every label H follows
//   U_0 = I_0(H),  k_j = K[j][U_j],  U_{j+1} = Q_j(U_j - k_j digit-wise)
// and multiplies its weight denominator by (1 + k_j)^2.
constexpr int kFwdLP = 8;   // labels per thread of the forward reading

struct ArgsP {
    const MapP* Q;     // Q_j, j = 0 .. s-2
    uint8_t* T;        // N bytes: T_{j+1} before coordinate j's down pass, T_j after
    uint32_t* K;       // s x N: k_j(U)
    uint8_t* lev;      // levels 0 .. LB over all N labels
    unsigned* flags;   // [0] max T_0, [1] weight overflow, [2] a wait gave up, [3] arrivals
    long long N;
    int m, s, ng;
};

// per-level constants of the tiled sweep (shared memory, set once per launch):
// pw[i] = p^i; for i <= LB the offset of level i in a tile's levels (toff) and
// in the global levels (goff), and the nodes of level i per tile (per); for
// i >= LB the offset of level i in the coarse tree (coff)
struct LevelsP {
    uint32_t pw[33], toff[17], goff[17], per[17], coff[33];
};

// a tile of the tiled form: P^LB labels
template <int P, int LB_>
struct TileP {
    static constexpr int LB = LB_;
    static constexpr int TS = cpow_i(P, LB_);
};

// dynamic shared memory of the backward sweep: map | tile levels | A, A' | ok | coarse levels
template <int P, int LB>
struct SmemP {
    static constexpr int TS = TileP<P, LB>::TS;
    static constexpr size_t kMap = sizeof(MapP);
    static constexpr size_t kLev = ((size_t)2 * TS + 15) & ~(size_t)15;
    static constexpr size_t kA = ((size_t)2 * TS * 2 + 15) & ~(size_t)15;
    static constexpr size_t kFixed = kMap + kLev + kA + 16 + ((sizeof(LevelsP) + 15) & ~(size_t)15);
    static size_t bytes(long long nLB) { return kFixed + (((size_t)2 * nLB + 15) & ~(size_t)15); }
};

template <int P, int LB>
__device__ void levels_init(LevelsP* L, long long N, int m) {
    using SH = TileP<P, LB>;
    if (threadIdx.x == 0) {
        const long long nLB = N / SH::TS;
        long long w = 1;
        for (int i = 0; i <= m; ++i) {
            L->pw[i] = (uint32_t)w;
            if (i <= SH::LB) {
                long long per = 1;
                for (int l = i; l < SH::LB; ++l) per *= P;
                L->per[i] = (uint32_t)per;
                L->toff[i] = (uint32_t)loffP<P>(SH::TS, per);
                L->goff[i] = (uint32_t)loffP<P>(N, N / w);
            }
            if (i >= SH::LB) L->coff[i] = (uint32_t)loffP<P>(nLB, N / w);
            w *= P;
        }
    }
}

template <int P, int LB>
__device__ __forceinline__ void tileP_up(const ArgsP& a, uint32_t tile, const unsigned long long (*q)[256],
                                         uint8_t* sl, const LevelsP* L) {
    using SH = TileP<P, LB>;
    const uint32_t base = tile * (uint32_t)SH::TS;
    for (int e = threadIdx.x; e < SH::TS; e += blockDim.x) {
        const uint32_t U = base + (uint32_t)e;
        const uint8_t v = a.T[applyP<P>(q, U, a.ng, a.m)];
        sl[e] = v;
        a.lev[U] = v;
    }
    __syncthreads();
    for (int i = 1; i <= SH::LB; ++i) {
        const int np = (int)L->per[i];   // nodes of level i in the tile
        const uint8_t* src = sl + L->toff[i - 1];
        uint8_t* dst = sl + L->toff[i];
        uint8_t* gdst = a.lev + L->goff[i] + (size_t)tile * (uint32_t)np;
        for (int v = threadIdx.x; v < np; v += blockDim.x) {
            unsigned x = src[P * v];
#pragma unroll
            for (int c = 1; c < P; ++c) x = min(x, (unsigned)src[P * v + c]);
            dst[v] = (uint8_t)x;
            gdst[v] = (uint8_t)x;
        }
        __syncthreads();
    }
}

template <int P, int LB>
__device__ __forceinline__ void tileP_down(const ArgsP& a, uint32_t tile, int j, const uint8_t* cl, uint8_t* sl,
                                           uint16_t* a0, uint16_t* a1, const LevelsP* L, unsigned& mx) {
    using SH = TileP<P, LB>;
    const long long N = a.N;
    const int m = a.m;
    const uint32_t base = tile * (uint32_t)SH::TS;
    for (int i = 0; i < SH::LB; ++i) {
        const int n = (int)L->per[i];
        const uint8_t* g = a.lev + L->goff[i] + (size_t)tile * (uint32_t)n;
        uint8_t* d = sl + L->toff[i];
        for (int v = threadIdx.x; v < n; v += blockDim.x) d[v] = g[v];
    }
    if (threadIdx.x == 0) {
        // A at the tile root, down the coarse tree: node tile / p^(i - LB) of level i
        unsigned av = kInfP, ad = 0;
        for (int i = m - 1; i >= SH::LB; --i) {
            const uint32_t node = tile / L->pw[i - SH::LB];
            const unsigned c = sat_addP(sib_min<P>(cl + L->coff[i], node), (unsigned)(i + 1));
            if (c <= av) {
                av = c;
                ad = (unsigned)(i + 1);
            }
        }
        a0[0] = (uint16_t)(av | (ad << 8));
    }
    __syncthreads();
    uint16_t* cur = a0;
    uint16_t* nxt = a1;
    for (int i = SH::LB - 1; i >= 0; --i) {
        const int ni = (int)L->per[i];
        const uint8_t* S = sl + L->toff[i];
        for (int v = threadIdx.x; v < ni; v += blockDim.x) {
            const uint16_t par = cur[v / P];
            const unsigned c = sat_addP(sib_min<P>(S, (uint32_t)v), (unsigned)(i + 1));
            nxt[v] = c <= (unsigned)(par & 255) ? (uint16_t)(c | ((unsigned)(i + 1) << 8)) : par;
        }
        __syncthreads();
        uint16_t* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    for (int e = threadIdx.x; e < SH::TS; e += blockDim.x) {
        const unsigned t = sl[e], A = cur[e];
        const bool keep = t <= (A & 255);
        const int tau = (int)(keep ? t : (A & 255));
        const int d = keep ? 0 : (int)(A >> 8);
        const uint32_t U = base + (uint32_t)e;
        uint32_t k = 0;
        if (d) {
            // digits 0 .. d-1 of U (4 bits each); the reading changes digit i at level i only
            unsigned long long dg = 0;
            uint32_t x = U;
            for (int c = 0; c < d; ++c) {
                dg |= (unsigned long long)(x % P) << (4 * c);
                x /= P;
            }
            uint32_t node = x;                 // node of level d above U
            bool own = d - 1 < SH::LB;         // below level LB the nodes lie in this tile
            for (int i = d - 1; i >= 0; --i) {
                if (i == SH::LB - 1 && !own) own = node == tile;
                const uint32_t u = (uint32_t)(dg >> (4 * i)) & 15u;
                int av = i == d - 1 ? 1 : 0;
                uint32_t un = u;
                for (; av < P; ++av) {
                    un = u >= (uint32_t)av ? u - (uint32_t)av : u + P - (uint32_t)av;
                    const uint32_t cand = node * P + un;
                    unsigned v;
                    if (i >= SH::LB) v = cl[L->coff[i] + cand];
                    else if (own) v = sl[L->toff[i] + (cand - tile * L->per[i])];
                    else v = a.lev[L->goff[i] + cand];
                    if ((int)v + d == tau) break;
                }
                if (av == P) av = P - 1;   // unreachable for a consistent table
                node = node * P + un;
                k += (uint32_t)av * L->pw[i];
            }
        }
        a.T[U] = (uint8_t)tau;
        a.K[(size_t)j * N + U] = k;
        if (j == 0) mx = max(mx, (unsigned)tau);
    }
}

template <int P, int LB, int NT>
__global__ void __launch_bounds__(NT) k_treep_bwd(ArgsP a) {
    using SH = TileP<P, LB>;
    using L = SmemP<P, LB>;
    extern __shared__ __align__(16) unsigned char sm[];
    unsigned long long (*q)[256] = reinterpret_cast<unsigned long long (*)[256]>(sm);
    uint8_t* sl = sm + L::kMap;
    uint16_t* a0 = reinterpret_cast<uint16_t*>(sm + L::kMap + L::kLev);
    uint16_t* a1 = a0 + SH::TS;
    int* ok = reinterpret_cast<int*>(sm + L::kMap + L::kLev + L::kA);
    LevelsP* lv = reinterpret_cast<LevelsP*>(sm + L::kMap + L::kLev + L::kA + 16);
    uint8_t* cl = sm + L::kFixed;
    const long long N = a.N;
    const long long nLB = N / SH::TS;
    const int top = a.m - SH::LB;
    unsigned target = 0, mx = 0;
    levels_init<P, LB>(lv, N, a.m);
    __syncthreads();   // per-level constants
    for (int j = a.s - 1; j >= 0; --j) {
        if (j == a.s - 1) {
            // T_s is 0 at label 0 only, so T_{s-1}(U) = (position of the highest
            // nonzero digit of U) + 1 with the reading running down to label 0:
            // k_{s-1}(U) = U
            for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < N;
                 v += (long long)gridDim.x * blockDim.x) {
                const uint32_t U = (uint32_t)v;
                int n = 0;
                while (n < a.m && U >= lv->pw[n]) ++n;
                a.T[U] = (uint8_t)n;
                a.K[(size_t)j * N + U] = U;
                if (j == 0) mx = max(mx, (unsigned)n);
            }
            if (j > 0 && !grid_wait(a.flags, target, ok)) return;
            continue;
        }
        load_mapP<P>(q, a.Q + j, a.ng);
        __syncthreads();
        for (long long tl = blockIdx.x; tl < nLB; tl += gridDim.x) {
            tileP_up<P, LB>(a, (uint32_t)tl, q, sl, lv);
            __syncthreads();
        }
        if (!grid_wait(a.flags, target, ok)) return;
        // the coarse tree: level LB (tile minima) .. m
        for (long long v = threadIdx.x; v < nLB; v += blockDim.x) cl[v] = a.lev[lv->goff[SH::LB] + v];
        __syncthreads();
        long long n = nLB;
        for (int i = 1; i <= top; ++i) {
            const long long np = n / P;
            const uint8_t* src = cl + loffP<P>(nLB, n);
            uint8_t* dst = cl + loffP<P>(nLB, np);
            for (long long v = threadIdx.x; v < np; v += blockDim.x) {
                unsigned x = src[P * v];
#pragma unroll
                for (int c = 1; c < P; ++c) x = min(x, (unsigned)src[P * v + c]);
                dst[v] = (uint8_t)x;
            }
            __syncthreads();
            n = np;
        }
        for (long long tl = blockIdx.x; tl < nLB; tl += gridDim.x) {
            tileP_down<P, LB>(a, (uint32_t)tl, j, cl, sl, a0, a1, lv, mx);
            __syncthreads();
        }
        if (j > 0 && !grid_wait(a.flags, target, ok)) return;
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(a.flags, mx);
}

// a linear map applied from global memory (tables read through the read-only cache)
template <int P>
__device__ __forceinline__ uint32_t applyP_ldg(const MapP* M, uint32_t x, int ng, int m) {
    unsigned long long v = 0;
    for (int g = 0; g < ng; ++g) {
        const uint32_t q = x / TreeShape<P>::PG;
        v = padd<P>(v, __ldg(&M->t[g][x - q * TreeShape<P>::PG]));
        x = q;
    }
    return unpack<P>(v, m);
}

// U minus k, digit by digit mod p
template <int P>
__device__ __forceinline__ uint32_t sub_digits(uint32_t U, uint32_t k) {
    uint32_t r = 0, pw = 1;
    while (k) {
        const uint32_t ud = U % P, kd = k % P;
        U /= P;
        k /= P;
        r += ((ud + P - kd) % P) * pw;
        pw *= P;
    }
    return r + U * pw;
}

template <int P>
__global__ void __launch_bounds__(256) k_treep_read(const uint32_t* __restrict__ K, const MapP* __restrict__ I0,
                                                    const MapP* __restrict__ Q, unsigned* flags, float* W,
                                                    uint8_t* cls, long long N, int m, int s, int ng) {
    if (flags[0] >= kInfP || flags[2]) return;   // the backward sweep did not finish: nothing to read
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long h0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    uint32_t U[kFwdLP];
    unsigned long long pd[kFwdLP];
    uint32_t c[kFwdLP];   // last coordinate with k_j != 0 | count << 8
#pragma unroll
    for (int l = 0; l < kFwdLP; ++l) {
        const long long H = h0 + l * stride;
        U[l] = H < N ? applyP_ldg<P>(I0, (uint32_t)H, ng, m) : 0u;
        pd[l] = 1ull;
        c[l] = 0u;
    }
    bool over = false;
    for (int j = 0; j < s; ++j) {
        const uint32_t* Kj = K + (size_t)j * N;
#pragma unroll
        for (int l = 0; l < kFwdLP; ++l) {
            if (h0 + l * stride >= N) continue;
            const uint32_t k = __ldg(Kj + U[l]);
            if (k) {
                const unsigned long long qq = (unsigned long long)k + 1ull, q2 = qq * qq;
                if (__umul64hi(pd[l], q2) != 0ull) over = true;
                pd[l] *= q2;
                c[l] = (uint32_t)(j + 1) | (((c[l] >> 8) + 1u) << 8);
            }
            if (j + 1 < s) U[l] = applyP_ldg<P>(Q + j, sub_digits<P>(U[l], k), ng, m);
        }
    }
#pragma unroll
    for (int l = 0; l < kFwdLP; ++l) {
        const long long H = h0 + l * stride;
        if (H >= N) continue;
        W[H] = __fdiv_rn(1.0f, __ull2float_rn(pd[l]));
        cls[2 * H] = (uint8_t)(c[l] & 255u);
        cls[2 * H + 1] = (uint8_t)(c[l] >> 8);
    }
    if (over) atomicExch(flags + 1, 1u);
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
    // entry x of group g: the entry with x's lowest nonzero digit (position l,
    // value a) cleared, plus a * column gG + l -- one digit-wise addition each
    for (int g = 0; g < kMaxGroups; ++g) {
        M.t[g][0] = 0ull;
        for (int x = 1; x < 256; ++x) {
            if (g >= ng || x >= SH::PG) {
                M.t[g][x] = 0ull;
                continue;
            }
            int y = x, l = 0, w = 1;
            while (y % P == 0) {
                y /= P;
                ++l;
                w *= P;
            }
            const int a = y % P, i = g * SH::G + l;
            M.t[g][x] = i < m ? padd<P>(M.t[g][x - a * w], mult[(size_t)i * P + a]) : M.t[g][x - a * w];
        }
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

// Largest cooperative grid of the backward sweep (see the p = 2 form);
// DWT_TILE_GRID, if set to a positive number, caps it.
template <int P, int LB, int NT>
int treep_grid(long long tiles, size_t smem) {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_treep_bwd<P, LB, NT>, NT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    long long g = std::min(tiles, (long long)occ * sms);
    const char* e = getenv("DWT_TILE_GRID");
    const long long cap = e ? atoll(e) : 0;
    if (cap > 0) g = std::min(g, cap);
    return (int)g;
}

// The tiled form: one cooperative launch for the backward sweep, one launch
// for the forward reading, one synchronisation.
template <int P, int LB, int NT>
int treep_tiles(dwt_plan_s* Pl, const MapP& I0, const std::vector<MapP>& Qmap, int ng, cudaStream_t st) {
    using SH = TileP<P, LB>;
    const long long N = Pl->N;
    const int m = Pl->m, s = Pl->s;
    const long long tiles = N / SH::TS;
    // one scratch block: flags (16 B, padded), the maps I_0, Q_0 .. Q_{s-2},
    // then T, the levels and K (256-byte aligned pieces)
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_maps = 256, o_T = al(o_maps + sizeof(MapP) * s), o_lev = al(o_T + (size_t)N),
                 o_K = al(o_lev + (size_t)N * 2), total = al(o_K + (size_t)s * N * 4);
    unsigned char* ws = nullptr;
    auto cleanup = [&]() { dfree(ws, st); };
    int rc = DWT_OK;
    // CUDA failures after the allocation release the scratch block first
    auto ck = [&](cudaError_t e, const char* what) -> int {
        if (e == cudaSuccess) return DWT_OK;
        cleanup();
        return cuda_fail(e, what, __FILE__, __LINE__);
    };
    if (dmalloc((void**)&ws, total, st) || dmalloc((void**)&Pl->d_W, (size_t)N * 4, st) ||
        dmalloc((void**)&Pl->d_cls, (size_t)N * 2, st)) {
        cleanup();
        return DWT_ENOMEM;
    }
    unsigned* flags = reinterpret_cast<unsigned*>(ws);
    MapP* dmaps = reinterpret_cast<MapP*>(ws + o_maps);
    uint8_t* T = ws + o_T;
    uint8_t* lev = ws + o_lev;
    uint32_t* K = reinterpret_cast<uint32_t*>(ws + o_K);
    // flags zeroed and the maps in one upload, from page-locked staging when
    // there is some (the stream is synchronised below, before it is reused)
    const size_t nb = o_maps + sizeof(MapP) * s;
    std::vector<unsigned char> hv;
    unsigned char* hb = host_staging(nb);
    if (!hb) {
        hv.resize(nb);
        hb = hv.data();
    }
    memset(hb, 0, o_maps);
    memcpy(hb + o_maps, &I0, sizeof(MapP));
    for (int j = 0; j + 1 < s; ++j) memcpy(hb + o_maps + sizeof(MapP) * (1 + j), &Qmap[j], sizeof(MapP));
    if ((rc = ck(cudaMemcpyAsync(ws, hb, nb, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync"))) return rc;
    const size_t smem = SmemP<P, LB>::bytes(tiles);
    rc = smem_limit_max(k_treep_bwd<P, LB, NT>);
    if (rc) { cleanup(); return rc; }
    const int grid = treep_grid<P, LB, NT>(tiles, smem);
    if (grid < 1) {
        cleanup();
        set_error("no resident grid for the tiled coset-table sweep (%zu bytes of shared memory)", smem);
        return DWT_ECUDA;
    }
    ArgsP A;
    A.Q = dmaps + 1;
    A.T = T;
    A.K = K;
    A.lev = lev;
    A.flags = flags;
    A.N = N;
    A.m = m;
    A.s = s;
    A.ng = ng;
    {
        LaunchScope ls("tree_sweep", st);
        void* args[] = {&A};
        if ((rc = ck(cudaLaunchCooperativeKernel((const void*)k_treep_bwd<P, LB, NT>, dim3((unsigned)grid), dim3(NT),
                                                 args, smem, st),
                     "cooperative launch")))
            return rc;
    }
    {
        const long long per_cta = 256ll * kFwdLP;
        const unsigned fg = (unsigned)((N + per_cta - 1) / per_cta);
        LaunchScope ls("tree_read", st);
        k_treep_read<P><<<fg, 256, 0, st>>>(K, dmaps, dmaps + 1, flags, Pl->d_W, Pl->d_cls, N, m, s, ng);
    }
    if ((rc = ck(cudaGetLastError(), "tiled coset tables"))) return rc;
    unsigned hf[4] = {0, 0, 0, 0};
    if ((rc = ck(cudaMemcpyAsync(hf, flags, 16, cudaMemcpyDeviceToHost, st), "cudaMemcpyAsync"))) return rc;
    if ((rc = ck(cudaStreamSynchronize(st), "cudaStreamSynchronize"))) return rc;
    cleanup();
    if (hf[2]) {
        set_error("tiled coset tables: a grid-wide wait gave up");
        return DWT_ETIMEOUT;
    }
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
        if (m <= SmallTile<P>::LB) make_mapP<P>(rows[j], m, Fmap[j]);   // only the one-CTA form reads F_j
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
    // nets of few full tiles run on smaller tiles (more CTAs per coordinate);
    // a net of at most one small tile in one CTA
    constexpr int LBs = SmallTile<P>::LB;
    if (m <= LBs) return treep_one<P>(Pl, Imap, Fmap, Qmap, ng, st);
    if (N / SH::TS < 64) return treep_tiles<P, LBs, SmallTile<P>::NT>(Pl, Imap[0], Qmap, ng, st);
    return treep_tiles<P, SH::LB, kThreadsP>(Pl, Imap[0], Qmap, ng, st);
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
