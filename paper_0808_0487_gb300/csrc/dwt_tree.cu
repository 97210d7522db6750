// dwt_tree.cu -- the coset representatives K(C) (Sec. 2.1) for p = 2 in
// O(s N) work: the same least-nu / lexicographic answer as the coordinate
// dynamic programme of dwt_index.cu, organised so that each coordinate costs
// one bottom-up and one top-down sweep over a binary tree instead of m sweeps
// over all labels.
//
// For coordinate j let r_0 .. r_{m-1} be the labels of the rows of C_j and,
// when they are linearly independent, U(h) the coordinates of a label h in
// that basis (h = XOR of r_i over the set bits i of U).  The prefix minima of
// the programme, M_i[h] = min over h + span(r_0 .. r_{i-1}) of T_{j+1}, are
// then the minima of T'[U] = T_{j+1}[h(U)] over the 2^i labels that share the
// bits >= i of U: the node U >> i of level i of the min-tree S over T'.  The
// candidate with nu(k_j) = d is d + min_{a != 0} M_{d-1}[h - a r_{d-1}], the
// sibling S_{d-1}[(U >> (d-1)) ^ 1], so
//     T_j = min(T'[U], A_0[U]),   A_i[V] = min(i+1 + S_i[V ^ 1], A_{i+1}[V >> 1]),
// with A_m = infinity, keeping the smallest d on ties (T' first), exactly as
// the per-digit sweep does.  The representative is read forward coordinate by
// coordinate as before; its per-digit tests M_i[g] + d = tau become lookups
// S_i[U(g) >> i] in the tree of T_{j+1}.
//
// Tables are kept in the coordinates of their own coordinate's basis (T^U_j);
// consecutive coordinates are linked by the F_2-linear map U_j -> U_{j+1}.
// Linear maps are applied as four 256-entry XOR tables (one per byte).  The
// tree levels below 2^13 labels live in shared memory per tile; the levels
// above come from one small CTA.  Nets whose row sets are dependent, and
// m > 27, use the per-digit programme.
#include <algorithm>
#include <vector>

#include "dwt_internal.cuh"

namespace dwt {

namespace {

constexpr int kLB = 13;          // tile: 2^13 labels (levels 0 .. 13 in shared memory)
constexpr int kThreads = 512;
constexpr uint8_t kInfB = 255;

struct Map4 {
    uint32_t t[4][256];
};

__device__ __forceinline__ uint32_t apply4(const uint32_t (*t)[256], uint32_t x) {
    return t[0][x & 255] ^ t[1][(x >> 8) & 255] ^ t[2][(x >> 16) & 255] ^ t[3][x >> 24];
}

// byte offset of level i in a tree stored level after level over n leaves
__host__ __device__ __forceinline__ long long loff(long long n, int i) { return 2 * n - ((2 * n) >> i); }

__device__ __forceinline__ unsigned sat_add(unsigned v, unsigned d) {
    if (v >= kInfB) return kInfB;
    const unsigned c = v + d;
    return c > kInfB ? kInfB : c;
}

__device__ __forceinline__ void load_map(uint32_t (*sm)[256], const Map4* g) {
    for (int i = threadIdx.x; i < 4 * 256; i += blockDim.x) sm[i >> 8][i & 255] = g->t[i >> 8][i & 255];
}

// Leaves T'[U] = Tprev[Q(U)] (or, with no Tprev, the start T_{s+1}: 0 at U = 0,
// infinite elsewhere) of one 2^LB tile and the tile's tree levels 0 .. LB,
// written to the global level array.
__global__ void __launch_bounds__(kThreads) k_tree_up(const uint8_t* __restrict__ Tprev, const Map4* __restrict__ Q,
                                                      uint8_t* lev, long long N, int LB) {
    __shared__ uint32_t q[4][256];
    __shared__ uint8_t sl[2 << kLB];
    const int TS = 1 << LB;
    const long long base = (long long)blockIdx.x << LB;
    if (Tprev) load_map(q, Q);
    __syncthreads();
    for (int e = threadIdx.x; e < TS; e += blockDim.x) {
        const uint32_t U = (uint32_t)(base + e);
        const uint8_t v = Tprev ? Tprev[apply4(q, U)] : (U == 0 ? 0 : kInfB);
        sl[e] = v;
        lev[base + e] = v;
    }
    __syncthreads();
    for (int i = 1; i <= LB; ++i) {
        const int n = TS >> i;
        const uint8_t* src = sl + loff(TS, i - 1);
        uint8_t* dst = sl + loff(TS, i);
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            const uint8_t x = min(src[2 * v], src[2 * v + 1]);
            dst[v] = x;
            lev[loff(N, i) + (base >> i) + v] = x;
        }
        __syncthreads();
    }
}

// Levels LB+1 .. m of the tree from level LB (one CTA); with want_a, also the
// top-down minima A for levels m-1 .. LB, stored per level-LB node as
// (value | d << 8).  Dynamic shared memory: 2 * nLB bytes of levels and
// 2 * nLB uint16 of A.
__global__ void __launch_bounds__(1024) k_tree_coarse(uint8_t* lev, uint16_t* Aout, long long N, int m, int LB,
                                                      int want_a) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int nLB = (int)(N >> LB);
    uint8_t* sl = sm;                                              // levels LB.. : level LB+i at loff(nLB, i)
    uint16_t* A0 = reinterpret_cast<uint16_t*>(sm + ((2 * nLB + 15) & ~15));
    uint16_t* A1 = A0 + nLB;
    const int top = m - LB;                                        // levels above LB
    for (int v = threadIdx.x; v < nLB; v += blockDim.x) sl[v] = lev[loff(N, LB) + v];
    __syncthreads();
    for (int i = 1; i <= top; ++i) {
        const int n = nLB >> i;
        const uint8_t* src = sl + loff(nLB, i - 1);
        uint8_t* dst = sl + loff(nLB, i);
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            const uint8_t x = min(src[2 * v], src[2 * v + 1]);
            dst[v] = x;
            lev[loff(N, LB + i) + v] = x;
        }
        __syncthreads();
    }
    if (!want_a) return;
    // A at level m: one node, infinite
    uint16_t* cur = A0;
    uint16_t* nxt = A1;
    if (threadIdx.x == 0) cur[0] = kInfB;
    __syncthreads();
    for (int i = m - 1; i >= LB; --i) {
        const int n = (int)(N >> i);
        const uint8_t* S = sl + loff(nLB, i - LB);
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            const uint16_t par = cur[v >> 1];
            const unsigned c = sat_add(S[v ^ 1], (unsigned)(i + 1));
            nxt[v] = c <= (unsigned)(par & 255) ? (uint16_t)(c | ((unsigned)(i + 1) << 8)) : par;
        }
        __syncthreads();
        uint16_t* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    for (int v = threadIdx.x; v < nLB; v += blockDim.x) Aout[v] = cur[v];
}

// Top-down minima through one tile's levels LB-1 .. 0 and the coordinate's
// tables in its own basis: TU = min(T', A_0), DU = 0 if T' <= A_0 else d.
__global__ void __launch_bounds__(kThreads) k_tree_down(const uint8_t* __restrict__ lev,
                                                        const uint16_t* __restrict__ Acoarse, uint8_t* TU, uint8_t* DU,
                                                        long long N, int LB) {
    __shared__ uint8_t sl[2 << kLB];
    __shared__ uint16_t a0[1 << kLB], a1[1 << kLB];
    const int TS = 1 << LB;
    const long long base = (long long)blockIdx.x << LB;
    for (int i = 0; i < LB; ++i) {
        const int n = TS >> i;
        for (int v = threadIdx.x; v < n; v += blockDim.x) sl[loff(TS, i) + v] = lev[loff(N, i) + (base >> i) + v];
    }
    if (threadIdx.x == 0) a0[0] = Acoarse[blockIdx.x];
    __syncthreads();
    uint16_t* cur = a0;
    uint16_t* nxt = a1;
    for (int i = LB - 1; i >= 0; --i) {
        const int n = TS >> i;
        const uint8_t* S = sl + loff(TS, i);
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            const uint16_t par = cur[v >> 1];
            const unsigned c = sat_add(S[v ^ 1], (unsigned)(i + 1));
            nxt[v] = c <= (unsigned)(par & 255) ? (uint16_t)(c | ((unsigned)(i + 1) << 8)) : par;
        }
        __syncthreads();
        uint16_t* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    for (int e = threadIdx.x; e < TS; e += blockDim.x) {
        const unsigned t = sl[e], a = cur[e];
        const bool keep = t <= (a & 255);
        TU[base + e] = keep ? (uint8_t)t : (uint8_t)(a & 255);
        DU[base + e] = keep ? 0 : (uint8_t)(a >> 8);
    }
}

// Forward reading of coordinate j for every coset label: g (remaining label),
// U = U_j(g), tau = TU_j[U], d = DU_j[U]; the top digit of k_j is d-1, then the
// lower digits smallest-first against the tree of T_{j+1} (lev).
__global__ void __launch_bounds__(kThreads) k_tree_recon(uint32_t* G, unsigned long long* Pden, uint8_t* cls,
                                                         int* overflow, const uint8_t* __restrict__ TU,
                                                         const uint8_t* __restrict__ DU, const uint8_t* __restrict__ lev,
                                                         const Map4* __restrict__ Ij, const uint32_t* __restrict__ Rj,
                                                         int j, int m, long long N) {
    __shared__ uint32_t inv[4][256];
    __shared__ uint32_t r[32];
    load_map(inv, Ij);
    if (threadIdx.x < m) r[threadIdx.x] = Rj[threadIdx.x];
    __syncthreads();
    for (long long H = blockIdx.x * (long long)blockDim.x + threadIdx.x; H < N; H += (long long)gridDim.x * blockDim.x) {
        uint32_t g = G[H];
        uint32_t U = apply4(inv, g);
        const int tau = TU[U], d = DU[U];
        if (!d) continue;
        uint32_t k = 1u << (d - 1);
        U ^= k;
        g ^= r[d - 1];
        for (int i = d - 2; i >= 0; --i) {
            const int s = lev[loff(N, i) + (U >> i)];
            if (s + d != tau) {
                U ^= 1u << i;
                g ^= r[i];
                k |= 1u << i;
            }
        }
        G[H] = g;
        const unsigned long long q = (unsigned long long)k + 1ull, q2 = q * q;
        const unsigned long long pd = Pden[H];
        if (__umul64hi(pd, q2) != 0ull) *overflow = 1;
        Pden[H] = pd * q2;
        cls[2 * H] = (uint8_t)(j + 1);
        cls[2 * H + 1] = (uint8_t)(cls[2 * H + 1] + 1);
    }
}

__global__ void k_tree_max(const uint8_t* __restrict__ a, long long N, unsigned* out) {
    unsigned mx = 0;
    for (long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x; h < N; h += (long long)gridDim.x * blockDim.x)
        mx = max(mx, (unsigned)a[h]);
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

__global__ void k_tree_init(uint32_t* G, unsigned long long* Pden, uint8_t* cls, long long N) {
    for (long long H = blockIdx.x * (long long)blockDim.x + threadIdx.x; H < N; H += (long long)gridDim.x * blockDim.x) {
        G[H] = (uint32_t)H;
        Pden[H] = 1ull;
        cls[2 * H] = 0;
        cls[2 * H + 1] = 0;
    }
}

__global__ void k_tree_weights(const unsigned long long* __restrict__ Pden, float* W, long long N) {
    for (long long H = blockIdx.x * (long long)blockDim.x + threadIdx.x; H < N; H += (long long)gridDim.x * blockDim.x)
        W[H] = __fdiv_rn(1.0f, __ull2float_rn(Pden[H]));
}

// The whole construction for a net of N = 2^m <= 2^13 labels in one CTA: both
// sweeps over all coordinates with the tree, the previous coordinate's table
// and the maps in shared memory, and each thread carrying the reading state of
// its labels H = t + 1024 q in registers.  One launch per plan.
constexpr int kOneMax = 1 << kLB;
constexpr int kOneQ = kOneMax / 1024;

__global__ void __launch_bounds__(1024, 1) k_tree_one(const Map4* __restrict__ Imaps, const Map4* __restrict__ Qmaps,
                                                      const uint32_t* __restrict__ R, int m, int s, uint8_t* TU,
                                                      uint8_t* DU, uint8_t* cls, float* W, unsigned* flags) {
    extern __shared__ __align__(16) unsigned char sm[];
    uint32_t (*mq)[256] = reinterpret_cast<uint32_t (*)[256]>(sm);               // Q_j
    uint32_t (*mi)[256] = reinterpret_cast<uint32_t (*)[256]>(sm + 4096);        // I_j
    const int N = 1 << m;
    uint16_t* A0 = reinterpret_cast<uint16_t*>(sm + 8192);
    uint16_t* A1 = A0 + N;
    uint8_t* lv = reinterpret_cast<uint8_t*>(A1 + N);                             // 2N bytes of levels
    uint8_t* Tp = lv + 2 * N;                                                     // T of coordinate j+1
    uint32_t* r = reinterpret_cast<uint32_t*>(Tp + ((N + 15) & ~15));
    const int t = threadIdx.x;
    auto build_levels = [&](int j) {
        // leaves T'[U] = T_{j+1}[U_{j+1}(h(U))] and the levels above them
        for (int U = t; U < N; U += blockDim.x) lv[U] = j == s - 1 ? (U == 0 ? 0 : kInfB) : Tp[apply4(mq, U)];
        __syncthreads();
        for (int i = 1; i <= m; ++i) {
            const int n = N >> i;
            const uint8_t* src = lv + loff(N, i - 1);
            uint8_t* dst = lv + loff(N, i);
            for (int v = t; v < n; v += blockDim.x) dst[v] = min(src[2 * v], src[2 * v + 1]);
            __syncthreads();
        }
    };
    // backward sweep
    for (int j = s - 1; j >= 0; --j) {
        if (j < s - 1)
            for (int i = t; i < 1024; i += blockDim.x) mq[i >> 8][i & 255] = Qmaps[j].t[i >> 8][i & 255];
        __syncthreads();
        build_levels(j);
        uint16_t* cur = A0;
        uint16_t* nxt = A1;
        if (t == 0) cur[0] = kInfB;
        __syncthreads();
        for (int i = m - 1; i >= 0; --i) {
            const int n = N >> i;
            const uint8_t* S = lv + loff(N, i);
            for (int v = t; v < n; v += blockDim.x) {
                const uint16_t par = cur[v >> 1];
                const unsigned c = sat_add(S[v ^ 1], (unsigned)(i + 1));
                nxt[v] = c <= (unsigned)(par & 255) ? (uint16_t)(c | ((unsigned)(i + 1) << 8)) : par;
            }
            __syncthreads();
            uint16_t* tmp = cur;
            cur = nxt;
            nxt = tmp;
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
    // least total over every coset must stay below the saturation value
    {
        unsigned mx = 0;
        for (int U = t; U < N; U += blockDim.x) mx = max(mx, (unsigned)Tp[U]);
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((t & 31) == 0) atomicMax(flags, mx);
        __syncthreads();
        if (*(volatile unsigned*)flags >= kInfB) return;
    }
    // forward reading, labels H = t + 1024 q held by this thread
    uint32_t g[kOneQ];
    unsigned long long pd[kOneQ];
    uint8_t ct[kOneQ], cs[kOneQ];
#pragma unroll
    for (int q = 0; q < kOneQ; ++q) {
        g[q] = (uint32_t)(t + 1024 * q);
        pd[q] = 1ull;
        ct[q] = cs[q] = 0;
    }
    bool over = false;
    for (int j = 0; j < s; ++j) {
        __syncthreads();   // previous coordinate done with the maps and levels
        for (int i = t; i < 1024; i += blockDim.x) {
            mi[i >> 8][i & 255] = Imaps[j].t[i >> 8][i & 255];
            if (j < s - 1) mq[i >> 8][i & 255] = Qmaps[j].t[i >> 8][i & 255];
        }
        if (t < m) r[t] = R[(size_t)j * m + t];
        if (j < s - 1)
            for (int U = t; U < N; U += blockDim.x) Tp[U] = TU[(size_t)(j + 1) * N + U];
        __syncthreads();
        build_levels(j);
#pragma unroll
        for (int q = 0; q < kOneQ; ++q) {
            if (t + 1024 * q >= N) continue;
            uint32_t U = apply4(mi, g[q]);
            const int tau = TU[(size_t)j * N + U], d = DU[(size_t)j * N + U];
            if (!d) continue;
            uint32_t k = 1u << (d - 1);
            U ^= k;
            g[q] ^= r[d - 1];
            for (int i = d - 2; i >= 0; --i) {
                if ((int)lv[loff(N, i) + (U >> i)] + d != tau) {
                    U ^= 1u << i;
                    g[q] ^= r[i];
                    k |= 1u << i;
                }
            }
            const unsigned long long qq = (unsigned long long)k + 1ull, q2 = qq * qq;
            if (__umul64hi(pd[q], q2) != 0ull) over = true;
            pd[q] *= q2;
            ct[q] = (uint8_t)(j + 1);
            ++cs[q];
        }
    }
#pragma unroll
    for (int q = 0; q < kOneQ; ++q) {
        const int H = t + 1024 * q;
        if (H >= N) continue;
        W[H] = __fdiv_rn(1.0f, __ull2float_rn(pd[q]));
        cls[2 * H] = ct[q];
        cls[2 * H + 1] = cs[q];
    }
    if (over) atomicExch(flags + 1, 1u);
}

// inverse of the F_2 matrix with columns c[0 .. m-1] (bit a of c[i] = row a):
// ci[a] = B^{-1} e_a as a bit vector; false if singular
bool gf2_inverse(const uint32_t* c, int m, uint32_t* ci) {
    // rows of [B | I]: row a has B's row a in bits 0..m-1 and e_a in bits 32..
    std::vector<unsigned long long> row(m);
    for (int a = 0; a < m; ++a) {
        unsigned long long x = 0;
        for (int i = 0; i < m; ++i)
            if ((c[i] >> a) & 1u) x |= 1ull << i;
        row[a] = x | (1ull << (32 + a));
    }
    for (int col = 0; col < m; ++col) {
        int piv = -1;
        for (int a = col; a < m; ++a)
            if ((row[a] >> col) & 1ull) { piv = a; break; }
        if (piv < 0) return false;
        std::swap(row[col], row[piv]);
        for (int a = 0; a < m; ++a)
            if (a != col && ((row[a] >> col) & 1ull)) row[a] ^= row[col];
    }
    // row i now reads U_i = sum_a (bit 32+a) h_a: column a of B^{-1} collects bit 32+a of every row
    for (int a = 0; a < m; ++a) {
        uint32_t x = 0;
        for (int i = 0; i < m; ++i)
            if ((row[i] >> (32 + a)) & 1ull) x |= 1u << i;
        ci[a] = x;
    }
    return true;
}

void make_map(const uint32_t* cols, int m, Map4& M) {
    for (int b = 0; b < 4; ++b) {
        M.t[b][0] = 0;
        for (int x = 1; x < 256; ++x) {   // x = (x with its lowest set bit cleared) + that bit
            const int l = __builtin_ctz((unsigned)x);
            M.t[b][x] = M.t[b][x & (x - 1)] ^ (8 * b + l < m ? cols[8 * b + l] : 0u);
        }
    }
}

uint32_t host_apply(const Map4& M, uint32_t x) {
    return M.t[0][x & 255] ^ M.t[1][(x >> 8) & 255] ^ M.t[2][(x >> 16) & 255] ^ M.t[3][x >> 24];
}

unsigned grid_n(long long n) { return (unsigned)std::max(1ll, std::min((n + 255) / 256, 8ll * 152)); }

// the one-CTA form for N <= 2^13
int tree_one(dwt_plan_s* Pl, const std::vector<Map4>& Imap, const std::vector<Map4>& Qmap, cudaStream_t st) {
    const long long N = Pl->N;
    const int m = Pl->m, s = Pl->s;
    uint8_t *TU = nullptr, *DU = nullptr;
    Map4* dmaps = nullptr;
    unsigned* flags = nullptr;
    auto cleanup = [&]() {
        dfree(TU, st); dfree(DU, st); dfree(dmaps, st); dfree(flags, st);
    };
    if (dmalloc((void**)&TU, (size_t)s * N, st) || dmalloc((void**)&DU, (size_t)s * N, st) ||
        dmalloc((void**)&dmaps, sizeof(Map4) * 2 * s, st) || dmalloc((void**)&flags, 8, st) ||
        dmalloc((void**)&Pl->d_W, (size_t)N * 4, st) || dmalloc((void**)&Pl->d_cls, (size_t)N * 2, st)) {
        cleanup();
        return DWT_ENOMEM;
    }
    std::vector<Map4> hm(2 * s);
    for (int j = 0; j < s; ++j) {
        hm[j] = Imap[j];
        hm[s + j] = Qmap[j];
    }
    DWT_CK(cudaMemcpyAsync(dmaps, hm.data(), sizeof(Map4) * 2 * s, cudaMemcpyHostToDevice, st));
    DWT_CK(cudaMemsetAsync(flags, 0, 8, st));
    const size_t smem = 8192 + (size_t)4 * N + 2 * N + ((N + 15) & ~15ll) + 32 * 4;
    int rc = smem_limit_max(k_tree_one);
    if (rc) { cleanup(); return rc; }
    {
        LaunchScope ls("tree_one", st);
        k_tree_one<<<1, 1024, smem, st>>>(dmaps, dmaps + s, Pl->d_R, m, s, TU, DU, Pl->d_cls, Pl->d_W, flags);
    }
    DWT_CK_LAUNCH("k_tree_one");
    unsigned hf[2] = {0, 0};
    DWT_CK(cudaMemcpyAsync(hf, flags, 8, cudaMemcpyDeviceToHost, st));
    DWT_CK(cudaStreamSynchronize(st));
    cleanup();
    if (hf[0] >= kInfB) {
        set_error("a least nu over some coset reaches 255");
        return DWT_EUNSUPPORTED;
    }
    if (hf[1]) {
        set_error("a weight denominator prod (1+k_j)^2 exceeds 64 bits");
        return DWT_EUNSUPPORTED;
    }
    return DWT_OK;
}

}  // namespace

// Tables W, cls of a p = 2 plan by the tree form.  *used = false (nothing
// allocated or launched, DWT_OK returned) when a coordinate's rows are
// dependent or m > 27: the caller then runs the per-digit programme.
int coset_tables_tree2(dwt_plan_s* Pl, cudaStream_t st, bool* used) {
    const long long N = Pl->N;
    const int m = Pl->m, s = Pl->s;
    *used = false;
    if (Pl->p != 2 || m > 27 || m < 1) return DWT_OK;
    const std::vector<uint32_t>& R = Pl->R_host;
    // maps: I_j (labels -> U_j) and Q_j (U_j -> U_{j+1})
    std::vector<Map4> Imap(s), Qmap(s);
    std::vector<uint32_t> inv(m);
    std::vector<Map4> Fmap(s);
    for (int j = 0; j < s; ++j) {
        if (!gf2_inverse(&R[(size_t)j * m], m, inv.data())) return DWT_OK;
        make_map(inv.data(), m, Imap[j]);
        make_map(&R[(size_t)j * m], m, Fmap[j]);
    }
    for (int j = 0; j + 1 < s; ++j) {
        std::vector<uint32_t> qc(m);
        for (int i = 0; i < m; ++i) qc[i] = host_apply(Imap[j + 1], R[(size_t)j * m + i]);
        make_map(qc.data(), m, Qmap[j]);
    }
    *used = true;
    if (m <= kLB) return tree_one(Pl, Imap, Qmap, st);
    const int LB = std::min(m, kLB);
    const long long nLB = N >> LB;
    uint8_t *TU = nullptr, *DU = nullptr, *lev = nullptr;
    uint16_t* Ac = nullptr;
    Map4* dmaps = nullptr;
    uint32_t* G = nullptr;
    unsigned long long* Pden = nullptr;
    unsigned* flags = nullptr;
    auto cleanup = [&]() {
        dfree(TU, st); dfree(DU, st); dfree(lev, st); dfree(Ac, st); dfree(dmaps, st);
        dfree(G, st); dfree(Pden, st); dfree(flags, st);
    };
    if (dmalloc((void**)&TU, (size_t)s * N, st) || dmalloc((void**)&DU, (size_t)s * N, st) ||
        dmalloc((void**)&lev, (size_t)2 * N, st) || dmalloc((void**)&Ac, (size_t)2 * nLB, st) ||
        dmalloc((void**)&dmaps, sizeof(Map4) * 2 * s, st) || dmalloc((void**)&flags, 8, st)) {
        cleanup();
        return DWT_ENOMEM;
    }
    std::vector<Map4> hm(2 * s);
    for (int j = 0; j < s; ++j) {
        hm[j] = Imap[j];
        hm[s + j] = Qmap[j];
    }
    DWT_CK(cudaMemcpyAsync(dmaps, hm.data(), sizeof(Map4) * 2 * s, cudaMemcpyHostToDevice, st));
    DWT_CK(cudaMemsetAsync(flags, 0, 8, st));
    const Map4* dI = dmaps;
    const Map4* dQ = dmaps + s;
    const size_t coarse_smem = (size_t)((2 * nLB + 15) & ~15ll) + (size_t)4 * nLB;
    {
        int rc = smem_limit_max(k_tree_coarse);
        if (rc) { cleanup(); return rc; }
    }
    const unsigned tiles = (unsigned)nLB;
    // backward sweep
    for (int j = s - 1; j >= 0; --j) {
        const uint8_t* Tn = j + 1 < s ? TU + (size_t)(j + 1) * N : nullptr;
        {
            LaunchScope ls("tree_up", st);
            k_tree_up<<<tiles, kThreads, 0, st>>>(Tn, Tn ? dQ + j : nullptr, lev, N, LB);
        }
        {
            LaunchScope ls("tree_coarse", st);
            k_tree_coarse<<<1, 1024, coarse_smem, st>>>(lev, Ac, N, m, LB, 1);
        }
        {
            LaunchScope ls("tree_down", st);
            k_tree_down<<<tiles, kThreads, 0, st>>>(lev, Ac, TU + (size_t)j * N, DU + (size_t)j * N, N, LB);
        }
    }
    DWT_CK_LAUNCH("coset tree backward sweep");
    {
        LaunchScope ls("tree_check", st);
        k_tree_max<<<grid_n(N), 256, 0, st>>>(TU, N, flags);
    }
    unsigned mx = 0;
    DWT_CK(cudaMemcpyAsync(&mx, flags, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    DWT_CK(cudaStreamSynchronize(st));
    if (mx >= kInfB) {
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
        k_tree_init<<<grid_n(N), 256, 0, st>>>(G, Pden, Pl->d_cls, N);
    }
    int* over = reinterpret_cast<int*>(flags + 1);
    for (int j = 0; j < s; ++j) {
        const uint8_t* Tn = j + 1 < s ? TU + (size_t)(j + 1) * N : nullptr;
        {
            LaunchScope ls("tree_up", st);
            k_tree_up<<<tiles, kThreads, 0, st>>>(Tn, Tn ? dQ + j : nullptr, lev, N, LB);
        }
        if (m > LB) {
            LaunchScope ls("tree_coarse", st);
            k_tree_coarse<<<1, 1024, coarse_smem, st>>>(lev, Ac, N, m, LB, 0);
        }
        {
            LaunchScope ls("tree_recon", st);
            k_tree_recon<<<grid_n(N), kThreads, 0, st>>>(G, Pden, Pl->d_cls, over, TU + (size_t)j * N,
                                                         DU + (size_t)j * N, lev, dI + j, Pl->d_R + (size_t)j * m, j,
                                                         m, N);
        }
    }
    {
        LaunchScope ls("tree_weights", st);
        k_tree_weights<<<grid_n(N), 256, 0, st>>>(Pden, Pl->d_W, N);
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

}  // namespace dwt
