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
// Linear maps are applied as four 256-entry XOR tables (one per byte).  Nets
// of up to 2^11 labels run in one CTA; larger ones in tiles of 2^12 labels
// (the tiled form below).  Nets whose row sets are dependent, and m > 27, use
// the per-digit programme.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "dwt_grid.cuh"
#include "dwt_internal.cuh"

namespace dwt {

namespace {

constexpr int kLB = 13;          // tile: 2^13 labels (levels 0 .. 13 in shared memory)
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

// ---------------------------------------------------------------------------
// The tiled form, 12 <= m <= 27.  Tiles of 2^12 labels in groups of 16 (one
// thread each); a tile's work in a pass may be split over `parts` CTAs of 256
// threads, so that small nets still keep many SMs busy.
//
// Tree storage.  Levels are kept as 32-byte records.  A record of base level L
// holds the 16 nodes of level L under one node of level L + 4 (bytes 0..15),
// the 8, 4 and 2 nodes of levels L+1 .. L+3 between (bytes 16..23, 24..27,
// 28..29) and that node (byte 30).  Records of base level 0 (one per group)
// and 4 (one per block of 256 labels) are stored; the record of base level 8
// (one per tile) is its 16 block minima, stored as such, the rest derived
// where needed.  Every CTA builds levels 12 .. m (from the tile minima) in its
// shared memory.  Reading a representative downwards from level 11 touches at
// most one record of each base level.
//
// Backward sweep, one cooperative launch with two grid-wide waits per
// coordinate j = s-2 .. 0 (T_{s-1} and k_{s-1} have a closed form):
//   up    leaves T'[U] = T_{j+1}[Q_j(U)] of every group and their records;
//   wait
//   down  the coarse tree, A down to the leaves, T_j = min(T', A_0) and the
//         digit vector k_j(U) of the representative: top digit d-1, then the
//         lower digits smallest-first against the same tree (the reading of
//         the per-digit programme, which depends on U alone); T_j replaces
//         T_{j+1} in place (its gathers are done) and k_j goes to K[j][U];
//   wait  (T_j complete before coordinate j-1 gathers from it).
// Forward reading, one ordinary launch: every label H follows its own chain
//   U_0 = I_0(H),  k_j = K[j][U_j],  U_{j+1} = Q_j(U_j ^ k_j)
// (U_j ^ k_j are the coordinates of the label left after coordinate j), and
// multiplies its weight denominator by (1 + k_j)^2 -- no label waits for
// another and no tree is read again.
constexpr int kTL = 12;                    // labels per tile: 2^12
constexpr int kTT = 256;                   // threads per tile CTA
constexpr int kRecBytes = 8192 + 512 + 32; // one tile's records
constexpr int kFwdL = 8;                   // labels per thread of the forward reading

struct TileArgs {
    const Map4* Q;     // Q_j, j = 0 .. s-2
    uint8_t* T;        // N bytes: T_{j+1} before coordinate j's down pass, T_j after
    uint32_t* K;       // s x N: k_j(U)
    uint8_t* rec0;     // N / 16 records
    uint8_t* rec4;     // N / 256 records
    uint8_t* bmin;     // N / 256 block minima: 16 per tile, the base nodes of the tile's record
    unsigned* flags;   // [0] max T_0, [1] weight overflow, [2] a wait gave up, [3] arrivals
    long long N;
    int m, s;
};

// byte of node x (any index at that level) of level L + i in a record of base level L
__device__ __forceinline__ int rec_off(int i, uint32_t x) { return (32 - (32 >> i)) + (int)(x & (15u >> i)); }

// bytes 16..31 of a record from its 16 base nodes (bytes 0..15, four per word)
__device__ __forceinline__ uint4 rec_upper(uint4 lo) {
    const uint32_t a0 = __vminu4(__byte_perm(lo.x, lo.y, 0x6420), __byte_perm(lo.x, lo.y, 0x7531));
    const uint32_t a1 = __vminu4(__byte_perm(lo.z, lo.w, 0x6420), __byte_perm(lo.z, lo.w, 0x7531));
    const uint32_t b = __vminu4(__byte_perm(a0, a1, 0x6420), __byte_perm(a0, a1, 0x7531));
    const uint32_t c = __vminu4(__byte_perm(b, 0u, 0x4420), __byte_perm(b, 0u, 0x4431));
    const uint32_t e = min(c & 255u, (c >> 8) & 255u);
    return make_uint4(a0, a1, b, (c & 0xffffu) | (e << 16));
}

__device__ __forceinline__ unsigned byte_of(uint32_t w, int b) { return (w >> (8 * b)) & 255u; }

// up, for part `part` of `parts` of tile `tile`: the groups part * G ..
// part * G + G - 1 (G = 256 / parts), one per thread: leaves, group records,
// and per 16 groups the block record and the block minimum (st4: 256 bytes of
// shared staging, 16-byte aligned)
__device__ __forceinline__ void tile_up(const TileArgs& a, uint32_t tile, int part, int parts, const uint32_t (*q)[256],
                                        uint8_t* st4) {
    const int t = threadIdx.x;
    const int G = kTT / parts;
    const uint32_t g = (tile << 8) | (uint32_t)(part * G + t);   // group, over all labels
    if (t < G) {
        const uint32_t U0 = g << 4;
        uint32_t w[4];
        const uint32_t base = apply4(q, U0);   // Q(U0 ^ e) = Q(U0) ^ Q(e), e < 16
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint32_t x = 0;
#pragma unroll
            for (int b = 0; b < 4; ++b) x |= (uint32_t)a.T[base ^ q[0][4 * i + b]] << (8 * b);
            w[i] = x;
        }
        const uint4 lo = make_uint4(w[0], w[1], w[2], w[3]);
        const uint4 hi = rec_upper(lo);
        uint4* r0 = reinterpret_cast<uint4*>(a.rec0 + ((size_t)g << 5));
        r0[0] = lo;
        r0[1] = hi;
        st4[t] = (uint8_t)(hi.w >> 16);
    }
    __syncwarp();
    if (t < G && (t & 15) == 0) {
        const uint4 l4 = *reinterpret_cast<const uint4*>(st4 + t);
        const uint4 h4 = rec_upper(l4);
        uint4* r4 = reinterpret_cast<uint4*>(a.rec4 + ((size_t)(g >> 4) << 5));
        r4[0] = l4;
        r4[1] = h4;
        a.bmin[g >> 4] = (uint8_t)(h4.w >> 16);
    }
}

// one step of the top-down minima: the candidate of level i (sibling value
// sv, nu = i + 1) against the running minimum (av, ad) of the parent; ties go
// to the candidate, as in the per-digit sweep
__device__ __forceinline__ void a_step(unsigned sv, int i, unsigned& av, unsigned& ad) {
    const unsigned c = sat_add(sv, (unsigned)(i + 1));
    if (c <= av) {
        av = c;
        ad = (unsigned)(i + 1);
    }
}

// 16-bit mask of the bytes 0..15 of a record equal to v
__device__ __forceinline__ uint32_t eq_mask16(const uint4& r, uint32_t v) {
    const uint32_t v4 = v * 0x01010101u;
    auto z = [v4](uint32_t w) {
        const uint32_t x = w ^ v4;
        uint32_t y = ~(((x & 0x7f7f7f7fu) + 0x7f7f7f7fu) | x | 0x7f7f7f7fu);   // 0x80 in each zero byte
        y >>= 7;
        return (y | (y >> 7) | (y >> 14) | (y >> 21)) & 15u;
    };
    return z(r.x) | (z(r.y) << 4) | (z(r.z) << 8) | (z(r.w) << 12);
}

// the x in the 16-bit set M minimising x ^ u (fallback when M is empty)
__device__ __forceinline__ uint32_t closest16(uint32_t M, uint32_t u, uint32_t fallback) {
    uint32_t P = M;
    P = (u & 1u) ? (((P & 0x5555u) << 1) | ((P >> 1) & 0x5555u)) : P;
    P = (u & 2u) ? (((P & 0x3333u) << 2) | ((P >> 2) & 0x3333u)) : P;
    P = (u & 4u) ? (((P & 0x0f0fu) << 4) | ((P >> 4) & 0x0f0fu)) : P;
    P = (u & 8u) ? (((P & 0x00ffu) << 8) | ((P >> 8) & 0x00ffu)) : P;
    return P ? ((uint32_t)(__ffs(P) - 1) ^ u) : fallback;
}

// One step of a reading inside a record of base level L: from `node` of level
// l (L <= l <= L + 4) down to level L, keeping at each level the child on U's
// side when its subtree holds the target value, else the other child -- that
// is, the node x of level L under `node` with value tgt that minimises x ^ U.
__device__ __forceinline__ uint32_t record_step(const uint8_t* R, int L, int l, uint32_t node, uint32_t U,
                                                uint32_t tgt) {
    const int h = l - L;
    const uint32_t first = (node << h) & 15u;
    const uint32_t span = (h == 4 ? 0xffffu : ((1u << (1u << h)) - 1u)) << first;
    const uint4 r = *reinterpret_cast<const uint4*>(R);
    const uint32_t x = closest16(eq_mask16(r, tgt) & span, (U >> L) & 15u, first);
    return ((node >> (4 - h)) << 4) | x;   // record index (node of level L + 4) and x
}

// The representative k_j(U) of a label with d > 0: the top digit d-1 selects
// the sibling of U's node of level d-1, then the lower digits read the tree
// downwards, smallest-first, keeping subtrees with value tau - d (levels above
// 12 from the coarse tree in shared memory, below through one tile, one block
// and one group record: this tile's from shared memory, others' from global
// memory).  k_j = U ^ (the leaf reached).
__device__ __forceinline__ uint32_t representative(const TileArgs& a, uint32_t U, int d, int tau, uint32_t tile,
                                                   const uint8_t* cl, long long nLB, const uint8_t* R0,
                                                   const uint8_t* R4, const uint8_t* R8) {
    const uint32_t tgt = (uint32_t)(tau - d) & 255u;
    int l = d - 1;
    uint32_t node = (U >> l) ^ 1u;
    for (; l > kTL; --l) {
        uint32_t c = (node << 1) | ((U >> (l - 1)) & 1u);
        if ((uint32_t)cl[loff(nLB, l - 1 - kTL) + c] != tgt) c ^= 1u;
        node = c;
    }
    if (l >= 8) {
        const uint32_t tl = node >> (kTL - l);
        const uint8_t* R = tl == tile ? R8 : a.bmin + ((size_t)tl << 4);
        node = record_step(R, 8, l, node, U, tgt);
        l = 8;
    }
    if (l >= 4) {
        const uint32_t bl = node >> (8 - l);
        const uint8_t* R = (bl >> 4) == tile ? R4 + ((bl & 15u) << 5) : a.rec4 + ((size_t)bl << 5);
        node = record_step(R, 4, l, node, U, tgt);
        l = 4;
    }
    {
        const uint32_t gr = node >> (4 - l);
        const uint8_t* R = (gr >> 8) == tile ? R0 + ((gr & 255u) << 5) : a.rec0 + ((size_t)gr << 5);
        node = record_step(R, 0, l, node, U, tgt);
    }
    return U ^ node;
}

// down, for part `part` of `parts` (a power of two <= 16) of tile `tile`: the
// groups g = part * G .. part * G + G - 1, G = 256 / parts, each by one thread
// (A down the tile to its 16 leaves, T_j), then the readings of their 16 G
// leaves by all kTT threads, 16 / parts each.  cl = levels 12 .. m (level
// 12 + i at loff(nLB, i)); sr = shared staging of kRecBytes bytes of records
// and 2 x 4096 bytes of T_j, d per leaf.
__device__ __forceinline__ void tile_down(const TileArgs& a, uint32_t tile, int part, int parts, int j,
                                          const uint8_t* cl, long long nLB, uint8_t* sr, unsigned& mx) {
    const int t = threadIdx.x;
    const int m = a.m;
    const long long N = a.N;
    {
        const uint4* s0 = reinterpret_cast<const uint4*>(a.rec0 + ((size_t)tile << 13));
        uint4* d = reinterpret_cast<uint4*>(sr);
        d[t] = s0[t];
        d[t + kTT] = s0[t + kTT];
        if (t < 32) {
            d[512 + t] = reinterpret_cast<const uint4*>(a.rec4 + ((size_t)tile << 9))[t];
        } else if (t == 32) {
            const uint4 l8 = *reinterpret_cast<const uint4*>(a.bmin + ((size_t)tile << 4));
            d[544] = l8;
            d[545] = rec_upper(l8);
        }
    }
    __syncthreads();
    const uint8_t* R0 = sr;          // 256 group records
    const uint8_t* R4 = sr + 8192;   // 16 block records
    const uint8_t* R8 = sr + 8704;   // the tile record
    uint8_t* stau = sr + kRecBytes;  // T_j of the part's leaves
    uint8_t* sd = stau + 4096;       // d of the part's leaves
    const int G = kTT / parts;
    if (t < G) {
        const int g = part * G + t;   // group within the tile
        // A at the tile root, down the coarse tree
        unsigned av = kInfB, ad = 0;
        for (int i = m - 1; i >= kTL; --i) a_step(cl[loff(nLB, i - kTL) + ((tile >> (i - kTL)) ^ 1u)], i, av, ad);
        // levels 11 .. 4: the group's ancestors, node g >> (i - 4) of level i in the tile
#pragma unroll
        for (int i = 11; i >= 8; --i) a_step(R8[rec_off(i - 8, ((uint32_t)g >> (i - 4)) ^ 1u)], i, av, ad);
#pragma unroll
        for (int i = 7; i >= 4; --i)
            a_step(R4[((g >> 4) << 5) + rec_off(i - 4, ((uint32_t)g >> (i - 4)) ^ 1u)], i, av, ad);
        // levels 3 .. 0 inside the group record
        const uint4 glo = *reinterpret_cast<const uint4*>(R0 + (g << 5));
        const uint4 ghi = *reinterpret_cast<const uint4*>(R0 + (g << 5) + 16);
        const uint32_t gw[8] = {glo.x, glo.y, glo.z, glo.w, ghi.x, ghi.y, ghi.z, ghi.w};
        unsigned v3[2], d3[2], v2[4], d2[4], v1[8], d1[8];
#pragma unroll
        for (int x = 0; x < 2; ++x) {
            const int b = 28 + (x ^ 1);
            v3[x] = av;
            d3[x] = ad;
            a_step(byte_of(gw[b >> 2], b & 3), 3, v3[x], d3[x]);
        }
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int b = 24 + (x ^ 1);
            v2[x] = v3[x >> 1];
            d2[x] = d3[x >> 1];
            a_step(byte_of(gw[b >> 2], b & 3), 2, v2[x], d2[x]);
        }
#pragma unroll
        for (int x = 0; x < 8; ++x) {
            const int b = 16 + (x ^ 1);
            v1[x] = v2[x >> 1];
            d1[x] = d2[x >> 1];
            a_step(byte_of(gw[b >> 2], b & 3), 1, v1[x], d1[x]);
        }
        uint32_t tw[4] = {0u, 0u, 0u, 0u}, dw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            unsigned v0 = v1[e >> 1], d0 = d1[e >> 1];
            a_step(byte_of(gw[(e ^ 1) >> 2], (e ^ 1) & 3), 0, v0, d0);
            const unsigned leaf = byte_of(gw[e >> 2], e & 3);
            const bool keep = leaf <= v0;
            const unsigned tau = keep ? leaf : v0;
            tw[e >> 2] |= tau << (8 * (e & 3));
            dw[e >> 2] |= (keep ? 0u : d0) << (8 * (e & 3));
            if (j == 0) mx = max(mx, tau);
        }
        const uint4 tv = make_uint4(tw[0], tw[1], tw[2], tw[3]);
        *reinterpret_cast<uint4*>(a.T + (((size_t)tile << kTL) | ((size_t)g << 4))) = tv;
        *reinterpret_cast<uint4*>(stau + (t << 4)) = tv;
        *reinterpret_cast<uint4*>(sd + (t << 4)) = make_uint4(dw[0], dw[1], dw[2], dw[3]);
    }
    __syncthreads();
    // the readings: leaf x = t + kTT i of the part (consecutive threads, consecutive leaves)
    const uint32_t L0 = (tile << kTL) | ((uint32_t)part << (kTL - __ffs(parts) + 1));
    uint32_t* Kj = a.K + (size_t)j * N;
    for (int x = t; x < 16 * G; x += kTT) {
        const int d = sd[x];
        Kj[L0 + x] = d ? representative(a, L0 + (uint32_t)x, d, stau[x], tile, cl, nLB, R0, R4, R8) : 0u;
    }
}

// The backward sweep (cooperative launch, every CTA resident).  The up pass
// runs one CTA per tile, the down pass one CTA per part of a tile (`parts`
// per tile).  Dynamic shared memory: map 4096 | records kRecBytes | T_j, d
// 2 x 4096 | st4 256 | ok 16 | coarse levels 2 nLB.
__global__ void __launch_bounds__(kTT) k_tiles_bwd(TileArgs a, int parts) {
    extern __shared__ __align__(16) unsigned char sm[];
    uint32_t (*q)[256] = reinterpret_cast<uint32_t (*)[256]>(sm);
    uint8_t* sr = sm + 4096;
    uint8_t* st4 = sr + kRecBytes + 8192;
    int* ok = reinterpret_cast<int*>(st4 + 256);
    uint8_t* cl = st4 + 256 + 16;
    const long long nLB = a.N >> kTL;
    const int top = a.m - kTL;
    unsigned target = 0, mx = 0;
    for (int j = a.s - 1; j >= 0; --j) {
        if (j == a.s - 1) {
            // T_s is 0 at label 0 only, so T_{s-1}(U) = (highest set bit of U) + 1
            // with the reading running down to label 0: k_{s-1}(U) = U
            for (long long tl = blockIdx.x; tl < nLB; tl += gridDim.x) {
                const uint32_t U0 = ((uint32_t)tl << kTL) | ((uint32_t)threadIdx.x << 4);
                uint32_t tw[4];
#pragma unroll
                for (int w = 0; w < 4; ++w) {
                    uint32_t x = 0;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const uint32_t U = U0 + (uint32_t)(4 * w + b);
                        x |= (U ? (uint32_t)(32 - __clz(U)) : 0u) << (8 * b);
                    }
                    tw[w] = x;
                    if (j == 0) mx = max(mx, (unsigned)(32 - __clz(U0 + 4 * w + 3)));
                }
                *reinterpret_cast<uint4*>(a.T + U0) = make_uint4(tw[0], tw[1], tw[2], tw[3]);
                uint4* kd = reinterpret_cast<uint4*>(a.K + (size_t)j * a.N + U0);
#pragma unroll
                for (int w = 0; w < 4; ++w) kd[w] = make_uint4(U0 + 4 * w, U0 + 4 * w + 1, U0 + 4 * w + 2, U0 + 4 * w + 3);
            }
            if (j > 0 && !grid_wait(a.flags, target, ok)) return;
            continue;
        }
        load_map(q, a.Q + j);
        __syncthreads();
        for (long long u = blockIdx.x; u < nLB * parts; u += gridDim.x) {
            tile_up(a, (uint32_t)(u / parts), (int)(u % parts), parts, q, st4);
            __syncthreads();
        }
        if (!grid_wait(a.flags, target, ok)) return;
        // levels 12 .. m of the tree, in every CTA
        for (long long v = threadIdx.x; v < nLB; v += kTT) {
            const uint4 b = *reinterpret_cast<const uint4*>(a.bmin + (v << 4));
            const uint32_t x = __vminu4(__vminu4(b.x, b.y), __vminu4(b.z, b.w));
            cl[v] = (uint8_t)min(min(x & 255u, (x >> 8) & 255u), min((x >> 16) & 255u, x >> 24));
        }
        __syncthreads();
        for (int i = 1; i <= top; ++i) {
            const long long n = nLB >> i;
            const uint8_t* src = cl + loff(nLB, i - 1);
            uint8_t* dst = cl + loff(nLB, i);
            for (long long v = threadIdx.x; v < n; v += kTT) dst[v] = min(src[2 * v], src[2 * v + 1]);
            __syncthreads();
        }
        for (long long u = blockIdx.x; u < nLB * parts; u += gridDim.x) {
            tile_down(a, (uint32_t)(u / parts), (int)(u % parts), parts, j, cl, nLB, sr, mx);
            __syncthreads();
        }
        if (j > 0 && !grid_wait(a.flags, target, ok)) return;
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(a.flags, mx);
}

__device__ __forceinline__ uint32_t apply4_ldg(const Map4* M, uint32_t x) {
    return __ldg(&M->t[0][x & 255]) ^ __ldg(&M->t[1][(x >> 8) & 255]) ^ __ldg(&M->t[2][(x >> 16) & 255]) ^
           __ldg(&M->t[3][x >> 24]);
}

// The forward reading: labels H = h0 + l * stride, l < kFwdL, of this thread.
__global__ void __launch_bounds__(256) k_tiles_fwd(const uint32_t* __restrict__ K, const Map4* __restrict__ I0,
                                                   const Map4* __restrict__ Q, unsigned* flags, float* W,
                                                   uint8_t* cls, long long N, int s) {
    if (flags[0] >= kInfB || flags[2]) return;   // the backward sweep did not finish: nothing to read
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long h0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    uint32_t U[kFwdL];
    unsigned long long pd[kFwdL];
    uint32_t c[kFwdL];   // last coordinate with k_j != 0 | count << 8
#pragma unroll
    for (int l = 0; l < kFwdL; ++l) {
        const long long H = h0 + l * stride;
        U[l] = H < N ? apply4_ldg(I0, (uint32_t)H) : 0u;
        pd[l] = 1ull;
        c[l] = 0u;
    }
    bool over = false;
    for (int j = 0; j < s; ++j) {
        const uint32_t* Kj = K + (size_t)j * N;
        const Map4* Qj = Q + j;
#pragma unroll
        for (int l = 0; l < kFwdL; ++l) {
            if (h0 + l * stride >= N) continue;
            const uint32_t k = __ldg(Kj + U[l]);
            if (k) {
                const unsigned long long qq = (unsigned long long)k + 1ull, q2 = qq * qq;
                if (__umul64hi(pd[l], q2) != 0ull) over = true;
                pd[l] *= q2;
                c[l] = (uint32_t)(j + 1) | (((c[l] >> 8) + 1u) << 8);
            }
            if (j + 1 < s) U[l] = apply4_ldg(Qj, U[l] ^ k);
        }
    }
#pragma unroll
    for (int l = 0; l < kFwdL; ++l) {
        const long long H = h0 + l * stride;
        if (H >= N) continue;
        W[H] = __fdiv_rn(1.0f, __ull2float_rn(pd[l]));
        cls[2 * H] = (uint8_t)(c[l] & 255u);
        cls[2 * H + 1] = (uint8_t)(c[l] >> 8);
    }
    if (over) atomicExch(flags + 1, 1u);
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

// Resident CTAs of the backward sweep on this GPU (0 if unknown).
static long long tiles_resident(size_t smem) {
    int dev = 0, sms = 0, occ = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_tiles_bwd, kTT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return (long long)occ * sms;
}

// The tiled form for 12 <= m <= 27 (one cooperative launch for the backward
// sweep, one launch for the forward reading, one synchronisation).
int tiles_build(dwt_plan_s* Pl, const Map4& I0, const std::vector<Map4>& Qmap, cudaStream_t st) {
    const long long N = Pl->N;
    const int m = Pl->m, s = Pl->s;
    const long long tiles = N >> kTL;
    // one scratch block: flags (16 B, padded), the maps I_0, Q_0 .. Q_{s-2},
    // then T, the records, the block minima and K (256-byte aligned pieces)
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_maps = 256, o_T = al(o_maps + sizeof(Map4) * s), o_rec0 = al(o_T + (size_t)N),
                 o_rec4 = al(o_rec0 + (size_t)N * 2), o_bmin = al(o_rec4 + (size_t)N / 8),
                 o_K = al(o_bmin + (size_t)N / 256), total = al(o_K + (size_t)s * N * 4);
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
    Map4* dmaps = reinterpret_cast<Map4*>(ws + o_maps);
    uint8_t* T = ws + o_T;
    uint8_t* rec0 = ws + o_rec0;
    uint8_t* rec4 = ws + o_rec4;
    uint8_t* bmin = ws + o_bmin;
    uint32_t* K = reinterpret_cast<uint32_t*>(ws + o_K);
    // flags zeroed and the maps in one upload, from page-locked staging when
    // there is some (the stream is synchronised below, before it is reused)
    const size_t nb = o_maps + sizeof(Map4) * s;
    std::vector<unsigned char> hv;
    unsigned char* hb = host_staging(nb);
    if (!hb) {
        hv.resize(nb);
        hb = hv.data();
    }
    memset(hb, 0, o_maps);
    memcpy(hb + o_maps, &I0, sizeof(Map4));
    for (int j = 0; j + 1 < s; ++j) memcpy(hb + o_maps + sizeof(Map4) * (1 + j), &Qmap[j], sizeof(Map4));
    if ((rc = ck(cudaMemcpyAsync(ws, hb, nb, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync"))) return rc;
    const size_t smem = 4096 + kRecBytes + 8192 + 256 + 16 + (size_t)((2 * tiles + 15) & ~15ll);
    rc = smem_limit_max(k_tiles_bwd);
    if (rc) { cleanup(); return rc; }
    // every resident CTA busy in the down pass: parts per tile (a power of two
    // <= 16); the grid is capped by DWT_TILE_GRID if set (a tuning and testing
    // knob: the tables do not depend on the grid or the parts)
    const long long resident = tiles_resident(smem);
    int parts = 1;
    while (parts < 16 && tiles * parts * 2 <= resident) parts *= 2;
    long long g = std::min(tiles * parts, resident);
    {
        const char* e = getenv("DWT_TILE_GRID");
        const long long cap = e ? atoll(e) : 0;
        if (cap > 0) g = std::min(g, cap);
    }
    if (g > 0) {
        // as few CTAs as give the same number of rounds over the parts
        const long long rounds = (tiles * parts + g - 1) / g;
        g = (tiles * parts + rounds - 1) / rounds;
    }
    const int grid = (int)g;
    if (grid < 1) {
        cleanup();
        set_error("no resident grid for the tiled coset-table sweep (%zu bytes of shared memory)", smem);
        return DWT_ECUDA;
    }
    TileArgs A;
    A.Q = dmaps + 1;
    A.T = T;
    A.K = K;
    A.rec0 = rec0;
    A.rec4 = rec4;
    A.bmin = bmin;
    A.flags = flags;
    A.N = N;
    A.m = m;
    A.s = s;
    {
        LaunchScope ls("tree_sweep", st);
        void* args[] = {&A, &parts};
        if ((rc = ck(cudaLaunchCooperativeKernel((const void*)k_tiles_bwd, dim3((unsigned)grid), dim3(kTT), args, smem,
                                                 st),
                     "cooperative launch")))
            return rc;
    }
    {
        const long long per_cta = 256ll * kFwdL;
        const unsigned fg = (unsigned)((N + per_cta - 1) / per_cta);
        LaunchScope ls("tree_read", st);
        k_tiles_fwd<<<fg, 256, 0, st>>>(K, dmaps, dmaps + 1, flags, Pl->d_W, Pl->d_cls, N, s);
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
    const int m = Pl->m, s = Pl->s;
    *used = false;
    if (Pl->p != 2 || m > 27 || m < 1) return DWT_OK;
    const std::vector<uint32_t>& R = Pl->R_host;
    // maps: I_j (labels -> U_j) and Q_j (U_j -> U_{j+1})
    std::vector<Map4> Imap(s), Qmap(s);
    std::vector<uint32_t> inv(m);
    for (int j = 0; j < s; ++j) {
        if (!gf2_inverse(&R[(size_t)j * m], m, inv.data())) return DWT_OK;
        make_map(inv.data(), m, Imap[j]);
    }
    for (int j = 0; j + 1 < s; ++j) {
        std::vector<uint32_t> qc(m);
        for (int i = 0; i < m; ++i) qc[i] = host_apply(Imap[j + 1], R[(size_t)j * m + i]);
        make_map(qc.data(), m, Qmap[j]);
    }
    *used = true;
    if (m < kTL) return tree_one(Pl, Imap, Qmap, st);
    return tiles_build(Pl, Imap[0], Qmap, st);
}

}  // namespace dwt
