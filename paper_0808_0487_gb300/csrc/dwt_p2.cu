// dwt_p2.cu -- register-tile kernels for p = 2 (FP32 and int32), the hot path
// of Algorithms 1 and 2 on large nets.
//
// For p = 2 the transform is the Walsh-Hadamard transform: every stage is the
// butterfly (a, b) -> (a + b, a - b) over one index bit, and the stages over
// different bits commute (Sec. 2.2).  A pass covers a tile of 2^LT elements;
// every thread keeps 64 of them in registers (32 packed pairs), so 6 index
// bits are "in thread" at a time and their stages run without data movement,
// two butterflies per packed f32x2 instruction.  Between register layouts the
// tile goes once through shared memory.  A padded layout (a few words inserted
// every 2^8, or 2^(p1+6), elements) keeps every exchange free of bank
// conflicts, and every register's shared-memory address is a per-thread base
// plus a compile-time offset.
//
//  k2_lo<L>: a contiguous tile of 2^L elements (L = 12..14), the low L digits.
//    layout A (load / first stages): float4 at 4(t + NT q): in-thread bits
//      {0,1} and {L-4..L-1}; layout B: bits {2..7}; layout C: bits {0,1,8..11}.
//  k2_hi<LT, B>: B digits d0..d0+B-1 above the low pass; the tile holds
//    2^B rows (distance S = 2^d0 apart) of Wc = 2^(LT-B) consecutive columns.
//    layout A: float4 at 4(t + NT q): bits {0,1} (columns) and {LT-4..LT-1};
//    layout P: bits [p1, p1+6) with p1 = min(LT-B, LT-6).
//    The fused variant runs the forward stages, the scale p^-m, the weight,
//    the per-class variance partials and the inverse stages of the same
//    digits in one tile: the top pass of dwt_interpolate.
#include <algorithm>
#include <type_traits>

#include "dwt_p2_tile.cuh"

namespace dwt {

// One low-pass job: nf functions, tiles of 2^L elements.
template <typename T> struct LoJob {
    const T* in;
    T* out;
    long long ld_in, ld_out;
    int nf;
    float scale;
    int do_scale;
    int stream_out;   // store with evict-first (final results)
};

// Tiles [0, tiles0) belong to job 0, the rest to job 1: two independent low
// passes share one launch (e.g. the inverse of one function and the forward of
// the next), which keeps the memory system busy while either one computes.
// the low pass of one tile of 2^L elements, src -> dst
template <typename T, int L>
__device__ __forceinline__ void lo_body(const T* src, T* dst, float scale, int do_scale, bool stream_out) {
    using V = typename P2<T>::t;
    constexpr int NT = 1 << (L - 6);
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int t = threadIdx.x;
    V v[32];
#pragma unroll
    for (int q = 0; q < 16; ++q) ld16_cs(src + 4 * (t + NT * q), v + 2 * q);
    bfly_range<0, 6>(v);
    lo_tile_compute<T, L>(sm, v, t);
    if (do_scale) {
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = pmul(v[k], scale);
    }
    lo_tile_store<T, L>(dst, v, t, stream_out);
}

template <typename T, int L>
__global__ void __launch_bounds__(1 << (L - 6), (L == 14 ? 3 : 4))
    k2_lo(LoJob<T> j0, LoJob<T> j1, unsigned tiles0) {
    static_assert(L >= 12 && L <= 14, "low-pass tile 2^12 .. 2^14");
    const bool second = blockIdx.x >= tiles0;
    if ((int)blockIdx.y >= (second ? j1.nf : j0.nf)) return;
    const long long tile = second ? blockIdx.x - tiles0 : blockIdx.x;
    const T* src = (second ? j1.in : j0.in) + blockIdx.y * (second ? j1.ld_in : j0.ld_in) + (tile << L);
    T* dst = (second ? j1.out : j0.out) + blockIdx.y * (second ? j1.ld_out : j0.ld_out) + (tile << L);
    lo_body<T, L>(src, dst, second ? j1.scale : j0.scale, second ? j1.do_scale : j0.do_scale,
                  (second ? j1.stream_out : j0.stream_out) != 0);
}

// Whole transforms of 2^L points (one tile per function) of several plans in
// one launch: job i owns the blocks [first, first + nf), one function each,
// each run by the tile body of k2_lo.
template <typename T> struct LoGroup {
    LoJob<T> j;
    long long first;
};

template <typename T, int L>
__global__ void __launch_bounds__(1 << (L - 6), (L == 14 ? 3 : 4))
    k2_lo_grouped(const LoGroup<T>* __restrict__ jobs, int njobs) {
    const long long b = blockIdx.x;
    int lo = 0, hi = njobs - 1;   // the last job starting at or before b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].first <= b) lo = mid;
        else hi = mid - 1;
    }
    const LoJob<T>& j = jobs[lo].j;
    const long long fn = b - jobs[lo].first;
    lo_body<T, L>(j.in + fn * j.ld_in, j.out + fn * j.ld_out, j.scale, j.do_scale, j.stream_out != 0);
}

// ---------------------------------------------------------------------------
// high pass: 2^B rows (stride S) x Wc = 2^(LT-B) columns
struct HiArgs {
    const void* in;
    void* out;
    long long ld_in, ld_out;
    long long S;         // row distance 2^d0
    long long nlo;       // S / Wc column chunks
    float scale;
    int do_scale;
    // fused top pass
    const float* W;      // tile-major weights, NULL = 1
    const uint8_t* cls;  // tile-major classes
    void* coef;          // optional output of the weighted coefficients
    double* part;        // [fn][class][tile]
    long long ntile;
    int nb;
};

template <typename T, int LT, int B, bool FUSED, bool HAS_COEF>
__global__ void __launch_bounds__(1 << (LT - 6), FUSED ? 4 : 1) k2_hi(HiArgs a) {
    static_assert(B >= 4 && B <= 10 && LT - B >= 2, "high-pass shape");
    using G = HiGeom<LT, B>;
    using V = typename P2<T>::t;
    constexpr int NT = G::NT, P1 = G::P1;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int t = threadIdx.x;
    const long long fn = blockIdx.y, tile = blockIdx.x;
    const long long base = ((tile % a.nlo) << G::CB) + (tile / a.nlo) * (a.S << B);
    const T* src = reinterpret_cast<const T*>(a.in) + fn * a.ld_in + base;
    T* dst = reinterpret_cast<T*>(a.out) + fn * a.ld_out + base;
    V v[32];
    // layout A loads
#pragma unroll
    for (int q = 0; q < 16; ++q) ld16(src + G::goff(4 * (t + NT * q), a.S), v + 2 * q);
    if constexpr (FUSED) {
        // this tile's weights (4 B per element) and classes (2 B) are contiguous
        // in the tile-major tables: start moving them from HBM into L2 now, to be
        // read after the forward stages
        if (t == 0) {
            if (a.W) prefetch_l2(a.W + ((long long)tile << LT), 4u << LT);
            prefetch_l2(a.cls + ((long long)tile << (LT + 1)), 2u << LT);
        }
    }
    bfly_range<2, 6>(v);   // e bits LT-4..LT-1 = row bits B-4..B-1
    // layout A in shared memory: pad(4(t + NT q)) = 4t + q 4NT + PADC (q >> QSH)
    T* pa = sm + 4 * t;
    if constexpr (B > 4) {
#pragma unroll
        for (int q = 0; q < 16; ++q) st16(pa + q * 4 * NT + G::PADC * (q >> G::QSH), v + 2 * q);
        __syncthreads();
    }
    // layout P: element ep | (j << P1) at pad(ep) + (j << P1)
    const int ep = (t & ((1 << P1) - 1)) | ((t >> P1) << (P1 + 6));
    T* pp = sm + ep + G::PADC * (ep >> G::PADSH);
    if constexpr (B > 4) {
#pragma unroll
        for (int j = 0; j < 64; ++j) comp(v[j >> 1], j & 1) = pp[j << P1];
        bfly_range<G::RLO, G::RHI>(v);
    }
    if constexpr (!FUSED) {
        if (a.do_scale) {
#pragma unroll
            for (int k = 0; k < 32; ++k) v[k] = pmul(v[k], a.scale);
        }
        if constexpr (B > 4) {
#pragma unroll
            for (int j = 0; j < 64; ++j) dst[G::goff(ep | (j << P1), a.S)] = comp(v[j >> 1], j & 1);
        } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) st16(dst + G::goff(4 * (t + NT * q), a.S), v + 2 * q);
        }
    } else {
        // The class bins alias the exchange buffer: wait until every thread has
        // read layout P, then zero them.
        float* bins = reinterpret_cast<float*>(smraw);
        const int nb2 = 2 * a.nb;
        const int lane = t & 31, w = t >> 5;
        if constexpr (B > 4) __syncthreads();
        {
            float4* b4 = reinterpret_cast<float4*>(bins);
            for (int i = t; i < (NT >> 5) * nb2 * 8; i += NT) b4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        float* bt = bins + w * nb2 * 32 + lane;   // max-support classes of this lane
        float* bs = bt + a.nb * 32;                 // support-size classes of this lane
        float* coef = HAS_COEF ? reinterpret_cast<float*>(a.coef) + fn * a.ld_out + base : nullptr;
        const bool has0 = base == 0 && t == 0;   // coset label H = 0 is register 0 of thread 0
        // tile-major tables: register group g (4 elements) of thread t at g NT + t;
        // the weights carry the factor 2^-m already (exact: a power of 2).  Groups
        // are read two at a time, one pair ahead of the pair being binned.
        const float4* wg = a.W ? reinterpret_cast<const float4*>(a.W) + ((long long)tile << (LT - 2)) + t : nullptr;
        const uint2* cg = reinterpret_cast<const uint2*>(a.cls) + ((long long)tile << (LT - 2)) + t;
        constexpr int CH = 2;
        float4 wq[2][CH];
        uint2 cq[2][CH];
        auto fetch = [&](int c, int slot) {
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int g = c * CH + i;
                wq[slot][i] = wg ? __ldcs(wg + g * NT) : make_float4(a.scale, a.scale, a.scale, a.scale);
                cq[slot][i] = __ldcs(cg + g * NT);
            }
        };
        fetch(0, 0);
#pragma unroll
        for (int c = 0; c < 16 / CH; ++c) {
            if (c + 1 < 16 / CH) fetch(c + 1, (c + 1) & 1);
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int g = c * CH + i;
                const float4 x4 = wq[c & 1][i];
                V& v01 = v[2 * g];
                V& v23 = v[2 * g + 1];
                v01 = __fmul2_rn(v01, make_float2(x4.x, x4.y));
                v23 = __fmul2_rn(v23, make_float2(x4.z, x4.w));
                const float2 q01 = __fmul2_rn(v01, v01), q23 = __fmul2_rn(v23, v23);
                if constexpr (HAS_COEF) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int j = 4 * g + u;
                        coef[G::goff(G::fused_e(t, j), a.S)] = comp(v[j >> 1], j & 1);
                    }
                }
                const float q[4] = {(g == 0 && has0) ? 0.f : q01.x, q01.y, q23.x, q23.y};
                bin_group(bt, bs, cq[c & 1][i], q);
            }
            asm volatile("" ::: "memory");   // keep the next pair's loads behind this pair's bins
        }
        __syncthreads();
        // per-tile class sums, fixed order: lane l of warp w sums whole classes
        // b = l, l+32, ... of its warp's [class][lane] block, reading the 32 lane
        // columns in the rotated order (k + l) & 31 (conflict-free) into a pairwise
        // tree; the NW warp sums are then added in warp order and stored in FP64
        // class-major: part[fn][class][tile].
        {
            constexpr int NW = NT >> 5;
            float* red = bins + NW * nb2 * 32;   // [NW][nb2]
            const float* wb = bins + w * nb2 * 32;
            for (int b = lane; b < nb2; b += 32) {
                float r[32];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float4 x = *reinterpret_cast<const float4*>(wb + b * 32 + 4 * ((i + lane) & 7));
                    r[4 * i] = x.x; r[4 * i + 1] = x.y; r[4 * i + 2] = x.z; r[4 * i + 3] = x.w;
                }
#pragma unroll
                for (int h = 16; h > 0; h >>= 1)
#pragma unroll
                    for (int k = 0; k < h; ++k) r[k] += r[k + h];
                red[w * nb2 + b] = r[0];
            }
            __syncthreads();
            for (int b = t; b < nb2; b += NT) {
                float x = red[b];
#pragma unroll
                for (int ww = 1; ww < NW; ++ww) x += red[ww * nb2 + b];
                a.part[(fn * nb2 + b) * a.ntile + tile] = (double)x;
            }
        }
        // inverse stages of the same digits: layout P, then back to layout A
        if constexpr (B > 4) {
            bfly_range<G::RLO, G::RHI>(v);
            __syncthreads();   // bins read out before the exchange reuses the buffer
#pragma unroll
            for (int j = 0; j < 64; ++j) pp[j << P1] = comp(v[j >> 1], j & 1);
            __syncthreads();
#pragma unroll
            for (int q = 0; q < 16; ++q) ld16(pa + q * 4 * NT + G::PADC * (q >> G::QSH), v + 2 * q);
        }
        bfly_range<2, 6>(v);
#pragma unroll
        for (int q = 0; q < 16; ++q) st16(dst + G::goff(4 * (t + NT * q), a.S), v + 2 * q);
    }
}

// tile-major copies of the weight and class tables for the fused pass: register
// group g (4 elements) of thread t of a tile at (tile 2^LT) + 4 (g NT + t)
template <int LT, int B>
__global__ void __launch_bounds__(1 << (LT - 6)) k2_tile_tables(const float* __restrict__ W,
                                                                const uint8_t* __restrict__ cls, float* Wt,
                                                                uint8_t* clst, long long S, long long nlo,
                                                                float scale) {
    using G = HiGeom<LT, B>;
    constexpr int NT = G::NT;
    const int t = threadIdx.x;
    const long long tile = blockIdx.x;
    const long long base = ((tile % nlo) << G::CB) + (tile / nlo) * (S << B);
    for (int j = 0; j < 64; ++j) {
        const long long H = base + G::goff(G::fused_e(t, j), S);
        const long long o = (tile << LT) + 4 * ((j >> 2) * NT + t) + (j & 3);
        Wt[o] = W[H] * scale;   // scale = 2^-m: exact
        clst[2 * o] = cls[2 * H];
        clst[2 * o + 1] = cls[2 * H + 1];
    }
}

// ---------------------------------------------------------------------------
// host side
template <typename F>
static int attr_smem(F* k, size_t bytes) {
    (void)bytes;
    return smem_limit_max(k);
}

// digit split of the fast path: one low pass of L = m digits for 12 <= m <= 14;
// otherwise a low pass of L = min(14, m - 4) digits and a high pass of B = m - L
// digits, 4 <= B <= 10 (16 <= m <= 24)
static int p2_low_digits(int m) { return m <= 14 ? m : std::min(14, m - 4); }

// the low-pass digits of a plan's transform: a measured choice (DWT_PLAN_TUNE)
// when one lies in the kernels' range 12 <= L <= 14, 4 <= m - L <= 10
static int p2_lo_digits_of(const dwt_plan_s* Pl) {
    const int m = Pl->m, L = Pl->tuned_lo;
    if (m >= 16 && L >= 12 && L <= 14 && m - L >= 4 && m - L <= 10) return L;
    return p2_low_digits(m);
}
bool p2_fast_ok(int m) { return (m >= 12 && m <= 14) || (m >= 16 && m <= 24); }

template <typename T>
static int launch_lo2(int L, const LoJob<T>& a, const LoJob<T>* b, long long N, const char* fam, cudaStream_t st) {
    const unsigned tiles = (unsigned)(N >> L);
    const size_t smem = (((size_t)1 << L) + ((size_t)1 << (L - 4))) * sizeof(T);
    const int nf = b ? std::max(a.nf, b->nf) : a.nf;
    dim3 grid(b ? 2 * tiles : tiles, (unsigned)nf);
    const LoJob<T> jb = b ? *b : a;
    int rc;
#define DWT_LO(LL)                                                                         \
    case LL: {                                                                             \
        auto k = k2_lo<T, LL>;                                                             \
        if ((rc = attr_smem(k, smem))) return rc;                                          \
        LaunchScope ls(fam, st);                                                           \
        k<<<grid, 1 << (LL - 6), smem, st>>>(a, jb, tiles);                                \
        break;                                                                             \
    }
    switch (L) {
        DWT_LO(12)
        DWT_LO(13)
        DWT_LO(14)
        default: set_error("low-pass tile"); return DWT_EUNSUPPORTED;
    }
#undef DWT_LO
    DWT_CK_LAUNCH("k2_lo");
    return DWT_OK;
}

template <typename T>
static int lo_grouped_t(int L, const std::vector<GroupJob>& jobs, int sgn, cudaStream_t st) {
    const bool scale = sgn < 0 && std::is_same<T, float>::value;
    std::vector<LoGroup<T>> h;
    long long blocks = 0;
    for (const GroupJob& g : jobs) {
        const long long N = g.plan->N;
        LoGroup<T> x;
        x.j = LoJob<T>{(const T*)g.in, (T*)g.out, g.ld_in, g.ld_out, g.batch, (float)(1.0 / (double)N), scale ? 1 : 0, 0};
        x.first = blocks;
        blocks += g.batch;
        h.push_back(x);
    }
    if (blocks > 0x7fffffffll) {
        set_error("grouped low pass: %lld blocks exceed one launch", blocks);
        return DWT_EINVAL;
    }
    LoGroup<T>* d = nullptr;
    if (dmalloc((void**)&d, sizeof(LoGroup<T>) * h.size(), st)) return DWT_ENOMEM;
    DWT_CK(cudaMemcpyAsync(d, h.data(), sizeof(LoGroup<T>) * h.size(), cudaMemcpyHostToDevice, st));
    const size_t smem = (((size_t)1 << L) + ((size_t)1 << (L - 4))) * sizeof(T);
    int rc = DWT_OK;
#define DWT_LOG(LL)                                                                       \
    case LL: {                                                                            \
        auto k = k2_lo_grouped<T, LL>;                                                    \
        if ((rc = attr_smem(k, smem))) break;                                             \
        LaunchScope ls("grouped_lo", st);                                                 \
        k<<<(unsigned)blocks, 1 << (LL - 6), smem, st>>>(d, (int)h.size());               \
        break;                                                                            \
    }
    switch (L) {
        DWT_LOG(12)
        DWT_LOG(13)
        DWT_LOG(14)
        default: set_error("low-pass tile"); rc = DWT_EUNSUPPORTED;
    }
#undef DWT_LOG
    dfree(d, st);
    if (rc) return rc;
    DWT_CK_LAUNCH("k2_lo_grouped");
    return DWT_OK;
}

// whole transforms of 2^L points, L = 12 .. 14, of several plans in one launch
int p2_lo_grouped(int L, const std::vector<GroupJob>& jobs, dwt_dtype t, int sgn, cudaStream_t st) {
    if (jobs.empty()) return DWT_OK;
    return t == DWT_F32 ? lo_grouped_t<float>(L, jobs, sgn, st) : lo_grouped_t<int>(L, jobs, sgn, st);
}

template <typename T>
static int launch_lo(int L, const T* in, T* out, long long ld_in, long long ld_out, int nf, long long N, float scale,
                     int do_scale, const char* fam, cudaStream_t st) {
    LoJob<T> a{in, out, ld_in, ld_out, nf, scale, do_scale, 0};
    return launch_lo2<T>(L, a, nullptr, N, fam, st);
}


template <typename T, int LT, int B, bool FUSED, bool HAS_COEF>
static int launch_hi_one(HiArgs a, int nf, size_t bins_bytes, const char* fam, cudaStream_t st) {
    using G = HiGeom<LT, B>;
    const size_t xbytes = (size_t)G::SMEM_ELEMS * sizeof(T);
    size_t smem = xbytes;
    if (FUSED) smem = (std::max(xbytes, bins_bytes) + 15) & ~(size_t)15;
    auto k = k2_hi<T, LT, B, FUSED, HAS_COEF>;
    int rc = attr_smem(k, smem);
    if (rc) return rc;
    dim3 grid((unsigned)a.ntile, (unsigned)nf);
    {
        LaunchScope ls(fam, st);
        k<<<grid, G::NT, smem, st>>>(a);
    }
    DWT_CK_LAUNCH("k2_hi");
    return DWT_OK;
}

template <typename T, int LT, bool FUSED, bool HAS_COEF>
static int launch_hi_t(int B, const HiArgs& a, int nf, size_t bins_bytes, const char* fam, cudaStream_t st) {
    switch (B) {
        case 4: return launch_hi_one<T, LT, 4, FUSED, HAS_COEF>(a, nf, bins_bytes, fam, st);
        case 5: return launch_hi_one<T, LT, 5, FUSED, HAS_COEF>(a, nf, bins_bytes, fam, st);
        case 6: return launch_hi_one<T, LT, 6, FUSED, HAS_COEF>(a, nf, bins_bytes, fam, st);
        case 7: return launch_hi_one<T, LT, 7, FUSED, HAS_COEF>(a, nf, bins_bytes, fam, st);
        case 8: return launch_hi_one<T, LT, 8, FUSED, HAS_COEF>(a, nf, bins_bytes, fam, st);
        case 9: return launch_hi_one<T, LT, 9, FUSED, HAS_COEF>(a, nf, bins_bytes, fam, st);
        case 10: return launch_hi_one<T, LT, 10, FUSED, HAS_COEF>(a, nf, bins_bytes, fam, st);
        default: set_error("high-pass digits"); return DWT_EUNSUPPORTED;
    }
}

static const long long kL2GroupP2 = 48ll << 20;

// forward (sgn < 0, scaled by 2^-m for FP32) or inverse transform, FP32 or int32
template <typename T>
static int p2_transform_t(dwt_plan_s* Pl, const T* in, T* out, int batch, long long ld_in, long long ld_out, int sgn,
                          cudaStream_t st) {
    const int m = Pl->m;
    const long long N = Pl->N;
    const bool scale = sgn < 0 && std::is_same<T, float>::value;
    const float sc = (float)(1.0 / (double)N);
    const long long fbytes = N * (long long)sizeof(T);
    int G = (int)std::max(1ll, kL2GroupP2 / fbytes);
    G = std::min(G, 65535);
    for (int f0 = 0; f0 < batch; f0 += G) {
        const int nf = std::min(G, batch - f0);
        const T* src = in + (long long)f0 * ld_in;
        T* dst = out + (long long)f0 * ld_out;
        if (m <= 14) {
            int rc = launch_lo<T>(m, src, dst, ld_in, ld_out, nf, N, sc, scale, sgn < 0 ? "p2_lo_fwd" : "p2_lo_inv", st);
            if (rc) return rc;
            continue;
        }
        const int L = p2_lo_digits_of(Pl);
        int rc = launch_lo<T>(L, src, dst, ld_in, ld_out, nf, N, 1.f, 0, sgn < 0 ? "p2_lo_fwd" : "p2_lo_inv", st);
        if (rc) return rc;
        HiArgs a{};
        a.in = dst;
        a.out = dst;
        a.ld_in = ld_out;
        a.ld_out = ld_out;
        a.S = 1ll << L;
        const int B = m - L;
        a.nlo = a.S >> (14 - B);
        a.ntile = N >> 14;
        a.scale = sc;
        a.do_scale = scale;
        rc = launch_hi_t<T, 14, false, false>(B, a, nf, 0, sgn < 0 ? "p2_hi_fwd" : "p2_hi_inv", st);
        if (rc) return rc;
    }
    return DWT_OK;
}

// only the FP32 high pass (digits L .. m-1) over data in place; forward scales by 2^-m
int p2_hi_only(dwt_plan_s* Pl, float* data, int batch, long long ld, int L, int sgn, cudaStream_t st) {
    if (L == 14 && p2i_transform_ok(Pl->m)) return p2i_hi_only(Pl, data, batch, ld, sgn, st);
    const int B = Pl->m - L;
    HiArgs a{};
    a.in = data;
    a.out = data;
    a.ld_in = ld;
    a.ld_out = ld;
    a.S = 1ll << L;
    a.nlo = a.S >> (14 - B);
    a.ntile = Pl->N >> 14;
    a.scale = (float)(1.0 / (double)Pl->N);
    a.do_scale = sgn < 0;
    for (int f0 = 0; f0 < batch; f0 += 65535) {
        HiArgs b = a;
        b.in = data + (long long)f0 * ld;
        b.out = data + (long long)f0 * ld;
        int rc = launch_hi_t<float, 14, false, false>(B, b, std::min(65535, batch - f0), 0,
                                                     sgn < 0 ? "p2_hi_fwd" : "p2_hi_inv", st);
        if (rc) return rc;
    }
    return DWT_OK;
}

int p2_transform(dwt_plan_s* Pl, const void* in, void* out, int batch, long long ld_in, long long ld_out,
                 dwt_dtype t, int sgn, cudaStream_t st) {
    if (t == DWT_F32 && p2i_transform_ok(Pl->m))
        return p2i_transform(Pl, (const float*)in, (float*)out, batch, ld_in, ld_out, sgn, st);
    if (t == DWT_F32)
        return p2_transform_t<float>(Pl, (const float*)in, (float*)out, batch, ld_in, ld_out, sgn, st);
    return p2_transform_t<int>(Pl, (const int*)in, (int*)out, batch, ld_in, ld_out, sgn, st);
}

// tile-major tables for the fused pass (plan time)
static constexpr int kFusedLT = 13;

int p2_build_tiled_tables(dwt_plan_s* Pl, cudaStream_t st) {
    const int m = Pl->m;
    if (Pl->p != 2 || m < 16 || m > 24) return DWT_OK;
    if (p2i_ok(m, Pl->s)) return DWT_OK;   // the TMA-staged top pass has its own tables
    constexpr int LT = kFusedLT;
    const int L = p2_low_digits(m);
    const int B = m - L;
    const long long N = Pl->N, S = 1ll << L, nlo = S >> (LT - B);
    if (dmalloc((void**)&Pl->d_Wt, (size_t)N * 4, st) || dmalloc((void**)&Pl->d_clst, (size_t)N * 2, st))
        return DWT_ENOMEM;
    const unsigned grid = (unsigned)(N >> LT);
    const float sc = (float)(1.0 / (double)N);
#define DWT_TT(BB)                                                                                          \
    case BB: {                                                                                              \
        LaunchScope ls("tile_tables", st);                                                                  \
        k2_tile_tables<LT, BB><<<grid, 1 << (LT - 6), 0, st>>>(Pl->d_W, Pl->d_cls, Pl->d_Wt, Pl->d_clst, S, nlo, sc); \
        break;                                                                                              \
    }
    switch (B) {
        DWT_TT(4)
        DWT_TT(5)
        DWT_TT(6)
        DWT_TT(7)
        DWT_TT(8)
        DWT_TT(9)
        DWT_TT(10)
        default: break;
    }
#undef DWT_TT
    DWT_CK_LAUNCH("k2_tile_tables");
    return DWT_OK;
}

// shared memory of the fused top pass: per-lane class bins of every warp and
// the per-warp class sums; the tile exchange buffer aliases them
static size_t fused_bins_bytes(int s) {
    const size_t nw = ((size_t)1 << (kFusedLT - 6)) >> 5, nb2 = 2 * (size_t)(s + 1);
    return (nw * nb2 * 32 + nw * nb2) * 4;
}

bool p2_interp_ok(int m, int s) {
    const size_t xbytes = ((size_t)1 << kFusedLT) * 4 + 1024;
    return m >= 16 && m <= 24 && std::max(fused_bins_bytes(s), xbytes) <= 227 * 1024;
}

// dwt_interpolate for p = 2, FP32, 16 <= m <= 24: forward low pass (f -> c),
// fused top pass (c -> c), inverse low pass (c -> c), per function so that c
// stays in L2 between the passes
int p2_interpolate(dwt_plan_s* Pl, const float* f, float* c, float* coef, int batch, long long ld, const float* W,
                   bool tc, double** part_out, long long* ntile_out, cudaStream_t st) {
    const int m = Pl->m;
    const long long N = Pl->N;
    constexpr int LT = kFusedLT;
    const int L = p2_low_digits(m);
    const int B = m - L;
    const int nb = Pl->s + 1, nb2 = 2 * nb;
    const size_t bins_bytes = fused_bins_bytes(Pl->s);
    if (!p2_interp_ok(m, Pl->s)) {
        set_error("shape outside the fused p = 2 pass");
        return DWT_EUNSUPPORTED;
    }
    const long long ntile = N >> LT;
    int rc = ensure_workspace(Pl, (size_t)batch * (ntile + 1) * nb2 * sizeof(double), st);
    if (rc) return rc;
    double* part = (double*)Pl->d_ws;
    const long long fbytes = N * 4;
    int G = (int)std::max(1ll, kL2GroupP2 / fbytes);
    G = std::min(G, 65535);
    // low passes: FP32 register tiles, or (tc) the split-BF16 tensor-core tiles
    int* err = nullptr;
    if (tc) {
        if (L != 14 || !tc_ok(m)) {
            set_error("the tensor-core interpolation covers 18 <= m <= 24");
            return DWT_EUNSUPPORTED;
        }
        if ((rc = dmalloc((void**)&err, sizeof(int), st))) return rc;
        DWT_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    }
    const long long tpf = N >> 14;
    // job a (n0 functions) and optionally job b; a is the inverse pass of the
    // final results when inv0 (stored with evict-first)
    auto low = [&](const float* i0, float* o0, int n0, bool inv0, const float* i1, float* o1, int n1,
                   const char* fam) {
        if (tc) {
            TcJob a{i0, o0, ld, ld, tpf, tpf * n0, 1.f};
            TcJob b{i1, o1, ld, ld, tpf, tpf * n1, 1.f};
            return launch_tc_lo14(a, i1 ? &b : nullptr, err, fam, st);
        }
        LoJob<float> a{i0, o0, ld, ld, n0, 1.f, 0, inv0 ? 1 : 0};
        LoJob<float> b{i1, o1, ld, ld, n1, 1.f, 0, 0};
        return launch_lo2<float>(L, a, i1 ? &b : nullptr, N, fam, st);
    };
    // forward low pass of the first group; then per group: fused top pass, and one
    // launch holding this group's inverse low pass and the next group's forward
    rc = low(f, c, std::min(G, batch), false, nullptr, nullptr, 0, "interp_fwd");
    if (rc) return rc;
    for (int f0 = 0; f0 < batch; f0 += G) {
        const int nf = std::min(G, batch - f0);
        const long long off = (long long)f0 * ld;
        HiArgs a{};
        a.in = c + off;
        a.out = c + off;
        a.ld_in = ld;
        a.ld_out = ld;
        a.S = 1ll << L;
        a.nlo = a.S >> (LT - B);
        a.ntile = ntile;
        a.scale = (float)(1.0 / (double)N);
        a.do_scale = 1;
        a.W = W ? Pl->d_Wt : nullptr;
        a.cls = Pl->d_clst;
        a.coef = coef ? (void*)(coef + off) : nullptr;
        a.part = part + (long long)f0 * ntile * nb2;
        a.nb = nb;
        rc = coef ? launch_hi_t<float, LT, true, true>(B, a, nf, bins_bytes, "interp_top", st)
                  : launch_hi_t<float, LT, true, false>(B, a, nf, bins_bytes, "interp_top", st);
        if (rc) return rc;
        const int g1 = f0 + G;
        if (g1 < batch) {
            const long long off1 = (long long)g1 * ld;
            rc = low(c + off, c + off, nf, true, f + off1, c + off1, std::min(G, batch - g1), "interp_inv_fwd");
        } else {
            rc = low(c + off, c + off, nf, true, nullptr, nullptr, 0, "interp_inv");
        }
        if (rc) return rc;
    }
    if (tc && (rc = tc_check(err, st))) return rc;
    *part_out = part;
    *ntile_out = ntile;
    return DWT_OK;
}

}  // namespace dwt
