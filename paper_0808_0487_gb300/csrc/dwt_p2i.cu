// dwt_p2i.cu -- the p = 2 interpolation step (forward transform, scale,
// weight, class variances, inverse transform) on nets of 2^20 .. 2^24 points.
//
// The step is three passes over each function (Algorithms 1 and 2 grouped by
// digits): a low pass over the 14 low digits (contiguous tiles of 2^14), the
// fused top pass over the B = m - 14 high digits, and the inverse low pass.
// Between the passes the function's 64 MB stay in L2.  This file holds
//
//  k2i_top<B>: the fused top pass.  A tile is 2^B rows (2^14 apart) of
//    Wc = 2^(14-B) consecutive columns, 64 KB, moved between L2 and shared
//    memory by the tensor-memory-access unit (cp.async.bulk.tensor), so that
//    the narrow row segments cost no load/store-unit work; 256 threads hold 64
//    elements each.  Register layouts as in the p = 2 high pass: layout A
//    (float4 at 4(t + 256 q), the top four row digits in thread) and layout P
//    (six row digits in thread).  Between the forward and inverse stages the
//    coefficients are scaled by 2^-m, weighted, squared and added to per-lane
//    class bins (truncation class = largest j with k_j != 0, superposition
//    class = number of j with k_j != 0, Sec. 4).
//  k2i_lo<L>: the low pass, two jobs per launch: the inverse of one group of
//    functions (whose top pass has finished) and the forward of the next,
//    tiles of the two jobs interleaved so that the HBM reads of the forward
//    overlap the HBM writes of the inverse.  Loads and stores carry L2
//    eviction priorities: data read for the last time and final results go
//    first, the intermediate of the next function stays.
//  k2i_tables<B>: plan-time per-coefficient tables in the order the top pass
//    reads them.  The weight prod_j (1 + k_j)^-2 of the coset leader k(H) is
//    1/Q^2 for the integer Q = prod_j (1 + k_j); when every Q is at most 2048
//    and every support size below 32 the table holds (Q - 1) | (|supp| << 11)
//    as 16 bits plus the max-support byte (3 bytes per coefficient), and the
//    pass forms the FP32 weight RN(1 / RN(Q^2)) (times 2^-m) itself; the plan
//    checks that value bit for bit against the weight table at every
//    coefficient.  Otherwise the table holds the FP32 weight (times 2^-m) and
//    both class bytes (6 bytes per coefficient).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "dwt_p2_tile.cuh"

namespace dwt {

// ---------------------------------------------------------------------------
// tensor-memory-access and mbarrier helpers (single CTA, no cluster multicast)
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void mbar_init1(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// Bounded wait on an mbarrier phase: each try suspends for at most ~1 us; after
// about two seconds of tries it gives up and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 21); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity), "r"(1000u)
            : "memory");
        if (done) return true;
    }
    return false;
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int x, int y, int z, uint32_t bar,
                                            uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint"
        " [%0], [%1, {%2, %3, %4}], [%5], %6;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(z), "r"(bar), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, int x, int y, int z, uint32_t src, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group.L2::cache_hint"
        " [%0, {%1, %2, %3}], [%4], %5;" ::"l"(reinterpret_cast<uint64_t>(tm)),
        "r"(x), "r"(y), "r"(z), "r"(src), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void bulk_load_1d(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar,
                                             uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ float4 ld_hint4(const float* p, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint4(float* p, float4 v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ uint4 ld_stream16(const void* p) {
    return __ldcs(reinterpret_cast<const uint4*>(p));
}

// ---------------------------------------------------------------------------
// fused top pass
struct TopArgs {
    float scale;            // 2^-m
    float two_m;            // 2^m
    int has_w;              // 0: weight 1 (scale only)
    const uint16_t* tq;     // compact tables: (Q - 1) | (|supp| << 11), or NULL
    const float* tw;        // full tables: W * 2^-m, or NULL
    const uint8_t* tkt;     // max-support class
    const uint8_t* tks;     // support-size class (full tables)
    float* coef;            // optional weighted coefficients (the group's first function)
    long long ld;
    double* part;           // [fn][class][tile]
    long long ntile;
    int nb;
    int codes_off;          // compact tables: byte offset of the tile's 16-bit codes in shared memory
    int* err;               // host-mapped: a bounded wait expired
};

// Per-lane class bins of one element pair (kt, ks bin indices of both): the
// pair's four bins are loaded first and stored last; when both elements fall
// in the same bin the second adds to the first's sum, so every bin ends with
// the element-order sum.
__device__ __forceinline__ void bin2(float* bt, float* bs, int kt0, int ks0, int kt1, int ks1, float q0, float q1) {
    const float xt0 = bt[32 * kt0], xt1 = bt[32 * kt1], xs0 = bs[32 * ks0], xs1 = bs[32 * ks1];
    const float rt0 = xt0 + q0, rs0 = xs0 + q0;
    const float rt1 = (kt1 == kt0 ? rt0 : xt1) + q1, rs1 = (ks1 == ks0 ? rs0 : xs1) + q1;
    bt[32 * kt0] = rt0;
    bs[32 * ks0] = rs0;
    bt[32 * kt1] = rt1;
    bs[32 * ks1] = rs1;
}

// Scaled FP32 weights of two coefficients from their Q: 2^-m RN(1 / RN(Q^2)) is
// RN(1 / x) with x = RN(Q^2) 2^m (exact: Q^2 < 2^24, powers of two).  The
// reciprocal is the hardware approximation refined by one Newton step
// (r' = r + r (1 - x r), with fused multiply-adds; Markstein's form), which
// the plan checks bit for bit against the weight table for every coefficient
// (otherwise the plan keeps the FP32 weights instead of Q).
__device__ __forceinline__ float rcp_newton(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return __fmaf_rn(r, __fmaf_rn(-x, r, 1.0f), r);
}
__device__ __forceinline__ float2 weights_of_q(unsigned q0, unsigned q1, float two_m) {
    const float2 q = make_float2((float)q0, (float)q1);
    const float2 x = __fmul2_rn(q, __fmul2_rn(q, make_float2(two_m, two_m)));
    return make_float2(rcp_newton(x.x), rcp_newton(x.y));
}

constexpr int kRowLog = 14;                 // a row of the top pass: the 2^14 points of a low-pass tile
constexpr int kTopLT = 13;                  // a top-pass tile: 2^13 points (2^B rows of 2^(13-B) columns)
constexpr int kTopNT = 1 << (kTopLT - 6);   // 64 points per thread
constexpr int kTopMinBlocks = kTopLT == 13 ? 4 : 2;

template <int B, int LT = kTopLT> struct TopGeom {
    using G = HiGeom<LT, B>;
    static constexpr int WC = 1 << G::CB;                  // columns per tile
    static constexpr int ROWS = 1 << B;
    static constexpr int BOXR = ROWS < 256 ? ROWS : 256;   // rows per tensor copy
    static constexpr int NBOX = ROWS / BOXR;
    static constexpr int TILE_BYTES = ROWS * WC * 4;       // 2^kTopLT points
};

template <int B, bool COMPACT, bool HAS_COEF>
__global__ void __launch_bounds__(kTopNT, kTopMinBlocks) k2i_top(const __grid_constant__ CUtensorMap tm, TopArgs a) {
    static_assert(B >= 6 && B <= 10, "top pass of 6 .. 10 digits");
    using G = HiGeom<kTopLT, B>;
    using TG = TopGeom<B>;
    using V = float2;
    constexpr int NT = kTopNT, P1 = G::P1, WC = TG::WC;
    // dynamic shared memory only (the kernel's limit is set to the device
    // maximum): the mbarrier first, the 128-byte aligned tile after it
    extern __shared__ __align__(16) unsigned char smraw[];
    uint64_t& bar = *reinterpret_cast<uint64_t*>(smraw);
    float* sm = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smraw) + 16 + 127) & ~(uintptr_t)127);
    const int t = threadIdx.x;
    const int fn = blockIdx.y;
    const long long tile = blockIdx.x;
    const int x0 = (int)(tile * WC);
    const uint64_t keep = policy_evict_last();
    const long long to = tile << kTopLT;
    // compact tables: the tile's 16-bit codes (32 KB, contiguous) come into
    // shared memory with the data tile; full tables are read into registers
    const uint4* qsm = COMPACT ? reinterpret_cast<const uint4*>(reinterpret_cast<const unsigned char*>(sm) + a.codes_off)
                               : nullptr;
    if (t == 0) {
        mbar_init1(smem_u32(&bar));
        mbar_expect_tx(smem_u32(&bar), TG::TILE_BYTES + (COMPACT ? (2u << kTopLT) : 0u));
#pragma unroll
        for (int b = 0; b < TG::NBOX; ++b)
            tma_load_3d(smem_u32(sm + b * TG::BOXR * WC), &tm, x0, b * TG::BOXR, fn, smem_u32(&bar), keep);
        if constexpr (COMPACT) {
            bulk_load_1d(smem_u32(qsm), a.tq + to, 2u << kTopLT, smem_u32(&bar), policy_evict_first());
        } else {
            // this tile's table range (contiguous) from HBM into L2, read after the forward stages
            prefetch_l2(a.tw + to, 4u << kTopLT);
            prefetch_l2(a.tks + to, 1u << kTopLT);
        }
    }
    // the max-support bytes: 16 per thread and table group, all four groups
    // requested now (compact); full tables: the first group now, then one ahead
    const uint4* kg = reinterpret_cast<const uint4*>(a.tkt + to) + t;
    const uint4* qg = reinterpret_cast<const uint4*>(COMPACT ? (const void*)(a.tq + to) : (const void*)(a.tw + to)) + t;
    const uint4* sg = reinterpret_cast<const uint4*>(a.tks + to) + t;
    constexpr int NK = COMPACT ? 4 : 2;
    uint4 tk[NK], tqv[2][5];
    auto fetch = [&](int g, int slot) {   // full tables
        tk[slot] = ld_stream16(kg + g * NT);
#pragma unroll
        for (int i = 0; i < 4; ++i) tqv[slot][i] = ld_stream16(qg + (4 * g + i) * NT);
        tqv[slot][4] = ld_stream16(sg + g * NT);
    };
    if constexpr (COMPACT) {
#pragma unroll
        for (int g = 0; g < 4; ++g) tk[g] = ld_stream16(kg + g * NT);
    } else {
        fetch(0, 0);
    }
    __syncthreads();   // barrier initialised before anyone waits on it
    if (!__syncthreads_and(mbar_wait_bounded(smem_u32(&bar), 0) ? 1 : 0)) {
        if (t == 0) atomicExch(a.err, 1);
        return;
    }
    V v[32];
    // layout A from the dense tile: float4 at 4(t + NT q)
#pragma unroll
    for (int q = 0; q < 16; ++q) ld16(sm + 4 * (t + NT * q), v + 2 * q);
    bfly_range<2, 6>(v);   // the top four row digits
    __syncthreads();       // the dense tile is read: the padded exchange may overwrite it
    float* pa = sm + 4 * t;
#pragma unroll
    for (int q = 0; q < 16; ++q) st16(pa + q * 4 * NT + G::PADC * (q >> G::QSH), v + 2 * q);
    __syncthreads();
    const int ep = (t & ((1 << P1) - 1)) | ((t >> P1) << (P1 + 6));
    float* pp = sm + ep + G::PADC * (ep >> G::PADSH);
#pragma unroll
    for (int j = 0; j < 64; ++j) comp(v[j >> 1], j & 1) = pp[j << P1];
    bfly_range<G::RLO, G::RHI>(v);   // the low row digits
    // class bins alias the exchange buffer
    float* bins = sm;
    const int nb2 = 2 * a.nb;
    const int lane = t & 31, w = t >> 5;
    __syncthreads();
    {
        float4* b4 = reinterpret_cast<float4*>(bins);
        for (int i = t; i < (NT >> 5) * nb2 * 8; i += NT) b4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    float* bt = bins + w * nb2 * 32 + lane;
    float* bs = bt + a.nb * 32;
    const bool has0 = tile == 0 && t == 0;   // coset label H = 0 is register 0 of thread 0 of tile 0
    float* coef = nullptr;
    if (HAS_COEF) coef = a.coef + (long long)fn * a.ld;
    // 16 elements per table group: j = 16 g + u
    auto body = [&](int g, uint4 kt16, const uint4* qw) {
        const uint32_t ktw[4] = {kt16.x, kt16.y, kt16.z, kt16.w};
#pragma unroll
        for (int u = 0; u < 16; u += 2) {
            const int j = 16 * g + u;
            const int kt0 = (int)((ktw[u >> 2] >> (8 * (u & 3))) & 0xffu);
            const int kt1 = (int)((ktw[(u + 1) >> 2] >> (8 * ((u + 1) & 3))) & 0xffu);
            float w0, w1;
            int ks0, ks1;
            if constexpr (COMPACT) {
                // qw: two uint4 of eight 16-bit codes
                const uint32_t c2 = reinterpret_cast<const uint32_t*>(qw)[u >> 1];
                const uint32_t c0 = c2 & 0xffffu, c1 = c2 >> 16;
                ks0 = (int)(c0 >> 11);
                ks1 = (int)(c1 >> 11);
                if (a.has_w) {
                    const float2 ww = weights_of_q((c0 & 2047u) + 1u, (c1 & 2047u) + 1u, a.two_m);
                    w0 = ww.x;
                    w1 = ww.y;
                } else {
                    w0 = w1 = a.scale;
                }
            } else {
                // qw: four float4 of weights, then one uint4 of support sizes
                const float* wf = reinterpret_cast<const float*>(qw);
                const uint32_t* ksw = reinterpret_cast<const uint32_t*>(qw + 4);
                w0 = a.has_w ? wf[u] : a.scale;
                w1 = a.has_w ? wf[u + 1] : a.scale;
                ks0 = (int)((ksw[u >> 2] >> (8 * (u & 3))) & 0xffu);
                ks1 = (int)((ksw[(u + 1) >> 2] >> (8 * ((u + 1) & 3))) & 0xffu);
            }
            V& vv = v[j >> 1];
            vv = __fmul2_rn(vv, make_float2(w0, w1));
            const float2 sq = __fmul2_rn(vv, vv);
            if constexpr (HAS_COEF) {
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int el = G::fused_e(t, j + e);
                    coef[(long long)(el >> G::CB) * (1ll << kRowLog) + x0 + (el & (WC - 1))] = comp(vv, e);
                }
            }
            bin2(bt, bs, kt0, ks0, kt1, ks1, (j == 0 && has0) ? 0.f : sq.x, sq.y);
        }
    };
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        if constexpr (COMPACT) {
            const uint4 q2[2] = {qsm[(2 * g) * NT + t], qsm[(2 * g + 1) * NT + t]};
            body(g, tk[g], q2);
        } else {
            if (g + 1 < 4) fetch(g + 1, (g + 1) & 1);
            body(g, tk[g & 1], tqv[g & 1]);
        }
        asm volatile("" ::: "memory");
    }
    __syncthreads();
    // per-tile class sums in a fixed order (as the p = 2 high pass): lane l of
    // warp w sums classes l, l+32, ... of its warp's block, reading the lane
    // columns rotated by l; the warp sums are added in warp order, in FP64.
    {
        constexpr int NW = NT >> 5;
        float* red = bins + NW * nb2 * 32;
        const float* wb = bins + w * nb2 * 32;
        for (int b = lane; b < nb2; b += 32) {
            float r[32];
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 x = *reinterpret_cast<const float4*>(wb + b * 32 + 4 * ((i + lane) & 7));
                r[4 * i] = x.x;
                r[4 * i + 1] = x.y;
                r[4 * i + 2] = x.z;
                r[4 * i + 3] = x.w;
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
            a.part[((long long)fn * nb2 + b) * a.ntile + tile] = (double)x;
        }
    }
    // inverse stages of the same digits: layout P, back to layout A, dense tile
    bfly_range<G::RLO, G::RHI>(v);
    __syncthreads();   // bins read out before the exchange reuses the buffer
#pragma unroll
    for (int j = 0; j < 64; ++j) pp[j << P1] = comp(v[j >> 1], j & 1);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) ld16(pa + q * 4 * NT + G::PADC * (q >> G::QSH), v + 2 * q);
    bfly_range<2, 6>(v);
    __syncthreads();   // padded layout read before the dense tile overwrites it
#pragma unroll
    for (int q = 0; q < 16; ++q) st16(sm + 4 * (t + NT * q), v + 2 * q);
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
#pragma unroll
        for (int b = 0; b < TG::NBOX; ++b) tma_store_3d(&tm, x0, b * TG::BOXR, fn, smem_u32(sm + b * TG::BOXR * WC), keep);
        bulk_commit();
        bulk_wait_read();   // shared memory may be released; the writes complete on their own
    }
}

// ---------------------------------------------------------------------------
// Plain high pass: the stages of the B digits above the 14 low ones (forward
// or inverse: for p = 2 the same butterflies), scaled by `scale` when asked
// (the forward's 2^-m), with the tile moved by the tensor-memory-access unit as
// in the top pass; in place.
constexpr int kHiLT = 14;                  // plain high pass: 2^14-point tiles (rows of 2^(14-B) columns)
constexpr int kHiNT = 1 << (kHiLT - 6);

template <int B>
__global__ void __launch_bounds__(kHiNT, 3) k2i_hi(const __grid_constant__ CUtensorMap tm, float scale, int do_scale,
                                                   int* err) {
    using G = HiGeom<kHiLT, B>;
    using TG = TopGeom<B, kHiLT>;
    using V = float2;
    constexpr int NT = kHiNT, P1 = G::P1, WC = TG::WC;
    extern __shared__ __align__(16) unsigned char smraw[];
    uint64_t& bar = *reinterpret_cast<uint64_t*>(smraw);
    float* sm = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smraw) + 16 + 127) & ~(uintptr_t)127);
    const int t = threadIdx.x;
    const int fn = blockIdx.y;
    const int x0 = (int)((long long)blockIdx.x * WC);
    const uint64_t first = policy_evict_first();
    if (t == 0) {
        mbar_init1(smem_u32(&bar));
        mbar_expect_tx(smem_u32(&bar), TG::TILE_BYTES);
#pragma unroll
        for (int b = 0; b < TG::NBOX; ++b)
            tma_load_3d(smem_u32(sm + b * TG::BOXR * WC), &tm, x0, b * TG::BOXR, fn, smem_u32(&bar), first);
    }
    __syncthreads();
    if (!__syncthreads_and(mbar_wait_bounded(smem_u32(&bar), 0) ? 1 : 0)) {
        if (t == 0) atomicExch(err, 1);
        return;
    }
    V v[32];
#pragma unroll
    for (int q = 0; q < 16; ++q) ld16(sm + 4 * (t + NT * q), v + 2 * q);
    bfly_range<2, 6>(v);
    __syncthreads();
    float* pa = sm + 4 * t;
#pragma unroll
    for (int q = 0; q < 16; ++q) st16(pa + q * 4 * NT + G::PADC * (q >> G::QSH), v + 2 * q);
    __syncthreads();
    const int ep = (t & ((1 << P1) - 1)) | ((t >> P1) << (P1 + 6));
    float* pp = sm + ep + G::PADC * (ep >> G::PADSH);
#pragma unroll
    for (int j = 0; j < 64; ++j) comp(v[j >> 1], j & 1) = pp[j << P1];
    bfly_range<G::RLO, G::RHI>(v);
    if (do_scale) {
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = pmul(v[k], scale);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 64; ++j) pp[j << P1] = comp(v[j >> 1], j & 1);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) ld16(pa + q * 4 * NT + G::PADC * (q >> G::QSH), v + 2 * q);
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 16; ++q) st16(sm + 4 * (t + NT * q), v + 2 * q);
    fence_async_smem();
    __syncthreads();
    if (t == 0) {
#pragma unroll
        for (int b = 0; b < TG::NBOX; ++b)
            tma_store_3d(&tm, x0, b * TG::BOXR, fn, smem_u32(sm + b * TG::BOXR * WC), first);
        bulk_commit();
        bulk_wait_read();
    }
}

// ---------------------------------------------------------------------------
// plan-time tables in the top pass's order: register j of thread t of tile T
// holds element e = fused_e(t, j) of the tile (row e >> CB, column e & (WC-1)),
// coefficient index H = row 2^14 + T WC + column.  16-bit codes: 8 per thread
// and group, at T 2^14 + 8 (g8 NT + t) + (j & 7); bytes: 16 per thread and
// group, at T 2^14 + 16 (g16 NT + t) + (j & 15); FP32 weights: 4 per thread
// and group, at T 2^14 + 4 (g4 NT + t) + (j & 3).
template <int B>
__global__ void __launch_bounds__(kTopNT) k2i_tables(const float* __restrict__ W, const uint8_t* __restrict__ cls,
                                                     uint16_t* tq, uint8_t* tkt, float* tw, uint8_t* tks, float scale,
                                                     float two_m, int* not_compact) {
    using G = HiGeom<kTopLT, B>;
    constexpr int NT = kTopNT, WC = TopGeom<B>::WC;
    const int t = threadIdx.x;
    const long long tile = blockIdx.x;
    const long long to = tile << kTopLT;
    for (int j = 0; j < 64; ++j) {
        const int el = G::fused_e(t, j);
        const long long H = (long long)(el >> G::CB) * (1ll << kRowLog) + tile * WC + (el & (WC - 1));
        const float w = W[H];
        const int kt = cls[2 * H], ks = cls[2 * H + 1];
        tkt[to + 16 * ((j >> 4) * NT + t) + (j & 15)] = (uint8_t)kt;
        if (tq) {
            // Q from the weight 1/Q^2: exact when it round-trips through RN(1 / RN(Q^2))
            const double qd = rint(1.0 / sqrt((double)w));
            const unsigned q = qd >= 1.0 && qd <= 2048.0 ? (unsigned)qd : 0u;
            if (q == 0u || ks > 31 || weights_of_q(q, q, two_m).x != w * scale) {
                atomicExch(not_compact, 1);
                tq[to + 8 * ((j >> 3) * NT + t) + (j & 7)] = 0;
            } else {
                tq[to + 8 * ((j >> 3) * NT + t) + (j & 7)] = (uint16_t)((q - 1u) | ((unsigned)ks << 11));
            }
        } else {
            tw[to + 4 * ((j >> 2) * NT + t) + (j & 3)] = w * scale;   // scale = 2^-m: exact
            tks[to + 16 * ((j >> 4) * NT + t) + (j & 15)] = (uint8_t)ks;
        }
    }
}

// ---------------------------------------------------------------------------
// low pass, two interleaved jobs
struct LoJobI {
    const float* in;
    float* out;
    long long ld;
    int nf;
    int final_out;   // 1: the inverse producing final results (in read for the last time)
};

template <int L>
__global__ void __launch_bounds__(1 << (L - 6), 3) k2i_lo(LoJobI j0, LoJobI j1, int njobs) {
    static_assert(L >= 12 && L <= 14, "low-pass tile 2^12 .. 2^14");
    using V = float2;
    constexpr int NT = 1 << (L - 6);
    extern __shared__ __align__(16) unsigned char smraw[];
    float* sm = reinterpret_cast<float*>(smraw);
    const int t = threadIdx.x;
    const bool second = njobs == 2 && (blockIdx.x & 1);
    const long long tile = njobs == 2 ? (blockIdx.x >> 1) : blockIdx.x;
    const LoJobI& J = second ? j1 : j0;
    if ((int)blockIdx.y >= J.nf) return;
    const float* src = J.in + blockIdx.y * J.ld + (tile << L);
    float* dst = J.out + blockIdx.y * J.ld + (tile << L);
    const uint64_t first = policy_evict_first(), keep = policy_evict_last();
    V v[32];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const float4 x = ld_hint4(src + 4 * (t + NT * q), first);
        v[2 * q] = make_float2(x.x, x.y);
        v[2 * q + 1] = make_float2(x.z, x.w);
    }
    bfly_range<0, 6>(v);
    lo_tile_compute<float, L>(sm, v, t);
    float* pd = dst + 4 * (t & 15) + 1024 * (t >> 4);
    const uint64_t pol = J.final_out ? first : keep;
#pragma unroll
    for (int g = 0; g < 16; ++g)
        st_hint4(pd + 64 * g, make_float4(v[2 * g].x, v[2 * g].y, v[2 * g + 1].x, v[2 * g + 1].y), pol);
}

// ---------------------------------------------------------------------------
// host side
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

static int tensor_map_fn() {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return DWT_ECUDA;
    }
    return DWT_OK;
}

// [nf][2^B rows][2^14] FP32 view of a group of functions (row pitch 2^14, function pitch ld), box WC x BOXR
template <int B, int LT = kTopLT>
static int top_tensor_map(CUtensorMap* tm, float* base, long long ld, int nf) {
    using TG = TopGeom<B, LT>;
    int rc = tensor_map_fn();
    if (rc) return rc;
    cuuint64_t dims[3] = {(cuuint64_t)1 << kRowLog, (cuuint64_t)TG::ROWS, (cuuint64_t)nf};
    cuuint64_t strides[2] = {((cuuint64_t)1 << kRowLog) * 4, (cuuint64_t)ld * 4};
    cuuint32_t box[3] = {(cuuint32_t)TG::WC, (cuuint32_t)TG::BOXR, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
        return DWT_ECUDA;
    }
    return DWT_OK;
}

static size_t top_bins_bytes(int s) {
    const size_t nw = kTopNT >> 5, nb2 = 2 * (size_t)(s + 1);
    return (nw * nb2 * 32 + nw * nb2) * 4;
}

// shared memory of the top pass: the mbarrier, the tile / exchange buffer /
// class bins (aliased; 128-byte aligned), then the compact tables' codes
static size_t top_region(int s, size_t x) { return (std::max(x, top_bins_bytes(s)) + 127) & ~(size_t)127; }
static constexpr size_t kCodesBytes = (size_t)2 << kTopLT;

template <int B>
static size_t top_smem(int s, bool compact) {
    const size_t x = (size_t)HiGeom<kTopLT, B>::SMEM_ELEMS * 4;
    return 16 + 128 + top_region(s, x) + (compact ? kCodesBytes : 0);
}

bool p2i_ok(int m, int s) {
    if (m < 20 || m > 24) return false;
    return 16 + 128 + top_region(s, (size_t)HiGeom<kTopLT, 10>::SMEM_ELEMS * 4) + kCodesBytes <= 227 * 1024;
}

template <int B, bool COMPACT, bool HAS_COEF>
static int launch_top_one(const CUtensorMap& tm, const TopArgs& a, int nf, int s, cudaStream_t st) {
    auto k = k2i_top<B, COMPACT, HAS_COEF>;
    int rc = smem_limit_max(k);
    if (rc) return rc;
    dim3 grid((unsigned)a.ntile, (unsigned)nf);
    {
        LaunchScope ls("interp_top", st);
        TopArgs a2 = a;
        a2.codes_off = (int)top_region(s, (size_t)HiGeom<kTopLT, B>::SMEM_ELEMS * 4);
        k<<<grid, kTopNT, top_smem<B>(s, COMPACT), st>>>(tm, a2);
    }
    DWT_CK_LAUNCH("k2i_top");
    return DWT_OK;
}

template <int B>
static int launch_top_b(float* base, long long ld, int nf, const TopArgs& a, int s, cudaStream_t st) {
    CUtensorMap tm;
    int rc = top_tensor_map<B>(&tm, base, ld, nf);
    if (rc) return rc;
    const bool compact = a.tq != nullptr;
    if (a.coef)
        return compact ? launch_top_one<B, true, true>(tm, a, nf, s, st) : launch_top_one<B, false, true>(tm, a, nf, s, st);
    return compact ? launch_top_one<B, true, false>(tm, a, nf, s, st) : launch_top_one<B, false, false>(tm, a, nf, s, st);
}

static int launch_top(int B, float* base, long long ld, int nf, const TopArgs& a, int s, cudaStream_t st) {
    switch (B) {
        case 6: return launch_top_b<6>(base, ld, nf, a, s, st);
        case 7: return launch_top_b<7>(base, ld, nf, a, s, st);
        case 8: return launch_top_b<8>(base, ld, nf, a, s, st);
        case 9: return launch_top_b<9>(base, ld, nf, a, s, st);
        case 10: return launch_top_b<10>(base, ld, nf, a, s, st);
        default: set_error("top-pass digits"); return DWT_EUNSUPPORTED;
    }
}

static int launch_lo_i(const LoJobI& a, const LoJobI* b, long long N, const char* fam, cudaStream_t st) {
    constexpr int L = 14;
    const unsigned tiles = (unsigned)(N >> L);
    const int nf = b ? std::max(a.nf, b->nf) : a.nf;
    dim3 grid(b ? 2 * tiles : tiles, (unsigned)nf);
    const size_t smem = (((size_t)1 << L) + ((size_t)1 << (L - 4))) * 4;
    auto k = k2i_lo<L>;
    int rc = smem_limit_max(k);
    if (rc) return rc;
    {
        LaunchScope ls(fam, st);
        k<<<grid, 1 << (L - 6), smem, st>>>(a, b ? *b : a, b ? 2 : 1);
    }
    DWT_CK_LAUNCH("k2i_lo");
    return DWT_OK;
}

static int status_word(int** host, int** dev);
static const long long kL2GroupP2i = 48ll << 20;   // functions per L2-resident group

template <int B>
static int launch_hi_b(float* base, long long ld, int nf, float scale, int do_scale, int* err, cudaStream_t st) {
    CUtensorMap tm;
    int rc = top_tensor_map<B, kHiLT>(&tm, base, ld, nf);
    if (rc) return rc;
    auto k = k2i_hi<B>;
    if ((rc = smem_limit_max(k))) return rc;
    const size_t smem = 16 + 128 + (size_t)HiGeom<kHiLT, B>::SMEM_ELEMS * 4;
    dim3 grid((unsigned)((1u << kRowLog) / TopGeom<B, kHiLT>::WC), (unsigned)nf);
    {
        LaunchScope ls(do_scale ? "p2_hi_fwd" : "p2_hi_inv", st);
        k<<<grid, kHiNT, smem, st>>>(tm, scale, do_scale, err);
    }
    DWT_CK_LAUNCH("k2i_hi");
    return DWT_OK;
}

static int launch_hi_i(int B, float* base, long long ld, int nf, float scale, int do_scale, int* err,
                       cudaStream_t st) {
    switch (B) {
        case 6: return launch_hi_b<6>(base, ld, nf, scale, do_scale, err, st);
        case 7: return launch_hi_b<7>(base, ld, nf, scale, do_scale, err, st);
        case 8: return launch_hi_b<8>(base, ld, nf, scale, do_scale, err, st);
        case 9: return launch_hi_b<9>(base, ld, nf, scale, do_scale, err, st);
        case 10: return launch_hi_b<10>(base, ld, nf, scale, do_scale, err, st);
        default: set_error("high-pass digits"); return DWT_EUNSUPPORTED;
    }
}

bool p2i_transform_ok(int m) { return m >= 20 && m <= 24; }

// The high digits 14 .. m-1 of FP32 data in place (after a low pass over the
// 14 low digits); the forward (sgn < 0) scales by 2^-m.
int p2i_hi_only(dwt_plan_s* Pl, float* data, int batch, long long ld, int sgn, cudaStream_t st) {
    int* err = nullptr;
    int* herr = nullptr;
    int rc = status_word(&herr, &err);
    if (rc) return rc;
    if (*(volatile int*)herr) {
        *herr = 0;
        set_error("an earlier call gave up a bounded wait in a p = 2 tensor-copied pass");
        return DWT_ETIMEOUT;
    }
    const float sc = (float)(1.0 / (double)Pl->N);
    for (int f0 = 0; f0 < batch; f0 += 65535) {
        const int nf = std::min(65535, batch - f0);
        rc = launch_hi_i(Pl->m - kRowLog, data + (long long)f0 * ld, ld, nf, sc, sgn < 0 ? 1 : 0, err, st);
        if (rc) return rc;
    }
    return DWT_OK;
}

// dwt_forward / dwt_inverse for p = 2, FP32, 20 <= m <= 24: per L2-sized group
// of functions the low pass (in -> out, the intermediate kept in L2) and the
// high pass in place.
int p2i_transform(dwt_plan_s* Pl, const float* in, float* out, int batch, long long ld_in, long long ld_out, int sgn,
                  cudaStream_t st) {
    const long long N = Pl->N;
    int G = (int)std::max(1ll, kL2GroupP2i / (N * 4));
    G = std::min(G, 65535);
    for (int f0 = 0; f0 < batch; f0 += G) {
        const int nf = std::min(G, batch - f0);
        if (ld_in != ld_out) {
            // the low pass takes one ld for both sides: run it per function
            for (int b = 0; b < nf; ++b) {
                LoJobI a{in + (long long)(f0 + b) * ld_in, out + (long long)(f0 + b) * ld_out, ld_out, 1, 0};
                int rc = launch_lo_i(a, nullptr, N, sgn < 0 ? "p2_lo_fwd" : "p2_lo_inv", st);
                if (rc) return rc;
            }
        } else {
            LoJobI a{in + (long long)f0 * ld_in, out + (long long)f0 * ld_out, ld_out, nf, 0};
            int rc = launch_lo_i(a, nullptr, N, sgn < 0 ? "p2_lo_fwd" : "p2_lo_inv", st);
            if (rc) return rc;
        }
        int rc = p2i_hi_only(Pl, out + (long long)f0 * ld_out, nf, ld_out, sgn, st);
        if (rc) return rc;
    }
    return DWT_OK;
}

template <int B>
static void launch_tables_b(dwt_plan_s* Pl, bool compact, int* flag, cudaStream_t st) {
    const unsigned grid = (unsigned)(Pl->N >> kTopLT);
    const float sc = (float)(1.0 / (double)Pl->N);
    LaunchScope ls("tile_tables", st);
    k2i_tables<B><<<grid, kTopNT, 0, st>>>(Pl->d_W, Pl->d_cls, compact ? Pl->d_tq : nullptr, Pl->d_tkt,
                                           compact ? nullptr : Pl->d_tw, compact ? nullptr : Pl->d_tks, sc,
                                           (float)(double)Pl->N, flag);
}

static int launch_tables(dwt_plan_s* Pl, bool compact, int* flag, cudaStream_t st) {
    switch (Pl->m - kRowLog) {
        case 6: launch_tables_b<6>(Pl, compact, flag, st); break;
        case 7: launch_tables_b<7>(Pl, compact, flag, st); break;
        case 8: launch_tables_b<8>(Pl, compact, flag, st); break;
        case 9: launch_tables_b<9>(Pl, compact, flag, st); break;
        case 10: launch_tables_b<10>(Pl, compact, flag, st); break;
        default: set_error("top-pass digits"); return DWT_EUNSUPPORTED;
    }
    DWT_CK_LAUNCH("k2i_tables");
    return DWT_OK;
}

// One host-mapped word for the whole process: a top pass that gives up a
// bounded wait sets it, and the next interpolation call on any plan reports
// DWT_ETIMEOUT and clears it.  Allocated once, never freed.
static int* g_status = nullptr;
static std::mutex g_status_mu;

static int status_word(int** host, int** dev) {
    std::lock_guard<std::mutex> lk(g_status_mu);
    if (!g_status) {
        count_host_alloc();
        if (cudaHostAlloc((void**)&g_status, sizeof(int), cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            g_status = nullptr;
            set_error("cudaHostAlloc of the status word failed");
            return DWT_ENOMEM;
        }
        *g_status = 0;
    }
    *host = g_status;
    DWT_CK(cudaHostGetDevicePointer((void**)dev, g_status, 0));
    return DWT_OK;
}

// Plan time: the top pass's tables (compact if every coefficient allows it).
int p2i_build_tables(dwt_plan_s* Pl, cudaStream_t st) {
    if (Pl->p != 2 || !p2i_ok(Pl->m, Pl->s)) return DWT_OK;
    const long long N = Pl->N;
    if (!Pl->h_err) {
        int rc0 = status_word(&Pl->h_err, &Pl->d_err);
        if (rc0) return rc0;
    }
    int* flag = nullptr;
    if (dmalloc((void**)&Pl->d_tq, (size_t)N * 2, st) || dmalloc((void**)&Pl->d_tkt, (size_t)N, st) ||
        dmalloc((void**)&flag, sizeof(int), st))
        return DWT_ENOMEM;
    DWT_CK(cudaMemsetAsync(flag, 0, sizeof(int), st));
    int rc = launch_tables(Pl, true, flag, st);
    if (rc) return rc;
    int hflag = 0;
    DWT_CK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWT_CK(cudaStreamSynchronize(st));
    dfree(flag, st);
    if (hflag) {
        // some coefficient needs the FP32 weight: full tables
        dfree(Pl->d_tq, st);
        Pl->d_tq = nullptr;
        if (dmalloc((void**)&Pl->d_tw, (size_t)N * 4, st) || dmalloc((void**)&Pl->d_tks, (size_t)N, st))
            return DWT_ENOMEM;
        rc = launch_tables(Pl, false, nullptr, st);
        if (rc) return rc;
    }
    return DWT_OK;
}

int p2i_table_bytes_per_point(dwt_plan_s* Pl) {
    if (Pl->d_tq) return 3;
    if (Pl->d_tw) return 6;
    return 0;
}


// dwt_interpolate for p = 2, FP32, 20 <= m <= 24: forward low pass (f -> c),
// fused top pass (c -> c), and the inverse low pass of each group of functions
// together with the forward low pass of the next; c stays in L2 in between.
// tc: the low passes on the tensor cores (split BF16).
int p2i_interpolate(dwt_plan_s* Pl, const float* f, float* c, float* coef, int batch, long long ld, bool weighted,
                    bool tc, double** part_out, long long* ntile_out, cudaStream_t st) {
    const int m = Pl->m;
    const long long N = Pl->N;
    const int B = m - kRowLog;
    const int nb = Pl->s + 1, nb2 = 2 * nb;
    if (!p2i_ok(m, Pl->s) || !Pl->d_tkt || !Pl->d_err) {
        set_error("shape outside the fused p = 2 top pass");
        return DWT_EUNSUPPORTED;
    }
    if (*(volatile int*)Pl->h_err) {
        *Pl->h_err = 0;
        set_error("an earlier interpolation call gave up a bounded wait in the p = 2 top pass");
        return DWT_ETIMEOUT;
    }
    const long long ntile = N >> kTopLT;
    int rc = ensure_workspace(Pl, (size_t)batch * (ntile + 1) * nb2 * sizeof(double), st);
    if (rc) return rc;
    double* part = (double*)Pl->d_ws;
    int G = (int)std::max(1ll, kL2GroupP2i / (N * 4));
    G = std::min(G, 65535);
    int* err = nullptr;
    if (tc) {
        if (!tc_ok(m)) {
            set_error("the tensor-core interpolation covers 18 <= m <= 24");
            return DWT_EUNSUPPORTED;
        }
        if ((rc = dmalloc((void**)&err, sizeof(int), st))) return rc;
        DWT_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    }
    const long long tpf = N >> 14;
    auto low = [&](const float* i0, float* o0, int n0, bool inv0, const float* i1, float* o1, int n1,
                   const char* fam) {
        if (tc) {
            TcJob a{i0, o0, ld, ld, tpf, tpf * n0, 1.f};
            TcJob b{i1, o1, ld, ld, tpf, tpf * n1, 1.f};
            return launch_tc_lo14(a, i1 ? &b : nullptr, err, fam, st);
        }
        LoJobI a{i0, o0, ld, n0, inv0 ? 1 : 0};
        LoJobI b{i1, o1, ld, n1, 0};
        return launch_lo_i(a, i1 ? &b : nullptr, N, fam, st);
    };
    rc = low(f, c, std::min(G, batch), false, nullptr, nullptr, 0, "interp_fwd");
    if (rc) return rc;
    for (int f0 = 0; f0 < batch; f0 += G) {
        const int nf = std::min(G, batch - f0);
        const long long off = (long long)f0 * ld;
        TopArgs a{};
        a.scale = (float)(1.0 / (double)N);
        a.two_m = (float)(double)N;
        a.has_w = weighted ? 1 : 0;
        a.tq = Pl->d_tq;
        a.tw = Pl->d_tw;
        a.tkt = Pl->d_tkt;
        a.tks = Pl->d_tks;
        a.coef = coef ? coef + off : nullptr;
        a.ld = ld;
        a.part = part + (long long)f0 * ntile * nb2;
        a.ntile = ntile;
        a.nb = nb;
        a.err = Pl->d_err;
        rc = launch_top(B, c + off, ld, nf, a, Pl->s, st);
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
