// dwt_tc.cu -- the split-BF16 tensor-core form of the p = 2 transform.
//
// For p = 2 the transform over 7 index digits is the product with the
// Sylvester-Hadamard matrix H_128 (entries +-1, exact in BF16), Sec. 2.2.  A
// contiguous tile of 2^14 elements is viewed as a 128 x 128 matrix X[n][k]
// (element k + 128 n); the 14 low digits are done by two tile products on the
// 5th-generation tensor cores:
//     round 1:  D1[h][n]  = sum_k H[h][k] X[n][k]          (digits 0..6)
//     round 2:  D2[h][h'] = sum_n D1[h][n] H[h'][n]        (digits 7..13)
// so that D2[h][h'] is the coefficient of H-index h + 128 h'.  Each FP32
// operand x is split as x = hi + lo with hi = bf16(x), lo = bf16(x - hi); both
// halves are multiplied by the exact +-1 matrix and accumulated in FP32 in
// tensor memory, which keeps about 16 bits of the mantissa (relative error of
// the split <= 2^-17 per element and round).
//
// Per CTA (4 warps, persistent over tiles, two CTAs per SM): H_128 stays in
// shared memory as a K-major 128B-swizzled BF16 operand, built once; X_hi /
// X_lo are written there by the threads; one elected thread issues tcgen05.mma
// (M = N = 128, K = 16 per instruction) into a 256-column TMEM allocation.
// Round 1 takes both operands from shared memory; its result D1 is read back
// (each thread one lane = one row), split, and written into tensor memory as
// the A operand of round 2, so the second product reads only H from shared
// memory.  The next tile is staged while round 2 runs.  Completion is
// signalled through an mbarrier; every wait is bounded: past the limit the
// kernel records an error and leaves, freeing its TMEM.
#include <cuda_bf16.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>

#include "dwt_internal.cuh"

namespace dwt {

bool p2_fast_ok(int m);
int p2_hi_only(dwt_plan_s* Pl, float* data, int batch, long long ld, int L, int sgn, cudaStream_t st);

// byte offset of BF16 element (row, k) in a K-major, 128B-swizzled operand
// block of 64 K-elements per row: 8-row atoms of 1024 B, 16-byte chunks of a
// row permuted by XOR with (row mod 8)
__device__ __forceinline__ uint32_t sw128(int row, int k) {
    return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((((k >> 3) ^ (row & 7)) & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                     // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024u >> 4) << 32;          // stride byte offset: 8-row atoms
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}

// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t dt, uint64_t ad, uint64_t bd, uint32_t idesc, int acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dt),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

// bounded wait for the mbarrier phase; false on timeout.  Each try suspends
// the thread for at most kWaitHintNs unless the phase completes, so a wait
// gives up after about iters microseconds.
constexpr uint32_t kWaitHintNs = 1000;
constexpr uint32_t kWaitIters = 1u << 21;   // about two seconds
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t iters = kWaitIters) {
    for (uint32_t it = 0; it < iters; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity), "r"(kWaitHintNs)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// split x into bf16 hi and lo, returned as raw 16-bit patterns
__device__ __forceinline__ void split_bf16(float x, unsigned short& hi, unsigned short& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    hi = __bfloat16_as_ushort(h);
    lo = __bfloat16_as_ushort(l);
}

// the same split for two values packed as one 32-bit column (element 2i in the
// low half): hi and lo words
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);   // .x = bf16(a) in the low half
    const float2 hf = __bfloat1622float2(h);
    unsigned long long ab, hh, d;
    const float2 abf = make_float2(a, b);
    memcpy(&ab, &abf, 8);
    memcpy(&hh, &hf, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(ab), "l"(hh));
    float2 df;
    memcpy(&df, &d, 8);
    const __nv_bfloat162 l = __floats2bfloat162_rn(df.x, df.y);
    memcpy(&hi, &h, 4);
    memcpy(&lo, &l, 4);
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t* r) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
            taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
        "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}

// A operand from tensor memory (M = 128 rows on the lanes, K packed two BF16 per column)
__device__ __forceinline__ void mma_bf16_ta(uint32_t dt, uint32_t at, uint64_t bd, uint32_t idesc, int acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(dt),
        "r"(at), "l"(bd), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void prefetch_l2_tc(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// shared-memory plan of the CTA (bytes, 1024-aligned operand blocks)
constexpr int kOpBytes = 128 * 128 * 2;   // one 128 x 128 BF16 operand (two 64-wide K blocks)
constexpr int kSmemH = 0;
constexpr int kSmemXhi = kOpBytes;
constexpr int kSmemXlo = 2 * kOpBytes;
constexpr int kSmemBar = 3 * kOpBytes;     // mbarrier (8 B) + TMEM address (4 B)
constexpr int kSmemTotal = 3 * kOpBytes + 64 + 1024;   // + slack to align the base to 1024
// tensor-memory plan (256 columns per CTA): two 128-column halves, one holding
// a tile's accumulator (D1, then D2), the other its round-2 A operand (P_hi in
// the first 64 columns, P_lo in the next 64); the roles swap from tile to tile

// element (row, k) of a 128-row, 128-wide operand = two 64-wide swizzled blocks
__device__ __forceinline__ uint32_t op_off(int row, int k) { return (uint32_t)((k >> 6) * (128 * 128)) + sw128(row, k & 63); }

constexpr int kTcThreads = 256;   // two warps per 32-lane quarter of tensor memory

// X (tile elements k + 128 n as rows n) -> hi / lo operands in shared memory;
// all 16 loads of a thread are issued before the first split
__device__ __forceinline__ void stage_x(unsigned char* sm, const float* src, int t) {
    // thread t takes 8 consecutive elements per step (one 16-byte chunk of
    // each operand): e = 8 (t + 256 q), q < 8
    float4 x4[16];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4* p = reinterpret_cast<const float4*>(src + 8 * (t + kTcThreads * q));
        x4[2 * q] = __ldcs(p);
        x4[2 * q + 1] = __ldcs(p + 1);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int e = 8 * (t + kTcThreads * q);
        const float4 x = x4[2 * q], y = x4[2 * q + 1];
        uint4 hw, lw;
        split2(x.x, x.y, hw.x, lw.x);
        split2(x.z, x.w, hw.y, lw.y);
        split2(y.x, y.y, hw.z, lw.z);
        split2(y.z, y.w, hw.w, lw.w);
        const uint32_t o = op_off(e >> 7, e & 127);
        *reinterpret_cast<uint4*>(sm + kSmemXhi + o) = hw;
        *reinterpret_cast<uint4*>(sm + kSmemXlo + o) = lw;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Transform of the low 14 digits of every 2^14-element tile of each function.
// Persistent: CTA b takes tiles b, b + gridDim.x, ... of the nf x tpf tiles
// (two CTAs per SM, 256 threads each; warps w and w + 4 share the 32 lanes
// 32 (w mod 4) of tensor memory and take one half of the columns each).  Per tile:
//   round 1: D1 = H X^T, A = H and B = X_hi, X_lo from shared memory;
//   the threads read D1 (lane h = row h), split it and store the BF16 halves
//   into tensor memory as the A operand of
//   round 2: D2 = P H^T, A = P_hi, P_lo from tensor memory, B = H;
// while round 2 runs the threads stage the next tile's X; then they read D2
// and store it.  scale multiplies the result.
__global__ void __launch_bounds__(kTcThreads, 2) k_tc_lo14(TcJob j0, TcJob j1, int* err) {
    const long long ntiles = j0.ntiles + j1.ntiles;
    extern __shared__ __align__(1024) unsigned char smraw_unaligned[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smraw_unaligned + 1023) & ~(uintptr_t)1023);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(sm);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kSmemBar + 8);
    const uint32_t bar_addr = s_base + kSmemBar;
    long long tile = blockIdx.x;
    if (tile >= ntiles) return;

    if (warp == 0) {
        const uint32_t slot = s_base + kSmemBar + 8;
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(slot) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_addr) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // H_128 (symmetric, entries (-1)^popcount(i & j)) as a K-major operand, once per CTA
    for (int idx = t; idx < 128 * 16; idx += kTcThreads) {
        const int i = idx >> 4, j0 = (idx & 15) * 8;   // 8 consecutive k = one 16-byte chunk
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint32_t a = (__popc(i & (j0 + 2 * u)) & 1) ? 0xBF80u : 0x3F80u;
            const uint32_t b = (__popc(i & (j0 + 2 * u + 1)) & 1) ? 0xBF80u : 0x3F80u;
            w[u] = a | (b << 16);
        }
        *reinterpret_cast<uint4*>(sm + kSmemH + op_off(i, j0)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    auto src_of = [&](long long i) {
        const TcJob& j = i < j0.ntiles ? j0 : j1;
        const long long k = i < j0.ntiles ? i : i - j0.ntiles;
        return j.in + (k / j.tpf) * j.ld_in + ((k % j.tpf) << 14);
    };
    // this CTA's first kPre tiles start moving into L2 at once; each iteration
    // then asks for the tile kPre steps ahead
    constexpr int kPre = 2;
    if (t == 0)
        for (int i = 1; i < kPre; ++i)
            if (tile + (long long)i * gridDim.x < ntiles) prefetch_l2_tc(src_of(tile + (long long)i * gridDim.x), 1u << 16);
    stage_x(sm, src_of(tile), t);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t ID = idesc_bf16(128, 128);
    const int h = 32 * (warp & 3) + lane, half = warp >> 2;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
    uint32_t phase = 0;
    bool ok = true;
    // The two 128-column halves of the allocation alternate: tile k accumulates
    // D1 and D2 in half R = k & 1 and keeps its round-2 operand P in the other
    // half, where tile k+1's D1 goes once round 2 of tile k has read P.  So the
    // next tile's round 1 is issued as soon as round 2 finishes, and runs while
    // the threads store this tile's D2.
    auto issue_round1 = [&](uint32_t dcol) {
        if (t == 0) {
            for (int part = 0; part < 2; ++part) {
                const uint32_t xb = s_base + (part ? kSmemXlo : kSmemXhi);
                for (int ks = 0; ks < 8; ++ks) {
                    const uint32_t koff = (uint32_t)((ks >> 2) * (128 * 128) + (ks & 3) * 32);
                    mma_bf16(tmem + dcol, desc_sw128(s_base + kSmemH + koff), desc_sw128(xb + koff), ID, part | ks);
                }
            }
            mma_commit(bar_addr);
        }
    };
    issue_round1(0);   // X of the first tile staged and fenced before the barrier above
    ok = __syncthreads_and(mbar_wait(bar_addr, phase) ? 1 : 0) != 0;
    phase ^= 1;
    for (int it = 0; ok && tile < ntiles; ++it, tile += gridDim.x) {
        const long long next = tile + gridDim.x;
        const uint32_t R = (it & 1) ? 128u : 0u, Ro = 128u - R;
        if (t == 0 && tile + (long long)kPre * gridDim.x < ntiles)
            prefetch_l2_tc(src_of(tile + (long long)kPre * gridDim.x), 1u << 16);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // round 1 of this tile has finished: D1 row h, this warp's half of the
        // columns -> P_hi / P_lo in the other half (two BF16 per column, element 2i low)
#pragma unroll 1
        for (int c = 2 * half; c < 2 * half + 2; ++c) {
            float v[32];
            tmem_ld32(lane_base + R + 32 * c, v);
            uint32_t hw[16], lw[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) split2(v[2 * i], v[2 * i + 1], hw[i], lw[i]);
            tmem_st16(lane_base + Ro + 16 * c, hw);
            tmem_st16(lane_base + Ro + 64 + 16 * c, lw);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // round 2: D2 = P H^T over n, into half R
        if (t == 0) {
            for (int part = 0; part < 2; ++part) {
                const uint32_t pa = tmem + Ro + (part ? 64u : 0u);
                for (int ks = 0; ks < 8; ++ks) {
                    const uint32_t koff = (uint32_t)((ks >> 2) * (128 * 128) + (ks & 3) * 32);
                    mma_bf16_ta(tmem + R, pa + 8 * ks, desc_sw128(s_base + kSmemH + koff), ID, part | ks);
                }
            }
            mma_commit(bar_addr);
        }
        // the next tile's X while round 2 runs (round 1 has finished reading X)
        if (next < ntiles) stage_x(sm, src_of(next), t);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        ok = __syncthreads_and(mbar_wait(bar_addr, phase) ? 1 : 0) != 0;
        phase ^= 1;
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // round 2 has read P: the next tile's round 1 into half Ro, then this
        // tile's D2[h][h'] -> out[h + 128 h'] (lanes write consecutive h)
        if (next < ntiles) issue_round1(Ro);
        const bool second = tile >= j0.ntiles;
        const TcJob& jb = second ? j1 : j0;
        const long long k = second ? tile - j0.ntiles : tile;
        float* dst = jb.out + (k / jb.tpf) * jb.ld_out + ((k % jb.tpf) << 14);
        const float scale = jb.scale;
#pragma unroll 1
        for (int c = 2 * half; c < 2 * half + 2; ++c) {
            float v[32];
            tmem_ld32(lane_base + R + 32 * c, v);
            if (scale == 1.f) {
#pragma unroll
                for (int i = 0; i < 32; ++i) __stcg(dst + h + 128 * (32 * c + i), v[i]);
            } else {
#pragma unroll
                for (int i = 0; i < 32; ++i) __stcg(dst + h + 128 * (32 * c + i), v[i] * scale);
            }
        }
        // every thread's D2 reads are done before the next tile writes its P
        // into half R; the next round 1 must have finished before its D1 is read
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (next < ntiles) {
            ok = __syncthreads_and(mbar_wait(bar_addr, phase) ? 1 : 0) != 0;
            phase ^= 1;
        }
    }
    if (!ok && t == 0) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

// Tensor-core low pass over one job, or two independent jobs in one launch
// (the first job's tiles first); err is the bounded-wait error flag.
int launch_tc_lo14(const TcJob& a, const TcJob* b, int* err, const char* fam, cudaStream_t st) {
    auto kern = k_tc_lo14;
    int rc = smem_limit_max(kern);
    if (rc) return rc;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    TcJob jb{};
    if (b) jb = *b;
    const long long ntiles = a.ntiles + jb.ntiles;
    if (ntiles == 0) return DWT_OK;
    const unsigned grid = (unsigned)std::min<long long>(ntiles, 2ll * std::max(nsm, 1));
    {
        LaunchScope ls(fam, st);
        kern<<<grid, kTcThreads, kSmemTotal, st>>>(a, jb, err);
    }
    DWT_CK_LAUNCH("k_tc_lo14");
    return DWT_OK;
}

// dwt_forward / dwt_inverse with DWT_ALGO_TC_SPLIT_BF16 for p = 2, FP32:
// the low 14 digits on the tensor cores; the digits above (m - 14 in 4..10)
// with the FP32 high pass, per group of functions whose data fits in L2 (about
// 48 MB), so that the high pass reads what the tensor-core pass has just written.
int run_tc_transform(dwt_plan_s* Pl, const float* in, float* out, int batch, long long ld_in, long long ld_out,
                     int sgn, cudaStream_t st) {
    const int m = Pl->m;
    if (!tc_ok(m)) {
        set_error("the tensor-core form covers m = 14 and 18 <= m <= 24");
        return DWT_EUNSUPPORTED;
    }
    if (((uintptr_t)in & 15) || ((uintptr_t)out & 15) || (ld_in & 3) || (ld_out & 3)) {
        set_error("the tensor-core form needs 16-byte aligned rows");
        return DWT_EUNSUPPORTED;
    }
    int* err = nullptr;
    int rc = dmalloc((void**)&err, sizeof(int), st);
    if (rc) return rc;
    DWT_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    const long long N = Pl->N, tpf = N >> 14;
    const float scale = (sgn < 0 && m == 14) ? (float)(1.0 / (double)N) : 1.f;
    const int G = (int)std::max(1ll, std::min(65535ll, (48ll << 20) / (N * 4)));
    for (int f0 = 0; f0 < batch && !rc; f0 += G) {
        const int nf = std::min(G, batch - f0);
        TcJob a{in + (long long)f0 * ld_in, out + (long long)f0 * ld_out, ld_in, ld_out, tpf, tpf * nf, scale};
        rc = launch_tc_lo14(a, nullptr, err, "tc_lo14", st);
        if (!rc && m > 14) rc = p2_hi_only(Pl, out + (long long)f0 * ld_out, nf, ld_out, 14, sgn, st);
    }
    if (!rc) rc = tc_check(err, st);
    else dfree(err, st);
    return rc;
}

// A wait that can never complete (an mbarrier that expects one arrival that
// never comes), bounded as every wait of the tensor-core kernels: it must give
// up and report, leaving the context usable.
__global__ void k_tc_wait_probe(uint32_t iters, int* err) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const bool ok = __syncthreads_and(mbar_wait(a, 0, iters) ? 1 : 0) != 0;
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
}

int run_wait_probe(cudaStream_t st) {
    int* err = nullptr;
    int rc = dmalloc((void**)&err, sizeof(int), st);
    if (rc) return rc;
    DWT_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
    {
        LaunchScope ls("tc_wait_probe", st);
        k_tc_wait_probe<<<1, 128, 0, st>>>(256u, err);
    }
    DWT_CK_LAUNCH("k_tc_wait_probe");
    return tc_check(err, st);
}

bool tc_ok(int m) { return m == 14 || (m >= 18 && m <= 24); }

// reads and releases the error flag of the tensor-core passes queued on st
int tc_check(int* err, cudaStream_t st) {
    int herr = 0;
    DWT_CK(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    DWT_CK(cudaStreamSynchronize(st));
    dfree(err, st);
    if (herr) {
        set_error("tensor-core pass: a bounded wait expired");
        return DWT_ETIMEOUT;
    }
    return DWT_OK;
}

}  // namespace dwt
