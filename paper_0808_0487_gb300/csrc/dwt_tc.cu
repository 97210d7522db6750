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
// Per CTA (4 warps, one tile at a time): H_128 stays in shared memory as a
// K-major 128B-swizzled BF16 operand; X_hi / X_lo are written there by the
// threads; one elected thread issues tcgen05.mma (M = N = 128, K = 16 per
// instruction) into a 256-column TMEM allocation (D1 at column 0, D2 at 128);
// completion is signalled through an mbarrier; the warps read their 32 lanes
// of the accumulator with tcgen05.ld.  Every mbarrier wait is bounded: past the
// limit the kernel records an error and leaves, freeing its TMEM.
#include <cuda_bf16.h>
#include <stdint.h>

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

// bounded wait for the mbarrier phase; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(parity)
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

// shared-memory plan of the CTA (bytes, 1024-aligned operand blocks)
constexpr int kOpBytes = 128 * 128 * 2;   // one 128 x 128 BF16 operand (two 64-wide K blocks)
constexpr int kSmemH = 0;
constexpr int kSmemXhi = kOpBytes;
constexpr int kSmemXlo = 2 * kOpBytes;
constexpr int kSmemBar = 3 * kOpBytes;     // mbarrier (8 B) + TMEM address (4 B)
constexpr int kSmemTotal = 3 * kOpBytes + 64 + 1024;   // + slack to align the base to 1024

// element (row, k) of a 128-row, 128-wide operand = two 64-wide swizzled blocks
__device__ __forceinline__ uint32_t op_off(int row, int k) { return (uint32_t)((k >> 6) * (128 * 128)) + sw128(row, k & 63); }

// Transform of the low 14 digits of every 2^14-element tile of each function.
// grid: (tiles, functions); 128 threads.  scale multiplies the result.
__global__ void __launch_bounds__(128, 1) k_tc_lo14(const float* in, float* out, long long ld_in, long long ld_out,
                                                    float scale, int* err) {
    extern __shared__ __align__(1024) unsigned char smraw_unaligned[];
    unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smraw_unaligned + 1023) & ~(uintptr_t)1023);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(sm);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sm + kSmemBar + 8);
    const uint32_t bar_addr = s_base + kSmemBar;

    if (warp == 0) {
        const uint32_t slot = s_base + kSmemBar + 8;
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(slot) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_addr) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // H_128 (symmetric, entries (-1)^popcount(i & j)) as the K-major operand
    for (int idx = t; idx < 128 * 128; idx += 128) {
        const int i = idx >> 7, j = idx & 127;
        const unsigned short v = (__popc(i & j) & 1) ? 0xBF80u : 0x3F80u;   // -1.0 / +1.0 in BF16
        *reinterpret_cast<unsigned short*>(sm + kSmemH + op_off(i, j)) = v;
    }
    // the tile: X[n][k] = element k + 128 n, split into hi / lo operands
    const float* src = in + blockIdx.y * ld_in + ((long long)blockIdx.x << 14);
    float* dst = out + blockIdx.y * ld_out + ((long long)blockIdx.x << 14);
#pragma unroll 4
    for (int q = 0; q < 32; ++q) {
        const int e = 4 * (t + 128 * q);
        const float4 x = __ldcs(reinterpret_cast<const float4*>(src + e));
        const int n = e >> 7, k = e & 127;
        unsigned short h0, h1, h2, h3, l0, l1, l2, l3;
        split_bf16(x.x, h0, l0);
        split_bf16(x.y, h1, l1);
        split_bf16(x.z, h2, l2);
        split_bf16(x.w, h3, l3);
        const uint32_t o = op_off(n, k);   // 4 consecutive k stay inside one 16-byte chunk
        *reinterpret_cast<uint2*>(sm + kSmemXhi + o) = make_uint2(h0 | ((uint32_t)h1 << 16), h2 | ((uint32_t)h3 << 16));
        *reinterpret_cast<uint2*>(sm + kSmemXlo + o) = make_uint2(l0 | ((uint32_t)l1 << 16), l2 | ((uint32_t)l3 << 16));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    constexpr uint32_t ID = idesc_bf16(128, 128);
    bool ok = true;

    // round 1: D1 = H * X^T over k (8 K-steps of 16), hi then lo
    if (t == 0) {
        for (int part = 0; part < 2; ++part) {
            const uint32_t xb = s_base + (part ? kSmemXlo : kSmemXhi);
            for (int ks = 0; ks < 8; ++ks) {
                const uint32_t koff = (uint32_t)((ks >> 2) * (128 * 128) + (ks & 3) * 32);
                mma_bf16(tmem, desc_sw128(s_base + kSmemH + koff), desc_sw128(xb + koff), ID, part | ks);
            }
        }
        mma_commit(bar_addr);
    }
    ok = __syncthreads_and(mbar_wait(bar_addr, 0) ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // D1 row h = 32 warp + lane -> round-2 operand A[h][n] (K-major), hi / lo
    const int h = 32 * warp + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
    if (ok) {
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
            float v[32];
            tmem_ld32(lane_base + 32 * c, v);
#pragma unroll
            for (int g = 0; g < 4; ++g) {   // 8 values = one 16-byte chunk
                uint32_t hw[4], lw[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    unsigned short a0, a1, b0, b1;
                    split_bf16(v[8 * g + 2 * u], a0, b0);
                    split_bf16(v[8 * g + 2 * u + 1], a1, b1);
                    hw[u] = a0 | ((uint32_t)a1 << 16);
                    lw[u] = b0 | ((uint32_t)b1 << 16);
                }
                const uint32_t o = op_off(h, 32 * c + 8 * g);
                *reinterpret_cast<uint4*>(sm + kSmemXhi + o) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
                *reinterpret_cast<uint4*>(sm + kSmemXlo + o) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // round 2: D2 = D1 * H over n, into TMEM columns 128..255
    if (t == 0 && ok) {
        for (int part = 0; part < 2; ++part) {
            const uint32_t ab = s_base + (part ? kSmemXlo : kSmemXhi);
            for (int ks = 0; ks < 8; ++ks) {
                const uint32_t koff = (uint32_t)((ks >> 2) * (128 * 128) + (ks & 3) * 32);
                mma_bf16(tmem + 128, desc_sw128(ab + koff), desc_sw128(s_base + kSmemH + koff), ID, part | ks);
            }
        }
        mma_commit(bar_addr);
    }
    if (ok) ok = __syncthreads_and(mbar_wait(bar_addr, 1) ? 1 : 0) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // D2[h][h'] -> out[h + 128 h']: lanes write consecutive h
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
            float v[32];
            tmem_ld32(lane_base + 128 + 32 * c, v);
#pragma unroll
            for (int i = 0; i < 32; ++i) __stcg(dst + h + 128 * (32 * c + i), v[i] * scale);
        }
    } else if (t == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

// dwt_forward / dwt_inverse with DWT_ALGO_TC_SPLIT_BF16 for p = 2, FP32:
// the low 14 digits on the tensor cores; the digits above (m - 14 in 4..10)
// with the FP32 high pass.
int run_tc_transform(dwt_plan_s* Pl, const float* in, float* out, int batch, long long ld_in, long long ld_out,
                     int sgn, cudaStream_t st) {
    const int m = Pl->m;
    if (m < 14 || (m > 14 && (m - 14 < 4 || m - 14 > 10))) {
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
    cudaMemsetAsync(err, 0, sizeof(int), st);
    auto kern = k_tc_lo14;
    rc = smem_limit_max(kern);
    if (rc) return rc;
    const long long N = Pl->N;
    const float scale = (sgn < 0 && m == 14) ? (float)(1.0 / (double)N) : 1.f;
    for (int f0 = 0; f0 < batch; f0 += 65535) {
        const int nf = std::min(65535, batch - f0);
        {
            LaunchScope ls("tc_lo14", st);
            kern<<<dim3((unsigned)(N >> 14), (unsigned)nf), 128, kSmemTotal, st>>>(
                in + (long long)f0 * ld_in, out + (long long)f0 * ld_out, ld_in, ld_out, scale, err);
        }
        DWT_CK_LAUNCH("k_tc_lo14");
        if (m > 14) {
            rc = p2_hi_only(Pl, out + (long long)f0 * ld_out, nf, ld_out, 14, sgn, st);
            if (rc) return rc;
        }
    }
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
