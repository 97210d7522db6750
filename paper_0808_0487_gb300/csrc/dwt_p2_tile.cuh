// dwt_p2_tile.cuh -- register-tile building blocks shared by the p = 2 kernels
// (packed butterflies, 16-byte moves, the low-pass tile layouts, the high-pass
// tile geometry and the per-lane class bins).  Internal to libdwt.
#pragma once

#include <string.h>

#include "dwt_internal.cuh"

namespace dwt {

// ---------------------------------------------------------------------------
// packed pairs: float2 uses the f32x2 pipe, int2 two scalar ops
template <typename T> struct P2;
template <> struct P2<float> { using t = float2; using v4 = float4; };
template <> struct P2<int> { using t = int2; using v4 = int4; };

__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
    unsigned long long ua, ub, ud;
    memcpy(&ua, &a, 8);
    memcpy(&ub, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ud) : "l"(ua), "l"(ub));
    float2 d;
    memcpy(&d, &ud, 8);
    return d;
}
__device__ __forceinline__ int2 padd(int2 a, int2 b) { return make_int2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ int2 psub(int2 a, int2 b) { return make_int2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 pmul(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ int2 pmul(int2 a, float) { return a; }

// register j of the 64 lives in v[j >> 1], component j & 1
template <typename V> __device__ __forceinline__ auto& comp(V& v, int c) { return c ? v.y : v.x; }

// butterflies over register-index bit RB
template <int RB, typename V>
__device__ __forceinline__ void bfly(V* v) {
    if constexpr (RB == 0) {
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            const auto a = v[k].x, b = v[k].y;
            v[k].x = a + b;
            v[k].y = a - b;
        }
    } else {
        constexpr int D = 1 << (RB - 1);
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            if (k & D) continue;
            const V a = v[k], b = v[k | D];
            v[k] = padd(a, b);
            v[k | D] = psub(a, b);
        }
    }
}
template <int LO, int HI, typename V>
__device__ __forceinline__ void bfly_range(V* v) {
    if constexpr (LO < HI) {
        bfly<LO, V>(v);
        bfly_range<LO + 1, HI, V>(v);
    }
}

// 16-byte moves between memory and two register pairs
template <typename T, typename V>
__device__ __forceinline__ void ld16(const T* p, V* v2) {
    const typename P2<T>::v4 x = *reinterpret_cast<const typename P2<T>::v4*>(p);
    v2[0].x = x.x; v2[0].y = x.y; v2[1].x = x.z; v2[1].y = x.w;
}
template <typename T, typename V>
__device__ __forceinline__ void ld16_cs(const T* p, V* v2) {   // read once: evict first
    const typename P2<T>::v4 x = __ldcs(reinterpret_cast<const typename P2<T>::v4*>(p));
    v2[0].x = x.x; v2[0].y = x.y; v2[1].x = x.z; v2[1].y = x.w;
}
template <typename T, typename V>
__device__ __forceinline__ void st16(T* p, const V* v2) {
    typename P2<T>::v4 x;
    x.x = v2[0].x; x.y = v2[0].y; x.z = v2[1].x; x.w = v2[1].y;
    *reinterpret_cast<typename P2<T>::v4*>(p) = x;
}

// bulk prefetch of [p, p + bytes) from global memory into L2 (bytes a multiple of 16)
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ---------------------------------------------------------------------------
// low pass: tile of 2^L contiguous elements.  Every shared-memory access moves
// 16 bytes: index bits 0,1 always stay in a thread's float4.
//   layout A: float4 at 4(t + NT q): in-thread bits {0,1} + {L-4..L-1}
//   layout B: 64 consecutive elements 64 t + (0..63): bits {0..5}
//   layout C: float4 at 4(t & 15) + 64 g + 1024 (t >> 4): bits {0,1} + {6..9}
// Stages: A all six, B bits 2..5, C the bits of 6..9 below L-4.
// Shared layout pad(e) = e + 4 (e >> 6): conflict-free for A, B and C.
__device__ __forceinline__ int pad_lo(int e) { return e + ((e >> 6) << 2); }

template <typename T, int L>
__device__ __forceinline__ void lo_tile_compute(T* sm, typename P2<T>::t* v, int t) {
    using V = typename P2<T>::t;
    constexpr int NT = 1 << (L - 6);
    // layout A -> shared (padded)
    {
        T* pa = sm + pad_lo(4 * t);
#pragma unroll
        for (int q = 0; q < 16; ++q) st16(pa + q * (4 * NT + NT / 4), v + 2 * q);
    }
    __syncthreads();
    // layout B: thread t holds elements 64 t .. 64 t + 63
    {
        T* pb = sm + pad_lo(64 * t);
#pragma unroll
        for (int g = 0; g < 16; ++g) ld16(pb + 4 * g, v + 2 * g);
        bfly_range<2, 6>(v);
#pragma unroll
        for (int g = 0; g < 16; ++g) st16(pb + 4 * g, v + 2 * g);
    }
    __syncthreads();
    // layout C
    {
        const T* pc = sm + pad_lo(4 * (t & 15) + 1024 * (t >> 4));
#pragma unroll
        for (int g = 0; g < 16; ++g) ld16(pc + 68 * g, v + 2 * g);
        bfly_range<2, 2 + (L - 10 < 4 ? L - 10 : 4)>(v);   // e bits 6 .. min(9, L-5)
    }
    (void)sizeof(V);
}

template <typename T, int L>
__device__ __forceinline__ void lo_tile_store(T* dst, const typename P2<T>::t* v, int t, bool stream_out) {
    T* pd = dst + 4 * (t & 15) + 1024 * (t >> 4);
    if (stream_out) {   // final output: evict first from L2
#pragma unroll
        for (int g = 0; g < 16; ++g) {
            typename P2<T>::v4 x;
            x.x = v[2 * g].x; x.y = v[2 * g].y; x.z = v[2 * g + 1].x; x.w = v[2 * g + 1].y;
            __stcs(reinterpret_cast<typename P2<T>::v4*>(pd + 64 * g), x);
        }
    } else {
#pragma unroll
        for (int g = 0; g < 16; ++g) st16(pd + 64 * g, v + 2 * g);
    }
}

template <int LT, int B> struct HiGeom {
    static constexpr int NT = 1 << (LT - 6);
    static constexpr int CB = LT - B;                                  // column bits
    static constexpr int P1 = (LT - B) < (LT - 6) ? (LT - B) : (LT - 6);
    static constexpr int PADSH = P1 + 6;                               // pad(e) = e + PADC (e >> PADSH)
    static constexpr int PADC = P1 < 5 ? (1 << P1) : 0;
    static constexpr int QSH = PADSH - (LT - 4);                       // layout A: e >> PADSH = q >> QSH
    static constexpr int SMEM_ELEMS = (1 << LT) + PADC * ((1 << LT) >> PADSH);
    // register bits of layout P that are row bits not transformed in layout A
    static constexpr int RLO = (LT - B) - P1;
    static constexpr int RHI = (LT - 4) - P1 < 6 ? (LT - 4) - P1 : 6;
    static __device__ __forceinline__ long long goff(int e, long long S) {
        return (long long)(e & ((1 << CB) - 1)) + S * (long long)(e >> CB);
    }
    // element held in register j by thread t when the fused pass weights the
    // coefficients: layout P (B > 4) or layout A (B = 4)
    static __host__ __device__ __forceinline__ int fused_e(int t, int j) {
        if constexpr (B > 4) return (t & ((1 << P1) - 1)) | ((t >> P1) << (P1 + 6)) | (j << P1);
        else return 4 * (t + NT * (j >> 2)) + (j & 3);
    }
};

// Class sums of one register group (4 consecutive elements of a thread, one
// 8-byte cls word: kt at byte 2u, ks at byte 2u + 1 for element u).  Element u
// adds q[u] to the lane's max-support bin bt[32 kt_u] and support-size bin
// bs[32 ks_u].  Elements go in pairs: the pair's four bins are loaded first and
// stored last, so their shared-memory round trips overlap; if both elements of
// the pair hit the same bin the second adds to the first's sum, so every bin
// ends with exactly the element-order sum (bin + q_0) + q_1 ... of the
// one-at-a-time form.
__device__ __forceinline__ void bin_pair(float* bt, float* bs, unsigned w, float q0, float q1) {
    const int kt0 = (int)(w & 0xffu), ks0 = (int)((w >> 8) & 0xffu);
    const int kt1 = (int)((w >> 16) & 0xffu), ks1 = (int)(w >> 24);
    const float xt0 = bt[32 * kt0], xt1 = bt[32 * kt1], xs0 = bs[32 * ks0], xs1 = bs[32 * ks1];
    const float rt0 = xt0 + q0, rs0 = xs0 + q0;
    const float rt1 = (kt1 == kt0 ? rt0 : xt1) + q1, rs1 = (ks1 == ks0 ? rs0 : xs1) + q1;
    bt[32 * kt0] = rt0;
    bs[32 * ks0] = rs0;
    bt[32 * kt1] = rt1;
    bs[32 * ks1] = rs1;
}

__device__ __forceinline__ void bin_group(float* bt, float* bs, uint2 c, const float (&q)[4]) {
    bin_pair(bt, bs, c.x, q[0], q[1]);
    bin_pair(bt, bs, c.y, q[2], q[3]);
}

}  // namespace dwt
