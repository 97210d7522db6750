// dwt_transform.cu -- radix-p Walsh (Chrestenson) transforms over digital nets,
// Algorithm 1 (forward, eq. fdwt) and Algorithm 2 (inverse), plus the fused
// weighting / effective-dimension pass of the interpolation (Sec. 3, Sec. 4).
//
// The transform of Sec. 2.2 is the Kronecker power over the m index digits of
// the p-point DFT F[h][n] = omega^{-hn}: the sum over digit n_r touches nothing
// but digit r, and the sums over different digits commute.  Digits are
// therefore processed in passes of b digits each; a pass covers a tile of p^b
// "rows" (one per value of its digits) times Wc "columns" (consecutive values
// of the digits below the pass).  Inside a tile every thread takes p^K elements
// that differ only in K consecutive digits and runs those K stages in
// registers; groups of K digits follow one another through shared memory, the
// first read straight from global memory and the last, where the rows allow,
// written straight back.
#include <string.h>

#include <type_traits>

#include "dwt_internal.cuh"

namespace dwt {

bool p2_fast_ok(int m);
bool p2_interp_ok(int m, int s);
int p2_transform(dwt_plan_s* Pl, const void* in, void* out, int batch, long long ld_in, long long ld_out,
                 dwt_dtype t, int sgn, cudaStream_t st);
int p2_interpolate(dwt_plan_s* Pl, const float* f, float* c, float* coef, int batch, long long ld, const float* W,
                   bool tc, double** part_out, long long* ntile_out, cudaStream_t st);

static bool aligned16(const void* p, long long ld, int elem) {
    return ((uintptr_t)p & 15) == 0 && ((ld * elem) & 15) == 0;
}

// ---------------------------------------------------------------------------
// element helpers
struct Tw {
    float c[32], s[32];   // cos, sin of 2 pi e / p, e < p <= 31
    double cd[32], sd[32];
};

template <typename T> struct IsCplx : std::false_type {};
template <> struct IsCplx<float2> : std::true_type {};
template <> struct IsCplx<double2> : std::true_type {};

template <typename T> __device__ __forceinline__ T zero_of();
template <> __device__ __forceinline__ float zero_of<float>() { return 0.f; }
template <> __device__ __forceinline__ double zero_of<double>() { return 0.0; }
template <> __device__ __forceinline__ int zero_of<int>() { return 0; }
template <> __device__ __forceinline__ float2 zero_of<float2>() { return make_float2(0.f, 0.f); }
template <> __device__ __forceinline__ double2 zero_of<double2>() { return make_double2(0.0, 0.0); }

template <typename T, typename TI> __device__ __forceinline__ T promote(TI v) { return v; }
template <> __device__ __forceinline__ float2 promote<float2, float>(float v) { return make_float2(v, 0.f); }
template <> __device__ __forceinline__ double2 promote<double2, double>(double v) { return make_double2(v, 0.0); }

// complex FP32 on the packed f32x2 pipe: one instruction per complex add
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
    unsigned long long ua, ub, ud;
    memcpy(&ua, &a, 8);
    memcpy(&ub, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ud) : "l"(ua), "l"(ub));
    float2 d;
    memcpy(&d, &ud, 8);
    return d;
}
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }

template <typename T> __device__ __forceinline__ T scale_by(T v, double s);
template <> __device__ __forceinline__ float scale_by<float>(float v, double s) { return v * (float)s; }
template <> __device__ __forceinline__ double scale_by<double>(double v, double s) { return v * s; }
template <> __device__ __forceinline__ int scale_by<int>(int v, double) { return v; }
template <> __device__ __forceinline__ float2 scale_by<float2>(float2 v, double s) {
    return make_float2(v.x * (float)s, v.y * (float)s);
}
template <> __device__ __forceinline__ double2 scale_by<double2>(double2 v, double s) {
    return make_double2(v.x * s, v.y * s);
}

// shared-memory index with one pad element per 128 bytes (bank spreading)
template <typename T> struct PadLog { static constexpr int v = sizeof(T) == 4 ? 5 : sizeof(T) == 8 ? 4 : 3; };
template <typename T> __device__ __forceinline__ int spad(int i) { return i + (i >> PadLog<T>::v); }
template <typename T> static inline size_t spad_bytes(int nel) {
    int last = nel - 1;
    return (size_t)(last + (last >> PadLog<T>::v) + 1) * sizeof(T);
}

constexpr int cpow(int p, int k) { return k == 0 ? 1 : p * cpow(p, k - 1); }

// ---------------------------------------------------------------------------
// one p-point DFT y_t = sum_u omega^{SGN u t} x_u in registers, odd p.  The
// terms u and p - u pair up: with s_u = x_u + x_{p-u} and d_u = x_u - x_{p-u},
//   y_t     = x_0 + sum_u cos(2 pi ut/p) s_u + i SGN sum_u sin(2 pi ut/p) d_u,
//   y_{p-t} = the same with the sine sum negated,
// for u, t = 1 .. (p-1)/2: real-by-complex products only, shared by both outputs.
template <typename T> struct TwOf;
template <> struct TwOf<float2> {
    static __device__ __forceinline__ float c(const Tw& tw, int e) { return tw.c[e]; }
    static __device__ __forceinline__ float s(const Tw& tw, int e) { return tw.s[e]; }
};
template <> struct TwOf<double2> {
    static __device__ __forceinline__ double c(const Tw& tw, int e) { return tw.cd[e]; }
    static __device__ __forceinline__ double s(const Tw& tw, int e) { return tw.sd[e]; }
};

// y = c x + a for real c and complex x, a
__device__ __forceinline__ float2 cfma(float c, float2 x, float2 a) { return __ffma2_rn(make_float2(c, c), x, a); }
__device__ __forceinline__ double2 cfma(double c, double2 x, double2 a) {
    return make_double2(fma(c, x.x, a.x), fma(c, x.y, a.y));
}
// a + g i b with g = +-1: (a.x - g b.y, a.y + g b.x)
template <int G> __device__ __forceinline__ float2 add_ib(float2 a, float2 b) {
    return __ffma2_rn(make_float2(-(float)G, (float)G), make_float2(b.y, b.x), a);
}
template <int G> __device__ __forceinline__ double2 add_ib(double2 a, double2 b) {
    return make_double2(a.x - G * b.y, a.y + G * b.x);
}

template <int P, int SGN, typename T> struct Dft {
    static __device__ __forceinline__ void run(T* x, const Tw& tw) {
        static_assert(IsCplx<T>::value, "p > 2 needs complex data");
        constexpr int H = (P - 1) / 2;
        T sp[H], dm[H];
        T y0 = x[0];
#pragma unroll
        for (int u = 1; u <= H; ++u) {
            sp[u - 1] = x[u] + x[P - u];
            dm[u - 1] = x[u] - x[P - u];
            y0 = y0 + sp[u - 1];
        }
#pragma unroll
        for (int t = 1; t <= H; ++t) {
            T a = x[0], b = zero_of<T>();
#pragma unroll
            for (int u = 1; u <= H; ++u) {
                const int e = (u * t) % P;
                a = cfma(TwOf<T>::c(tw, e), sp[u - 1], a);
                b = cfma(TwOf<T>::s(tw, e), dm[u - 1], b);
            }
            x[t] = add_ib<SGN>(a, b);
            x[P - t] = add_ib<-SGN>(a, b);
        }
        x[0] = y0;
    }
};

// p = 2: omega = -1 both ways
template <int SGN, typename T> struct Dft<2, SGN, T> {
    static __device__ __forceinline__ void run(T* x, const Tw&) {
        T a = x[0], b = x[1];
        x[0] = a + b;
        x[1] = a - b;
    }
};

// K stages over the K digits of a register array of P^K elements
template <int P, int NK, int ST, int SGN, typename T> struct RegStages {
    static __device__ __forceinline__ void run(T* v, const Tw& tw) {
#pragma unroll
        for (int blk = 0; blk < NK; blk += ST * P) {
#pragma unroll
            for (int off = 0; off < ST; ++off) {
                T x[P];
#pragma unroll
                for (int u = 0; u < P; ++u) x[u] = v[blk + off + u * ST];
                Dft<P, SGN, T>::run(x, tw);
#pragma unroll
                for (int u = 0; u < P; ++u) v[blk + off + u * ST] = x[u];
            }
        }
        RegStages<P, NK, ST * P, SGN, T>::run(v, tw);
    }
};
template <int P, int NK, int SGN, typename T> struct RegStages<P, NK, NK, SGN, T> {
    static __device__ __forceinline__ void run(T*, const Tw&) {}
};

// digits per register group: p^K elements per thread (27 complex FP32 at p = 3)
template <int P, typename T> struct KMax {
    static constexpr int v = P == 2 ? (sizeof(T) == 8 ? 4 : 5)
                                    : (sizeof(T) == 8 ? (P == 3 ? 3 : P == 5 ? 2 : 1) : (P == 3 ? 2 : 1));
};

// ---------------------------------------------------------------------------
struct PassArgs {
    const void* in;
    void* out;
    long long ld_in, ld_out;
    long long S, SR, nlo;
    int R, b, Wc, wlog;
    double scale;
    int do_scale;
    Tw tw;
};

// Register groups of a pass.  A tile has R = p^b rows (row digits 0 .. b-1) of
// Wc columns; element (r, c) sits at tile index (r << wlog) + c in shared
// memory and at offset c + S r from the tile base in global memory.  A group
// runs the stages of the k row digits [g0, g0 + k): each task holds the p^k
// elements that differ in those digits, rows r0 + i p^g0 with
// r0 = rl + rh p^(g0+k) (rl < p^g0, rh < R / p^(g0+k)), in one column.  Tasks
// are numbered column first, then rl, then rh, so that neighbouring threads
// touch neighbouring columns and rows (coalesced global access); with RHF the
// order of rl and rh is swapped, so that neighbouring threads are p^(g0+k)
// rows apart: an odd stride for odd p, which spreads them over all shared
// memory banks without padding.  A group reads from global memory (SRC_G) or
// shared memory and writes to global memory (DST_G) or shared memory.
template <int P, typename T> __device__ __forceinline__ int sx(int e) { return (P & 1) ? e : spad<T>(e); }

template <int P, int K, int SGN, typename T, typename TI, bool SRC_G, bool DST_G, bool RHF>
__device__ __forceinline__ void rgroup(T* sm, const TI* gin, T* gout, int g0, const PassArgs& a, int ncols) {
    constexpr int NK = cpow(P, K);
    unsigned pg0 = 1;
    for (int i = 0; i < g0; ++i) pg0 *= P;
    const unsigned pgk = pg0 * NK;
    const unsigned nrh = (unsigned)a.R / pgk;
    const unsigned ntask = ((unsigned)a.R / NK) << a.wlog;
    // q / dv = (q mg) >> 42, exact while q dv < 2^42 (q, dv <= R <= 2^16 here)
    const unsigned dv = RHF ? nrh : pg0;
    const unsigned long long mg = (1ull << 42) / dv + 1;
    const unsigned cmask = (unsigned)a.Wc - 1;
    const long long step = a.S * (long long)pg0;
    for (unsigned t = threadIdx.x; t < ntask; t += blockDim.x) {
        const unsigned c = t & cmask, q = t >> a.wlog;
        const unsigned qd = (unsigned)(((unsigned long long)q * mg) >> 42), qm = q - qd * dv;
        const unsigned rl = RHF ? qd : qm, rh = RHF ? qm : qd;
        const unsigned r0 = rl + rh * pgk;
        const bool live = (int)c < ncols;
        T v[NK];
        if constexpr (SRC_G) {
            const TI* src = gin + c + a.S * (long long)r0;
#pragma unroll
            for (int i = 0; i < NK; ++i) v[i] = live ? promote<T, TI>(src[i * step]) : zero_of<T>();
        } else {
#pragma unroll
            for (int i = 0; i < NK; ++i) v[i] = sm[sx<P, T>((int)(((r0 + i * pg0) << a.wlog) + c))];
        }
        RegStages<P, NK, 1, SGN, T>::run(v, a.tw);
        if constexpr (DST_G) {
            if (live) {
                T* dst = gout + c + a.S * (long long)r0;
#pragma unroll
                for (int i = 0; i < NK; ++i) dst[i * step] = a.do_scale ? scale_by<T>(v[i], a.scale) : v[i];
            }
        } else {
#pragma unroll
            for (int i = 0; i < NK; ++i) sm[sx<P, T>((int)(((r0 + i * pg0) << a.wlog) + c))] = v[i];
        }
    }
}

// mode bits: 1 read global, 2 write global, 4 rh-first numbering
template <int P, int SGN, typename T, typename TI, int K>
__device__ __forceinline__ void rgroup_k(int k, int mode, T* sm, const TI* gin, T* gout, int g0, const PassArgs& a,
                                         int ncols) {
    if constexpr (K >= 1) {
        if (k == K) {
            switch (mode) {
                case 1: rgroup<P, K, SGN, T, TI, true, false, false>(sm, gin, gout, g0, a, ncols); break;
                case 2: rgroup<P, K, SGN, T, TI, false, true, false>(sm, gin, gout, g0, a, ncols); break;
                case 3: rgroup<P, K, SGN, T, TI, true, true, false>(sm, gin, gout, g0, a, ncols); break;
                default:
                    if constexpr (P & 1) rgroup<P, K, SGN, T, TI, false, false, true>(sm, gin, gout, g0, a, ncols);
                    else rgroup<P, K, SGN, T, TI, false, false, false>(sm, gin, gout, g0, a, ncols);
                    break;
            }
            return;
        }
        rgroup_k<P, SGN, T, TI, K - 1>(k, mode, sm, gin, gout, g0, a, ncols);
    }
}

// One pass over the digits d0 .. d0+b-1 of every function: grid (tiles,
// functions).  The first group takes the top digits and reads the tile from
// global memory straight into registers (coalesced: neighbouring threads hold
// neighbouring rows, or columns); the other digits follow bottom-up through
// shared memory.  The last group, which then has the longest runs of
// neighbouring rows below it, writes straight to global memory when a run
// (p^g0 rows in the low pass, Wc columns in the others) spans at least 64
// bytes; otherwise it writes shared memory and the tile leaves in element
// order.  In place is safe: a tile is read in full before any of it is written
// (a one-group pass reads and writes the same elements per thread).
// Register cap: 96 x 512 threads fit the register file; a single digit of a
// prime above 13 holds p complex elements and the p-point sums, so those
// passes get 160 registers and at most 384 threads.
template <int P> constexpr int pass_maxnreg() { return P > 13 ? 160 : 96; }
template <int P> constexpr long long pass_max_threads() { return P > 13 ? 384 : 512; }

template <int P, typename T, typename TI, int SGN, int KM>
__device__ __forceinline__ void pass_body(const PassArgs& a, long long tile, long long fn) {
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const long long lo0 = (tile % a.nlo) << a.wlog;
    const long long base = lo0 + (tile / a.nlo) * a.SR;
    const int ncols = (int)min((long long)a.Wc, a.S - lo0);
    const TI* in = reinterpret_cast<const TI*>(a.in) + fn * a.ld_in + base;
    T* out = reinterpret_cast<T*>(a.out) + fn * a.ld_out + base;
    const int b = a.b;
    const int k0 = min(KM, b);
    // the last group: the top of the digits below the first group
    const int g_last = b == k0 ? 0 : ((b - k0 - 1) / KM) * KM;
    long long run = 1;
    if (a.S == 1) {
        for (int i = 0; i < g_last; ++i) run *= P;
    } else {
        run = a.Wc;
    }
    const bool direct_out = run * (long long)sizeof(T) >= 64;
    int g0 = b - k0, k = k0;
    for (;;) {
        const bool last = g0 == g_last;
        const int mode = (g0 + k == b ? 1 : 0) | (last && direct_out ? 2 : 0) | (g0 + k != b && !(last && direct_out) ? 4 : 0);
        rgroup_k<P, SGN, T, TI, KM>(k, mode, sm, in, out, g0, a, ncols);
        if (!(last && direct_out)) __syncthreads();
        if (last) break;
        g0 = g0 + k == b ? 0 : g0 + k;   // after the top group, bottom-up
        k = min(KM, b - k0 - g0);
    }
    if (!direct_out) {
        const int nel = a.R << a.wlog;
        const int cmask = a.Wc - 1;
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
            const int r = e >> a.wlog, c = e & cmask;
            if (c < ncols) {
                T v = sm[sx<P, T>(e)];
                if (a.do_scale) v = scale_by<T>(v, a.scale);
                out[c + (long long)r * a.S] = v;
            }
        }
    }
}

template <int P, typename T, typename TI, int SGN, int KM>
__global__ void __maxnreg__(pass_maxnreg<P>()) k_pass(PassArgs a) {
    pass_body<P, T, TI, SGN, KM>(a, blockIdx.x, blockIdx.y);
}

// One pass of several plans' transforms in one launch: job i owns the blocks
// [first, first + ntile * nf) (tile fastest).  Each block runs exactly the tile
// body of k_pass, so every element is computed as by the plan's own launch.
struct GroupPass {
    PassArgs a;
    long long ntile, first;
};

template <int P, typename T, typename TI, int SGN, int KM>
__global__ void __maxnreg__(pass_maxnreg<P>()) k_pass_grouped(const GroupPass* __restrict__ jobs, int njobs) {
    const long long b = blockIdx.x;
    int lo = 0, hi = njobs - 1;   // the last job starting at or before b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].first <= b) lo = mid;
        else hi = mid - 1;
    }
    const GroupPass& g = jobs[lo];
    const long long local = b - g.first;
    pass_body<P, T, TI, SGN, KM>(g.a, local % g.ntile, local / g.ntile);
}

// ---------------------------------------------------------------------------
// fused top pass of the interpolation: forward stages of the last digits,
// scale p^-m, weight, per-class variance partials, optional coefficient store,
// inverse stages of the same digits.
struct MidArgs {
    PassArgs pa;
    const float* W;        // NULL: weight 1
    const uint8_t* cls;    // [N][2]
    void* coef;            // optional output of g
    double* part;          // [fn][ntile][2*nb]
    long long ntile;
    int nb;                // s + 1
};

template <typename T> __device__ __forceinline__ float mag2(T v);
template <> __device__ __forceinline__ float mag2<float>(float v) { return v * v; }
template <> __device__ __forceinline__ float mag2<float2>(float2 v) { return v.x * v.x + v.y * v.y; }
template <typename T> __device__ __forceinline__ T mulw(T v, float w);
template <> __device__ __forceinline__ float mulw<float>(float v, float w) { return v * w; }
template <> __device__ __forceinline__ float2 mulw<float2>(float2 v, float w) { return make_float2(v.x * w, v.y * w); }

// per-lane FP32 class sums of the first nwb warps -> one FP64 value per class
// and tile, fixed order
__device__ __forceinline__ void reduce_bins(const float* bins, int nb2, int nwb, double* out, long long stride) {
    const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int bi = w; bi < nb2; bi += nw) {
        float x = 0.f;
        for (int ww = 0; ww < nwb; ++ww) x += bins[(ww * nb2 + bi) * 32 + lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) out[bi * stride] = (double)x;
    }
}

// The fused top pass in register groups (as k_pass): forward groups from the
// top digits down, the last one leaving the tile in shared memory; the scale,
// weight, optional coefficient store and class partials (per-lane FP32 bins of
// the first nwb warps, a fixed summation order) element by element; then the
// inverse groups, the last one writing global memory as in k_pass.
template <int P, typename T, typename TI, int KM>
__global__ void __maxnreg__(96) k_mid(MidArgs m, int nwb) {
    const PassArgs& a = m.pa;
    extern __shared__ __align__(16) unsigned char smraw[];
    T* sm = reinterpret_cast<T*>(smraw);
    const int nel = a.R << a.wlog;
    const int tile_elems = nel + ((nel - 1) >> PadLog<T>::v);   // as spad_bytes on the host
    float* bins = reinterpret_cast<float*>(smraw + ((tile_elems * sizeof(T) + 15) & ~(size_t)15));
    const int nb2 = 2 * m.nb;
    const long long fn = blockIdx.y;
    const long long tile = blockIdx.x;
    const long long lo0 = (tile % a.nlo) << a.wlog;
    const long long base = lo0 + (tile / a.nlo) * a.SR;
    const int ncols = (int)min((long long)a.Wc, a.S - lo0);
    const int cmask = a.Wc - 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const TI* in = reinterpret_cast<const TI*>(a.in) + fn * a.ld_in + base;
    T* out = reinterpret_cast<T*>(a.out) + fn * a.ld_out + base;
    for (int i = threadIdx.x; i < nwb * nb2 * 32; i += blockDim.x) bins[i] = 0.f;
    const int b = a.b;
    const int k0 = min(KM, b);
    const int g_last = b == k0 ? 0 : ((b - k0 - 1) / KM) * KM;
    long long run = 1;
    if (a.S == 1) {
        for (int i = 0; i < g_last; ++i) run *= P;
    } else {
        run = a.Wc;
    }
    const bool direct_out = run * (long long)sizeof(T) >= 64;
    // forward stages
    {
        int g0 = b - k0, k = k0;
        for (;;) {
            const bool first = g0 + k == b;
            rgroup_k<P, -1, T, TI, KM>(k, first ? 1 : 4, sm, in, out, g0, a, ncols);
            __syncthreads();
            if (g0 == g_last) break;
            g0 = first ? 0 : g0 + k;
            k = min(KM, b - k0 - g0);
        }
    }
    // scale, weight, coefficients, class partials; the weight and class loads
    // of 8 elements per thread are issued together
    if (w < nwb) {
        float* mybins = bins + (size_t)w * nb2 * 32 + lane;
        T* coef = m.coef ? reinterpret_cast<T*>(m.coef) + fn * a.ld_out + base : nullptr;
        const int step = nwb * 32;
        for (int e0 = threadIdx.x; e0 < nel; e0 += 8 * step) {
            float wv[8];
            uchar2 kc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int e = e0 + j * step;
                const int r = e >> a.wlog, c = e & cmask;
                const long long H = base + c + (long long)r * a.S;
                const bool ok = e < nel && c < ncols;
                wv[j] = ok && m.W ? __ldg(m.W + H) : 1.f;
                kc[j] = ok ? __ldg(reinterpret_cast<const uchar2*>(m.cls) + H) : make_uchar2(0, 0);
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int e = e0 + j * step;
                const int r = e >> a.wlog, c = e & cmask;
                if (e >= nel || c >= ncols) continue;
                const long long H = base + c + (long long)r * a.S;
                T v = mulw<T>(scale_by<T>(sm[sx<P, T>(e)], a.scale), wv[j]);
                if (coef) coef[c + (long long)r * a.S] = v;
                if (H != 0) {
                    const float q = mag2<T>(v);
                    mybins[(int)kc[j].x * 32] += q;
                    mybins[(m.nb + (int)kc[j].y) * 32] += q;
                }
                sm[sx<P, T>(e)] = v;
            }
        }
    }
    __syncthreads();
    reduce_bins(bins, nb2, nwb, m.part + fn * nb2 * m.ntile + tile, m.ntile);
    // inverse stages of the same digits, in the same order
    {
        int g0 = b - k0, k = k0;
        for (;;) {
            const bool last = g0 == g_last;
            const bool dst_g = last && direct_out;
            rgroup_k<P, +1, T, T, KM>(k, dst_g ? 2 : 4, sm, out, out, g0, a, ncols);
            if (!dst_g) __syncthreads();
            if (last) break;
            g0 = g0 + k == b ? 0 : g0 + k;
            k = min(KM, b - k0 - g0);
        }
    }
    if (!direct_out) {
        for (int e = threadIdx.x; e < nel; e += blockDim.x) {
            const int r = e >> a.wlog, c = e & cmask;
            if (c < ncols) out[c + (long long)r * a.S] = sm[sx<P, T>(e)];
        }
    }
}

// class sums of given coefficients: grid (chunks, functions), 8192 elements per chunk
template <typename T>
__global__ void __launch_bounds__(256) k_effdim_bins(const T* coef, long long ld, long long N, const uint8_t* cls,
                                                     int nb, long long nchunk, double* part) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float* bins = reinterpret_cast<float*>(smraw);
    const int nb2 = 2 * nb, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < (int)(blockDim.x >> 5) * nb2 * 32; i += blockDim.x) bins[i] = 0.f;
    __syncthreads();
    const long long fn = blockIdx.y, chunk = blockIdx.x;
    const long long h0 = chunk * 8192, h1 = min(N, h0 + 8192);
    float* mybins = bins + (size_t)w * nb2 * 32 + lane;
    const T* g = coef + fn * ld;
    for (long long H = h0 + threadIdx.x; H < h1; H += blockDim.x) {
        if (H == 0) continue;
        const float q = mag2<T>(g[H]);
        const uchar2 k = __ldg(reinterpret_cast<const uchar2*>(cls) + H);
        mybins[(int)k.x * 32] += q;
        mybins[(nb + (int)k.y) * 32] += q;
    }
    __syncthreads();
    reduce_bins(bins, nb2, blockDim.x >> 5, part + fn * nb2 * nchunk + chunk, nchunk);
}

// partials part[fn][class][tile] -> per-class totals: one block per (class,
// function); thread t sums tiles t, t+256, ... in order, then a fixed tree.
__global__ void __launch_bounds__(256) k_effdim_classes(const double* __restrict__ part, long long nchunk, int nb2,
                                                        double* csum) {
    __shared__ double red[256];
    const int bi = blockIdx.x;
    const long long fn = blockIdx.y;
    const double* pp = part + (fn * nb2 + bi) * nchunk;
    double acc = 0.0;
    long long t = threadIdx.x;
    for (; t + 3 * 256 < nchunk; t += 4 * 256) {   // four loads in flight, added in order
        const double a0 = pp[t], a1 = pp[t + 256], a2 = pp[t + 512], a3 = pp[t + 768];
        acc += a0;
        acc += a1;
        acc += a2;
        acc += a3;
    }
    for (; t < nchunk; t += 256) acc += pp[t];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) csum[fn * nb2 + bi] = red[0];
}

// per-class totals -> cumulative truncation / superposition variances and dimensions
__global__ void __launch_bounds__(32) k_effdim_finalize(const double* __restrict__ csum, int nb, double thr, EffOut o,
                                                         int batch) {
    // one warp per function: the class totals come into shared memory together,
    // then lane 0 forms the cumulative sums in class order
    __shared__ double c[2 * 256];
    const int fn = blockIdx.x;
    if (fn >= batch) return;
    const double* cs_ = csum + (long long)fn * 2 * nb;
    for (int i = threadIdx.x; i < 2 * nb; i += 32) c[i] = cs_[i];
    __syncwarp();
    if (threadIdx.x != 0) return;
    double tot = 0.0;
    for (int d = 0; d < nb; ++d) tot += c[d];
    double ct = 0.0, cs = 0.0;
    int dt = 0, ds = 0;
    bool ft = false, fs = false;
    for (int d = 0; d < nb; ++d) {
        ct += c[d];
        cs += c[nb + d];
        if (o.vt) o.vt[(long long)fn * o.vstride + d] = ct;
        if (o.vs) o.vs[(long long)fn * o.vstride + d] = cs;
        if (tot > 0.0) {
            if (!ft && ct >= thr * tot) { dt = d; ft = true; }
            if (!fs && cs >= thr * tot) { ds = d; fs = true; }
        }
    }
    if (o.dt) o.dt[(long long)fn * o.dstride] = dt;
    if (o.ds) o.ds[(long long)fn * o.dstride] = ds;
}

// ---------------------------------------------------------------------------
// host side
static Tw make_tw(int p) {
    Tw t;
    for (int e = 0; e < 32; ++e) {
        double ang = e < p ? 2.0 * 3.14159265358979323846 * e / p : 0.0;
        t.cd[e] = cos(ang);
        t.sd[e] = sin(ang);
        if (e == 0) { t.cd[e] = 1.0; t.sd[e] = 0.0; }
        t.c[e] = (float)t.cd[e];
        t.s[e] = (float)t.sd[e];
    }
    return t;
}

template <typename F>
static int set_smem(F* kern, size_t bytes) {
    (void)bytes;
    return smem_limit_max(kern);
}

static PassArgs pass_args(const PassGeom& g, const void* in, void* out, long long ld_in, long long ld_out,
                          const Tw& tw) {
    PassArgs a;
    a.in = in;
    a.out = out;
    a.ld_in = ld_in;
    a.ld_out = ld_out;
    a.S = g.S;
    a.SR = g.S * g.R;
    a.nlo = g.nlo;
    a.R = g.R;
    a.b = g.b;
    a.Wc = g.Wc;
    a.wlog = g.wlog;
    a.scale = 1.0;
    a.do_scale = 0;
    a.tw = tw;
    return a;
}

static const char* pass_family(int t, int q) { return t == 0 ? "pass_lo" : (t == q - 1 ? "pass_hi" : "pass_mid"); }

// threads of a pass: one per task of its first (top) group, 32 .. 512
template <int P, int KM>
static int pass_threads(const PassGeom& g) {
    const int k0 = std::min(KM, g.b);
    long long tasks = ((long long)g.R / ipow_ll(P, k0)) << g.wlog;
    tasks = (tasks + 31) / 32 * 32;
    return (int)std::min(pass_max_threads<P>(), std::max(32ll, tasks));
}

template <int P, typename T, typename TI, int SGN, int KM>
static int launch_pass_k(const PassGeom& g, const PassArgs& a, int nf, const char* fam, cudaStream_t st) {
    const size_t smem = spad_bytes<T>(g.R << g.wlog);
    auto kern = k_pass<P, T, TI, SGN, KM>;
    int rc = set_smem(kern, smem);
    if (rc) return rc;
    dim3 grid((unsigned)g.ntile, (unsigned)nf);
    {
        LaunchScope ls(fam, st);
        kern<<<grid, pass_threads<P, KM>(g), smem, st>>>(a);
    }
    DWT_CK_LAUNCH("k_pass");
    return DWT_OK;
}

template <int P, typename T, typename TI, int SGN>
static int launch_pass(const PassGeom& g, const PassArgs& a, int nf, const char* fam, cudaStream_t st) {
    return launch_pass_k<P, T, TI, SGN, KMax<P, T>::v>(g, a, nf, fam, st);
}

// L2-sized groups of functions: the passes of one group run back to back so
// that the intermediate stays in the 126 MB L2 between passes.
static const long long kL2Group = 48ll << 20;

template <int P, typename T, typename TI, int SGN>
static int transform_pp(dwt_plan_s* Pl, const PassPlan& pp, double scale_by_n, const void* in, void* out, int batch,
                        long long ld_in, long long ld_out, cudaStream_t st);

template <int P, typename T, typename TI, int SGN>
static int transform_t(dwt_plan_s* Pl, const void* in, void* out, int batch, long long ld_in, long long ld_out,
                       cudaStream_t st) {
    return transform_pp<P, T, TI, SGN>(Pl, pass_plan(Pl, sizeof(T)), 1.0 / (double)Pl->N, in, out, batch, ld_in,
                                       ld_out, st);
}

// The passes of pp over a batch; a forward (SGN < 0, not int32) scales by
// scale_by_n in its last pass.
template <int P, typename T, typename TI, int SGN>
static int transform_pp(dwt_plan_s* Pl, const PassPlan& pp, double scale_by_n, const void* in, void* out, int batch,
                        long long ld_in, long long ld_out, cudaStream_t st) {
    const Tw tw = make_tw(P);
    const long long fbytes = Pl->N * (long long)sizeof(T);
    int G = (int)std::max(1ll, (Pl->tuned_group_bytes > 0 ? Pl->tuned_group_bytes : kL2Group) / fbytes);
    G = std::min(G, 65535);
    const bool scale = SGN < 0 && !std::is_same<T, int>::value;
    for (int f0 = 0; f0 < batch; f0 += G) {
        const int nf = std::min(G, batch - f0);
        for (int t = 0; t < pp.q; ++t) {
            const PassGeom& g = pp.g[t];
            int rc;
            if (t == 0) {
                PassArgs a = pass_args(g, (const TI*)in + (long long)f0 * ld_in, (T*)out + (long long)f0 * ld_out,
                                       ld_in, ld_out, tw);
                if (scale && pp.q == 1) { a.do_scale = 1; a.scale = scale_by_n; }
                rc = launch_pass<P, T, TI, SGN>(g, a, nf, pass_family(t, pp.q), st);
            } else {
                PassArgs a = pass_args(g, (const T*)out + (long long)f0 * ld_out, (T*)out + (long long)f0 * ld_out,
                                       ld_out, ld_out, tw);
                if (scale && t == pp.q - 1) { a.do_scale = 1; a.scale = scale_by_n; }
                rc = launch_pass<P, T, T, SGN>(g, a, nf, pass_family(t, pp.q), st);
            }
            if (rc) return rc;
        }
    }
    return DWT_OK;
}

template <int P>
static int transform_p(dwt_plan_s* Pl, const void* in, void* out, int batch, long long ld_in, long long ld_out,
                       dwt_dtype in_t, dwt_dtype out_t, int sgn, cudaStream_t st) {
    if constexpr (P == 2) {
        if (in_t == DWT_F32)
            return sgn < 0 ? transform_t<2, float, float, -1>(Pl, in, out, batch, ld_in, ld_out, st)
                           : transform_t<2, float, float, +1>(Pl, in, out, batch, ld_in, ld_out, st);
        if (in_t == DWT_F64)
            return sgn < 0 ? transform_t<2, double, double, -1>(Pl, in, out, batch, ld_in, ld_out, st)
                           : transform_t<2, double, double, +1>(Pl, in, out, batch, ld_in, ld_out, st);
        return sgn < 0 ? transform_t<2, int, int, -1>(Pl, in, out, batch, ld_in, ld_out, st)
                       : transform_t<2, int, int, +1>(Pl, in, out, batch, ld_in, ld_out, st);
    } else {
        if (out_t == DWT_C64) {
            if (sgn < 0)
                return in_t == DWT_F32 ? transform_t<P, float2, float, -1>(Pl, in, out, batch, ld_in, ld_out, st)
                                       : transform_t<P, float2, float2, -1>(Pl, in, out, batch, ld_in, ld_out, st);
            return transform_t<P, float2, float2, +1>(Pl, in, out, batch, ld_in, ld_out, st);
        }
        if (sgn < 0)
            return in_t == DWT_F64 ? transform_t<P, double2, double, -1>(Pl, in, out, batch, ld_in, ld_out, st)
                                   : transform_t<P, double2, double2, -1>(Pl, in, out, batch, ld_in, ld_out, st);
        return transform_t<P, double2, double2, +1>(Pl, in, out, batch, ld_in, ld_out, st);
    }
}

// Stages of the digits d0 .. d0+nd-1 (generic passes), forward scaled by p^-nd.
template <int P>
static int digits_p(dwt_plan_s* Pl, const void* in, void* out, int batch, long long ld_in, long long ld_out,
                    dwt_dtype in_t, dwt_dtype out_t, int d0, int nd, int sgn, cudaStream_t st) {
    auto go = [&](auto tag_t, auto tag_i, auto sgn_c) {
        using T = decltype(tag_t);
        using TI = decltype(tag_i);
        constexpr int SG = decltype(sgn_c)::value;
        PassPlan pp;
        pass_plan_range(P, Pl->m, (int)sizeof(T), d0, nd, Pl->min_tiles, pp);
        return transform_pp<P, T, TI, SG>(Pl, pp, 1.0 / (double)ipow_ll(P, nd), in, out, batch, ld_in, ld_out, st);
    };
    using M = std::integral_constant<int, -1>;
    using Pp = std::integral_constant<int, +1>;
    if constexpr (P == 2) {
        if (in_t == DWT_F32) return sgn < 0 ? go(float(), float(), M()) : go(float(), float(), Pp());
        if (in_t == DWT_F64) return sgn < 0 ? go(double(), double(), M()) : go(double(), double(), Pp());
        return sgn < 0 ? go(int(), int(), M()) : go(int(), int(), Pp());
    } else {
        if (out_t == DWT_C64) {
            if (sgn < 0) return in_t == DWT_F32 ? go(float2(), float(), M()) : go(float2(), float2(), M());
            return go(float2(), float2(), Pp());
        }
        if (sgn < 0) return in_t == DWT_F64 ? go(double2(), double(), M()) : go(double2(), double2(), M());
        return go(double2(), double2(), Pp());
    }
}

int run_transform_digits(dwt_plan_s* Pl, const void* in, void* out, int batch, long long ld_in, long long ld_out,
                         dwt_dtype in_t, dwt_dtype out_t, int d0, int nd, int sgn, cudaStream_t st) {
    switch (Pl->p) {
        case 2: return digits_p<2>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, sgn, st);
        case 3: return digits_p<3>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, sgn, st);
        case 5: return digits_p<5>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, sgn, st);
        case 7: return digits_p<7>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, sgn, st);
        case 11: return digits_p<11>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, sgn, st);
        case 13: return digits_p<13>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, sgn, st);
        case 17: return digits_p<17>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, sgn, st);
        case 19: return digits_p<19>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, sgn, st);
        case 23: return digits_p<23>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, sgn, st);
        case 29: return digits_p<29>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, sgn, st);
        case 31: return digits_p<31>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, sgn, st);
        default: set_error("unsupported p"); return DWT_EUNSUPPORTED;
    }
}

// ---------------------------------------------------------------------------
// grouped transforms: pass t of every job in one launch of k_pass_grouped

template <int P, typename T, typename TI, int SGN>
static int launch_grouped(const std::vector<GroupPass>& h, long long blocks, int threads, size_t smem, const char* fam,
                          cudaStream_t st) {
    if (h.empty()) return DWT_OK;
    if (blocks > 0x7fffffffll) {
        set_error("grouped pass: %lld blocks exceed one launch", blocks);
        return DWT_EINVAL;
    }
    constexpr int KM = KMax<P, T>::v;
    auto kern = k_pass_grouped<P, T, TI, SGN, KM>;
    int rc = set_smem(kern, smem);
    if (rc) return rc;
    GroupPass* d = nullptr;
    if (dmalloc((void**)&d, sizeof(GroupPass) * h.size(), st)) return DWT_ENOMEM;
    DWT_CK(cudaMemcpyAsync(d, h.data(), sizeof(GroupPass) * h.size(), cudaMemcpyHostToDevice, st));
    {
        LaunchScope ls(fam, st);
        kern<<<(unsigned)blocks, threads, smem, st>>>(d, (int)h.size());
    }
    dfree(d, st);
    DWT_CK_LAUNCH("k_pass_grouped");
    return DWT_OK;
}

// The jobs' transforms by their plans' pass plans, pass t of all jobs in one
// launch; the same tile body, geometry and scaling as transform_pp, so every
// element equals the one of the job's own call.
template <int P, typename T, typename TI, int SGN>
static int grouped_t(const std::vector<GroupJob>& js, cudaStream_t st) {
    const Tw tw = make_tw(P);
    const bool scale = SGN < 0 && !std::is_same<T, int>::value;
    constexpr int KM = KMax<P, T>::v;
    std::vector<const PassPlan*> pps;
    int qmax = 0;
    for (const GroupJob& j : js) {
        pps.push_back(&pass_plan(j.plan, sizeof(T)));
        qmax = std::max(qmax, pps.back()->q);
    }
    for (int t = 0; t < qmax; ++t) {
        std::vector<GroupPass> h;
        long long blocks = 0;
        int threads = 32;
        size_t smem = 0;
        for (size_t i = 0; i < js.size(); ++i) {
            const PassPlan& pp = *pps[i];
            const GroupJob& j = js[i];
            if (t >= pp.q || j.batch <= 0) continue;
            const PassGeom& g = pp.g[t];
            GroupPass gp;
            if (t == 0) {
                gp.a = pass_args(g, j.in, j.out, j.ld_in, j.ld_out, tw);
                if (scale && pp.q == 1) {
                    gp.a.do_scale = 1;
                    gp.a.scale = 1.0 / (double)j.plan->N;
                }
            } else {
                gp.a = pass_args(g, j.out, j.out, j.ld_out, j.ld_out, tw);
                if (scale && t == pp.q - 1) {
                    gp.a.do_scale = 1;
                    gp.a.scale = 1.0 / (double)j.plan->N;
                }
            }
            gp.ntile = g.ntile;
            gp.first = blocks;
            blocks += g.ntile * (long long)j.batch;
            h.push_back(gp);
            threads = std::max(threads, pass_threads<P, KM>(g));
            smem = std::max(smem, spad_bytes<T>(g.R << g.wlog));
        }
        const int rc = t == 0 ? launch_grouped<P, T, TI, SGN>(h, blocks, threads, smem, "grouped_pass", st)
                              : launch_grouped<P, T, T, SGN>(h, blocks, threads, smem, "grouped_pass", st);
        if (rc) return rc;
    }
    return DWT_OK;
}

template <int P>
static int grouped_p(const std::vector<GroupJob>& js, dwt_dtype in_t, dwt_dtype out_t, int sgn, cudaStream_t st) {
    if constexpr (P == 2) {
        if (in_t == DWT_F32)
            return sgn < 0 ? grouped_t<2, float, float, -1>(js, st) : grouped_t<2, float, float, +1>(js, st);
        if (in_t == DWT_F64)
            return sgn < 0 ? grouped_t<2, double, double, -1>(js, st) : grouped_t<2, double, double, +1>(js, st);
        return sgn < 0 ? grouped_t<2, int, int, -1>(js, st) : grouped_t<2, int, int, +1>(js, st);
    } else {
        if (out_t == DWT_C64) {
            if (sgn < 0)
                return in_t == DWT_F32 ? grouped_t<P, float2, float, -1>(js, st)
                                       : grouped_t<P, float2, float2, -1>(js, st);
            return grouped_t<P, float2, float2, +1>(js, st);
        }
        if (sgn < 0)
            return in_t == DWT_F64 ? grouped_t<P, double2, double, -1>(js, st)
                                   : grouped_t<P, double2, double2, -1>(js, st);
        return grouped_t<P, double2, double2, +1>(js, st);
    }
}

// Grouped transforms of jobs that share p and the element types (checked by
// the caller).  p = 2 jobs that their own call sends to the register-tile
// kernels go there too: m = 12 .. 14 as one grouped low pass per tile size,
// larger ones one call each; all other jobs run the generic passes grouped.
int run_transform_grouped(const std::vector<GroupJob>& jobs, dwt_dtype in_t, dwt_dtype out_t, int sgn,
                          cudaStream_t st) {
    if (jobs.empty()) return DWT_OK;
    const int p = jobs[0].plan->p;
    std::vector<GroupJob> generic, lo[3];
    for (const GroupJob& j : jobs) {
        if (j.batch <= 0) continue;
        if (p == 2 && (in_t == DWT_F32 || in_t == DWT_I32) && p2_fast_ok(j.plan->m) && aligned16(j.in, j.ld_in, 4) &&
            aligned16(j.out, j.ld_out, 4)) {
            if (j.plan->m <= 14) {
                lo[j.plan->m - 12].push_back(j);
            } else {
                const int rc = p2_transform(j.plan, j.in, j.out, j.batch, j.ld_in, j.ld_out, in_t, sgn, st);
                if (rc) return rc;
            }
            continue;
        }
        generic.push_back(j);
    }
    for (int L = 12; L <= 14; ++L)
        if (!lo[L - 12].empty()) {
            const int rc = p2_lo_grouped(L, lo[L - 12], in_t, sgn, st);
            if (rc) return rc;
        }
    if (generic.empty()) return DWT_OK;
    switch (p) {
        case 2: return grouped_p<2>(generic, in_t, out_t, sgn, st);
        case 3: return grouped_p<3>(generic, in_t, out_t, sgn, st);
        case 5: return grouped_p<5>(generic, in_t, out_t, sgn, st);
        case 7: return grouped_p<7>(generic, in_t, out_t, sgn, st);
        case 11: return grouped_p<11>(generic, in_t, out_t, sgn, st);
        case 13: return grouped_p<13>(generic, in_t, out_t, sgn, st);
        case 17: return grouped_p<17>(generic, in_t, out_t, sgn, st);
        case 19: return grouped_p<19>(generic, in_t, out_t, sgn, st);
        case 23: return grouped_p<23>(generic, in_t, out_t, sgn, st);
        case 29: return grouped_p<29>(generic, in_t, out_t, sgn, st);
        case 31: return grouped_p<31>(generic, in_t, out_t, sgn, st);
        default: set_error("unsupported p"); return DWT_EUNSUPPORTED;
    }
}

int run_transform(dwt_plan_s* Pl, const void* in, void* out, int batch, long long ld_in, long long ld_out,
                  dwt_dtype in_t, dwt_dtype out_t, int sgn, cudaStream_t st) {
    if (Pl->p == 2 && (in_t == DWT_F32 || in_t == DWT_I32) && p2_fast_ok(Pl->m) && aligned16(in, ld_in, 4) &&
        aligned16(out, ld_out, 4))
        return p2_transform(Pl, in, out, batch, ld_in, ld_out, in_t, sgn, st);
    switch (Pl->p) {
        case 2: return transform_p<2>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, sgn, st);
        case 3: return transform_p<3>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, sgn, st);
        case 5: return transform_p<5>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, sgn, st);
        case 7: return transform_p<7>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, sgn, st);
        case 11: return transform_p<11>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, sgn, st);
        case 13: return transform_p<13>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, sgn, st);
        case 17: return transform_p<17>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, sgn, st);
        case 19: return transform_p<19>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, sgn, st);
        case 23: return transform_p<23>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, sgn, st);
        case 29: return transform_p<29>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, sgn, st);
        case 31: return transform_p<31>(Pl, in, out, batch, ld_in, ld_out, in_t, out_t, sgn, st);
        default: set_error("unsupported p"); return DWT_EUNSUPPORTED;
    }
}

// ---------------------------------------------------------------------------
// warps that keep class bins next to a tile: up to maxw within `budget` bytes
// of bins (at least one while it fits beside the tile)
static int bins_warps(size_t tile_bytes, int nb2, size_t budget = 227 * 1024, int maxw = 8) {
    const size_t avail = 227 * 1024 - ((tile_bytes + 15) & ~(size_t)15);
    const size_t per_warp = (size_t)nb2 * 32 * 4;
    if (per_warp > avail) return 0;
    return (int)std::max<size_t>(1, std::min<size_t>(maxw, std::min(avail, budget) / per_warp));
}

static int finalize(dwt_plan_s* Pl, const double* part, long long nchunk, int batch, double thr, const EffOut& o,
                    cudaStream_t st) {
    if (!o.vt && !o.vs && !o.dt && !o.ds) return DWT_OK;
    const int nb = Pl->s + 1, nb2 = 2 * nb;
    // per-class totals go right after the partials in the workspace
    double* csum = const_cast<double*>(part) + (size_t)batch * nb2 * nchunk;
    for (int f0 = 0; f0 < batch; f0 += 65535) {
        const int nf = std::min(65535, batch - f0);
        LaunchScope ls("effdim_classes", st);
        k_effdim_classes<<<dim3((unsigned)nb2, (unsigned)nf), 256, 0, st>>>(part + (size_t)f0 * nb2 * nchunk, nchunk,
                                                                            nb2, csum + (size_t)f0 * nb2);
    }
    DWT_CK_LAUNCH("k_effdim_classes");
    {
        LaunchScope ls("effdim_finalize", st);
        k_effdim_finalize<<<batch, 32, 0, st>>>(csum, nb, thr, o, batch);
    }
    DWT_CK_LAUNCH("k_effdim_finalize");
    return DWT_OK;
}

template <int P, typename T, typename TI>
static int interpolate_t(dwt_plan_s* Pl, const void* f, void* c, void* coef, int batch, long long ld,
                         dwt_weight weight, double* var, int* dim, double thr, cudaStream_t st) {
    const PassPlan& pp = pass_plan(Pl, sizeof(T));
    const Tw tw = make_tw(P);
    const int nb = Pl->s + 1, nb2 = 2 * nb;
    const PassGeom& gm = pp.g[pp.q - 1];
    const long long ntile = gm.ntile;
    constexpr int KM = KMax<P, T>::v;
    const size_t tile_bytes = spad_bytes<T>(gm.R << gm.wlog);
    const int nt = pass_threads<P, KM>(gm);
    // warps that bin: their bins within 48 KB, so that the tile and its bins
    // leave room for a second CTA
    const int nw = std::min(nt / 32, bins_warps(tile_bytes, nb2, 48 * 1024, 16));
    if (nw < 1) {
        set_error("s = %d too large for the fused variance pass", Pl->s);
        return DWT_EUNSUPPORTED;
    }
    const size_t smem = ((tile_bytes + 15) & ~(size_t)15) + (size_t)nw * nb2 * 32 * 4;
    int rc = ensure_workspace(Pl, (size_t)batch * (ntile + 1) * nb2 * sizeof(double), st);
    if (rc) return rc;
    double* part = (double*)Pl->d_ws;
    auto kmid_first = k_mid<P, T, TI, KM>;   // single pass: reads f directly
    auto kmid_next = k_mid<P, T, T, KM>;     // after lower passes: in place on c
    rc = set_smem(kmid_first, smem);
    if (rc) return rc;
    rc = set_smem(kmid_next, smem);
    if (rc) return rc;
    const long long fbytes = Pl->N * (long long)sizeof(T);
    int G = (int)std::max(1ll, kL2Group / fbytes);
    G = std::min(G, 65535);
    for (int f0 = 0; f0 < batch; f0 += G) {
        const int nf = std::min(G, batch - f0);
        const long long off = (long long)f0 * ld;
        // forward passes below the top one: f -> c
        for (int t = 0; t + 1 < pp.q; ++t) {
            const PassGeom& g = pp.g[t];
            if (t == 0) {
                PassArgs a = pass_args(g, (const TI*)f + off, (T*)c + off, ld, ld, tw);
                rc = launch_pass<P, T, TI, -1>(g, a, nf, "interp_fwd", st);
            } else {
                PassArgs a = pass_args(g, (const T*)c + off, (T*)c + off, ld, ld, tw);
                rc = launch_pass<P, T, T, -1>(g, a, nf, "interp_fwd", st);
            }
            if (rc) return rc;
        }
        // fused top pass
        MidArgs m;
        if (pp.q == 1) m.pa = pass_args(gm, (const TI*)f + off, (T*)c + off, ld, ld, tw);
        else m.pa = pass_args(gm, (const T*)c + off, (T*)c + off, ld, ld, tw);
        m.pa.scale = 1.0 / (double)Pl->N;
        m.W = weight == DWT_WEIGHT_INV_SQ_WAVENUMBER ? Pl->d_W : nullptr;
        m.cls = Pl->d_cls;
        m.coef = coef ? (void*)((T*)coef + off) : nullptr;
        m.part = part + (long long)f0 * ntile * nb2;   // [fn][class][tile] of this group
        m.ntile = ntile;
        m.nb = nb;
        {
            LaunchScope ls("interp_top", st);
            dim3 grid((unsigned)ntile, (unsigned)nf);
            if (pp.q == 1) kmid_first<<<grid, nt, smem, st>>>(m, nw);
            else kmid_next<<<grid, nt, smem, st>>>(m, nw);
        }
        DWT_CK_LAUNCH("k_mid");
        // inverse passes below the top one, in place on c
        for (int t = pp.q - 2; t >= 0; --t) {
            const PassGeom& g = pp.g[t];
            PassArgs a = pass_args(g, (const T*)c + off, (T*)c + off, ld, ld, tw);
            rc = launch_pass<P, T, T, +1>(g, a, nf, "interp_inv", st);
            if (rc) return rc;
        }
    }
    return finalize(Pl, part, ntile, batch, thr, eff_packed(var, dim, nb), st);
}

int run_interpolate(dwt_plan_s* Pl, const void* f, void* c, void* coef, int batch, long long ld, dwt_dtype f_t,
                    dwt_weight weight, dwt_algo algo, double* var, int* dim, double thr, cudaStream_t st) {
    const bool fast = Pl->p == 2 && p2_interp_ok(Pl->m, Pl->s) && aligned16(f, ld, 4) && aligned16(c, ld, 4);
    if (algo == DWT_ALGO_TC_SPLIT_BF16 && !(fast && Pl->m >= 18)) {
        set_error("the tensor-core interpolation needs p = 2, 18 <= m <= 24 and 16-byte aligned rows");
        return DWT_EUNSUPPORTED;
    }
    if (fast && Pl->d_tkt) {
        double* part = nullptr;
        long long ntile = 0;
        int rc = p2i_interpolate(Pl, (const float*)f, (float*)c, (float*)coef, batch, ld,
                                 weight == DWT_WEIGHT_INV_SQ_WAVENUMBER, algo == DWT_ALGO_TC_SPLIT_BF16, &part, &ntile,
                                 st);
        if (rc) return rc;
        return finalize(Pl, part, ntile, batch, thr, eff_packed(var, dim, Pl->s + 1), st);
    }
    if (fast) {
        double* part = nullptr;
        long long ntile = 0;
        int rc = p2_interpolate(Pl, (const float*)f, (float*)c, (float*)coef, batch, ld,
                                weight == DWT_WEIGHT_INV_SQ_WAVENUMBER ? Pl->d_W : nullptr,
                                algo == DWT_ALGO_TC_SPLIT_BF16, &part, &ntile, st);
        if (rc) return rc;
        return finalize(Pl, part, ntile, batch, thr, eff_packed(var, dim, Pl->s + 1), st);
    }
    switch (Pl->p) {
        case 2: return interpolate_t<2, float, float>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st);
        case 3:
            return f_t == DWT_F32 ? interpolate_t<3, float2, float>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st)
                                  : interpolate_t<3, float2, float2>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st);
        case 5:
            return f_t == DWT_F32 ? interpolate_t<5, float2, float>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st)
                                  : interpolate_t<5, float2, float2>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st);
        case 7:
            return f_t == DWT_F32 ? interpolate_t<7, float2, float>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st)
                                  : interpolate_t<7, float2, float2>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st);
        case 11:
            return f_t == DWT_F32 ? interpolate_t<11, float2, float>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st)
                                  : interpolate_t<11, float2, float2>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st);
        case 13:
            return f_t == DWT_F32 ? interpolate_t<13, float2, float>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st)
                                  : interpolate_t<13, float2, float2>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st);
        case 17:
            return f_t == DWT_F32 ? interpolate_t<17, float2, float>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st)
                                  : interpolate_t<17, float2, float2>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st);
        case 19:
            return f_t == DWT_F32 ? interpolate_t<19, float2, float>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st)
                                  : interpolate_t<19, float2, float2>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st);
        case 23:
            return f_t == DWT_F32 ? interpolate_t<23, float2, float>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st)
                                  : interpolate_t<23, float2, float2>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st);
        case 29:
            return f_t == DWT_F32 ? interpolate_t<29, float2, float>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st)
                                  : interpolate_t<29, float2, float2>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st);
        case 31:
            return f_t == DWT_F32 ? interpolate_t<31, float2, float>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st)
                                  : interpolate_t<31, float2, float2>(Pl, f, c, coef, batch, ld, weight, var, dim, thr, st);
        default: set_error("unsupported p"); return DWT_EUNSUPPORTED;
    }
}

template <typename T>
static int effdim_t(dwt_plan_s* Pl, const void* coef, int batch, long long ld, const EffOut& o, double thr,
                    cudaStream_t st) {
    const int nb = Pl->s + 1, nb2 = 2 * nb;
    const long long nchunk = (Pl->N + 8191) / 8192;
    const int nw = bins_warps(0, nb2);
    if (nw < 1) {
        set_error("s = %d too large for the variance pass", Pl->s);
        return DWT_EUNSUPPORTED;
    }
    const size_t smem = (size_t)nw * nb2 * 32 * 4;
    int rc = ensure_workspace(Pl, (size_t)batch * (nchunk + 1) * nb2 * sizeof(double), st);
    if (rc) return rc;
    double* part = (double*)Pl->d_ws;
    auto kern = k_effdim_bins<T>;
    rc = set_smem(kern, smem);
    if (rc) return rc;
    for (int f0 = 0; f0 < batch; f0 += 65535) {
        const int nf = std::min(65535, batch - f0);
        LaunchScope ls("effdim_bins", st);
        kern<<<dim3((unsigned)nchunk, (unsigned)nf), nw * 32, smem, st>>>(
            (const T*)coef + (long long)f0 * ld, ld, Pl->N, Pl->d_cls, nb, nchunk, part + (long long)f0 * nchunk * nb2);
    }
    DWT_CK_LAUNCH("k_effdim_bins");
    return finalize(Pl, part, nchunk, batch, thr, o, st);
}

// The class sums of effdim_t, with the partials and totals in a scratch array
// supplied by the caller (cap doubles) instead of the plan's workspace:
// functions go through in groups whose partials fit, one group after another
// on the stream, so the array is reused in stream order.  Makes no allocation.
template <typename T>
static int effdim_scratch_t(dwt_plan_s* Pl, const void* coef, int batch, long long ld, double* var, int* dim,
                            double thr, double* scratch, long long cap, cudaStream_t st) {
    const int nb = Pl->s + 1, nb2 = 2 * nb;
    const long long nchunk = (Pl->N + 8191) / 8192;
    const long long per = (long long)nb2 * (nchunk + 1);
    const int nw = bins_warps(0, nb2);
    if (nw < 1 || per > cap) {
        set_error("class partials of one function do not fit the scratch array");
        return DWT_EINVAL;
    }
    const size_t smem = (size_t)nw * nb2 * 32 * 4;
    auto kern = k_effdim_bins<T>;
    int rc = set_smem(kern, smem);
    if (rc) return rc;
    const int G = (int)std::min<long long>(std::min<long long>(cap / per, 65535), batch);
    for (int f0 = 0; f0 < batch; f0 += G) {
        const int nf = std::min(G, batch - f0);
        {
            LaunchScope ls("effdim_bins", st);
            kern<<<dim3((unsigned)nchunk, (unsigned)nf), nw * 32, smem, st>>>(
                (const T*)coef + (long long)f0 * ld, ld, Pl->N, Pl->d_cls, nb, nchunk, scratch);
        }
        DWT_CK_LAUNCH("k_effdim_bins");
        rc = finalize(Pl, scratch, nchunk, nf, thr, eff_packed(var ? var + (long long)f0 * 2 * nb : nullptr,
                                                                dim ? dim + (long long)f0 * 2 : nullptr, nb),
                      st);
        if (rc) return rc;
    }
    return DWT_OK;
}

int effdim_into_scratch(dwt_plan_s* Pl, const void* coef, int batch, long long ld, dwt_dtype t, double* var, int* dim,
                        double thr, double* scratch, long long cap, cudaStream_t st) {
    if (t == DWT_F32) return effdim_scratch_t<float>(Pl, coef, batch, ld, var, dim, thr, scratch, cap, st);
    return effdim_scratch_t<float2>(Pl, coef, batch, ld, var, dim, thr, scratch, cap, st);
}

int run_effdim(dwt_plan_s* Pl, const void* coef, int batch, long long ld, dwt_dtype t, const EffOut& o, double thr,
               cudaStream_t st) {
    if (t == DWT_F32) return effdim_t<float>(Pl, coef, batch, ld, o, thr, st);
    return effdim_t<float2>(Pl, coef, batch, ld, o, thr, st);
}

}  // namespace dwt
