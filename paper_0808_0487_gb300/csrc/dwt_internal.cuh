// dwt_internal.cuh -- shared internals of libdwt (plan object, error and launch
// bookkeeping, device helpers).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/dwt.h"

namespace dwt {

// ---------------------------------------------------------------------------
// errors
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define DWT_CK(call)                                                        \
    do {                                                                    \
        cudaError_t e_ = (call);                                            \
        if (e_ != cudaSuccess) return ::dwt::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define DWT_CK_LAUNCH(what)                                                 \
    do {                                                                    \
        cudaError_t e_ = cudaGetLastError();                                \
        if (e_ != cudaSuccess) return ::dwt::cuda_fail(e_, what, __FILE__, __LINE__); \
    } while (0)

// ---------------------------------------------------------------------------
// launch accounting and optional per-launch event timing
void launch_begin(const char* family, cudaStream_t st);
void launch_end(const char* family, cudaStream_t st);

struct LaunchScope {
    const char* fam;
    cudaStream_t st;
    LaunchScope(const char* f, cudaStream_t s) : fam(f), st(s) { launch_begin(fam, st); }
    ~LaunchScope() { launch_end(fam, st); }
};

// ---------------------------------------------------------------------------
// the plan
struct PassGeom {
    int d0;          // first digit of the pass
    int b;           // digits in the pass
    long long S;     // p^d0: distance between consecutive rows of a tile
    int R;           // p^b rows per tile
    int Wc;          // consecutive low indices (columns) per tile, power of 2
    int wlog;        // log2(Wc)
    long long nlo;   // ceil(S / Wc)
    long long ntile; // tiles per function
};

struct PassPlan {
    int q = 0;           // number of passes
    PassGeom g[32];
};

}  // namespace dwt

namespace dwt {
struct HostStage;
}

struct dwt_plan_s {
    int p = 0, m = 0, s = 0;
    long long N = 0;
    unsigned flags = 0;
    int tables_status = -1;
    std::vector<uint8_t> C;       // host copy [s][m][m]
    std::vector<uint32_t> R_host; // host copy of d_R
    cudaStream_t st_create = nullptr;   // stream the plan was built on
    // device copies of the generating data
    uint32_t* d_R = nullptr;      // [s][m]: coset label of row i of C_j, sum_c C[j][i][c] p^c
    uint32_t* d_col = nullptr;    // [s][m]: point contribution of index digit c = 1, sum_i C[j][i][c] p^{m-1-i}
    uint8_t* d_C = nullptr;       // [s][m][m]   (d_col and d_C lie in d_R's allocation)
    // coset tables
    float* d_W = nullptr;         // [N]
    uint8_t* d_cls = nullptr;     // [N][2]
    float* d_Wt = nullptr;        // W in the tile-major order of the fused p = 2 pass (16 <= m <= 19)
    uint8_t* d_clst = nullptr;    // cls in the same order
    // tables of the p = 2 top pass for 20 <= m <= 24, in its read order:
    // compact ((Q - 1) | (|supp| << 11) and max supp) or full (W 2^-m, both classes)
    uint16_t* d_tq = nullptr;
    float* d_tw = nullptr;
    uint8_t* d_tkt = nullptr;
    uint8_t* d_tks = nullptr;
    int* h_err = nullptr;         // process-wide host-mapped status word of the top pass (bounded waits)
    int* d_err = nullptr;         // its device address on the plan's device
    uint8_t* d_T = nullptr;       // [(s+1)][N] least-nu tables (kept only with KEEP_INDEX_MAP)
    uint8_t* d_D = nullptr;       // [s][N] smallest optimal nu(k_j) per coordinate (ditto)
    // per-call workspace (grown on demand, owned by the plan)
    void* d_ws = nullptr;
    size_t ws_bytes = 0;
    // pass decompositions by element size (4, 8, 16 bytes)
    dwt::PassPlan passes[3];
    long long min_tiles = 1;        // tiles per function the high passes aim for (two per SM)
    // measured choices of DWT_PLAN_TUNE (0: the heuristic)
    int tuned_lo = 0;               // p = 2 transforms: digits of the register-tile low pass
    int tuned_tc = 0;               // p = 2 FP32 DWT_ALGO_AUTO: 1 = the split-BF16 tensor-core form
    long long tuned_group_bytes = 0;   // generic passes: bytes of functions per L2-resident group
    // device slots, streams and events of dwt_interpolate_host (first use)
    dwt::HostStage* host = nullptr;
    // kernel spline tables (dwt_spline_prepare): W_K [N], then R~_d - [H=0] and E~_j, [2s][N], FP64
    double* d_splW = nullptr;
    double* d_splT = nullptr;
    double spl_alpha = 0.0;           // the kernel's parameters, kept for evaluations
    std::vector<double> spl_gamma;
};

namespace dwt {

int ensure_workspace(dwt_plan_s* P, size_t bytes, cudaStream_t st);
// stream-ordered device allocations (no device-wide synchronisation)
int dmalloc(void** p, size_t bytes, cudaStream_t st);
// counts a page-locked host allocation in dwt_alloc_count
void count_host_alloc();
void dfree(void* p, cudaStream_t st);
const PassPlan& pass_plan(dwt_plan_s* P, int elem_bytes);
void pass_geometry(int p, int m, int elem, const int* b, int q, long long min_tiles, int wc_div, PassPlan& pp);
void pass_splits(int p, int m, int elem, std::vector<std::vector<int>>& out);
void pass_plan_range(int p, int m, int elem, int d0, int nd, long long min_tiles, PassPlan& pp);
// one job of a grouped transform (the arguments of one dwt_forward call)
struct GroupJob {
    dwt_plan_s* plan;
    const void* in;
    void* out;
    int batch;
    long long ld_in, ld_out;
};
unsigned char* host_staging(size_t bytes);   // page-locked, per host thread (NULL if unavailable)
int run_transform_grouped(const std::vector<GroupJob>& jobs, dwt_dtype in_t, dwt_dtype out_t, int sgn,
                          cudaStream_t st);
int p2_lo_grouped(int L, const std::vector<GroupJob>& jobs, dwt_dtype t, int sgn, cudaStream_t st);
int tune_passes(dwt_plan_s* P, long long min_tiles, cudaStream_t st);
bool p2_fast_ok(int m);
bool p2i_ok(int m, int s);
bool p2i_transform_ok(int m);
int p2i_transform(dwt_plan_s* Pl, const float* in, float* out, int batch, long long ld_in, long long ld_out, int sgn,
                  cudaStream_t st);
int p2i_hi_only(dwt_plan_s* Pl, float* data, int batch, long long ld, int sgn, cudaStream_t st);
int p2i_build_tables(dwt_plan_s* P, cudaStream_t st);
int p2i_table_bytes_per_point(dwt_plan_s* P);
int p2i_interpolate(dwt_plan_s* Pl, const float* f, float* c, float* coef, int batch, long long ld, bool weighted,
                    bool tc, double** part_out, long long* ntile_out, cudaStream_t st);

// kernels' host entry points (implemented in the .cu files)
int run_transform(dwt_plan_s* P, const void* in, void* out, int batch, long long ld_in, long long ld_out,
                  dwt_dtype in_t, dwt_dtype out_t, int sgn, cudaStream_t st);
int run_transform_digits(dwt_plan_s* P, const void* in, void* out, int batch, long long ld_in, long long ld_out,
                         dwt_dtype in_t, dwt_dtype out_t, int d0, int nd, int sgn, cudaStream_t st);
int run_interpolate(dwt_plan_s* P, const void* f, void* c, void* coef, int batch, long long ld, dwt_dtype f_t,
                    dwt_weight weight, dwt_algo algo, double* var, int* dim, double thr, cudaStream_t st);
// outputs of the effective-dimension step: cumulative truncation / superposition
// variances (row stride vstride doubles per function) and d_trc / d_sup (stride
// dstride ints); any pointer may be NULL
struct EffOut {
    double* vt = nullptr;
    double* vs = nullptr;
    long long vstride = 0;
    int* dt = nullptr;
    int* ds = nullptr;
    long long dstride = 0;
};
// the packed layout var [batch][2][nb], dim [batch][2]
static inline EffOut eff_packed(double* var, int* dim, int nb) {
    EffOut o;
    o.vt = var;
    o.vs = var ? var + nb : nullptr;
    o.vstride = 2ll * nb;
    o.dt = dim;
    o.ds = dim ? dim + 1 : nullptr;
    o.dstride = 2;
    return o;
}
int run_effdim(dwt_plan_s* P, const void* coef, int batch, long long ld, dwt_dtype t, const EffOut& o, double thr,
               cudaStream_t st);
// tensor-core low pass (p = 2, low 14 digits): one job of ntiles tiles of
// 2^14 elements, tpf per function, result times scale
struct TcJob {
    const float* in;
    float* out;
    long long ld_in, ld_out, tpf, ntiles;
    float scale;
};
int launch_tc_lo14(const TcJob& a, const TcJob* b, int* err, const char* fam, cudaStream_t st);
bool tc_ok(int m);
int tc_check(int* err, cudaStream_t st);
int run_wait_probe(cudaStream_t st);
int run_interpolate_host(dwt_plan_s* P, const void* f_host, void* c_host, int batch, long long ld, dwt_dtype f_t,
                         dwt_weight weight, double* var_host, int* dim_host, double thr, cudaStream_t st);
// releases the plan's dwt_interpolate_host resources: after synchronising
// (sync) or in the order of stream st
void host_stage_free(dwt_plan_s* P, cudaStream_t st, bool sync);
int run_spline_prepare(dwt_plan_s* P, double alpha, const double* gamma, cudaStream_t st);
int run_spline(dwt_plan_s* P, const double* f, void* c, int batch, long long ld, double* var_trc, double* var_sup,
               int* dim, double thr, cudaStream_t st);
void spline_free(dwt_plan_s* P, cudaStream_t st, bool sync);
int run_spline_eval(dwt_plan_s* P, const void* c, int batch, long long ld, const uint32_t* X, int Q, int M,
                    double* values, long long ldv, cudaStream_t st);
int run_spline_shifted(dwt_plan_s* P, const void* c, const uint32_t* delta, int M, void* values, int batch,
                       long long ld, const double* f_shift, double* sse, cudaStream_t st);
int run_points(dwt_plan_s* P, uint32_t* Y, long long ldY, cudaStream_t st);
int run_k_to_h(dwt_plan_s* P, const uint32_t* k, uint32_t* H, long long cnt, cudaStream_t st);
int run_h_to_k(dwt_plan_s* P, const uint32_t* H, uint32_t* k, long long cnt, cudaStream_t st);
int build_coset_tables(dwt_plan_s* P, cudaStream_t st);
int p2_build_tiled_tables(dwt_plan_s* P, cudaStream_t st);
int run_eval_product(dwt_plan_s* P, const double* coef, void* f, int batch, long long ld, dwt_dtype t,
                     cudaStream_t st);
int run_eval_exp(dwt_plan_s* P, void* f, int batch, long long ld, dwt_dtype t, cudaStream_t st);
int run_tc_transform(dwt_plan_s* P, const float* in, float* out, int batch, long long ld_in, long long ld_out,
                     int sgn, cudaStream_t st);

// Raise a kernel's dynamic shared-memory limit to the device maximum, once per
// kernel and thread-safely (the attribute belongs to the function, so
// per-launch settings from concurrent host threads would race).
int smem_limit_max_ptr(const void* kern);
template <typename F>
static inline int smem_limit_max(F* kern) {
    return smem_limit_max_ptr(reinterpret_cast<const void*>(kern));
}

static inline long long ipow_ll(int p, int m) {
    long long v = 1;
    for (int i = 0; i < m; ++i) v *= p;
    return v;
}

}  // namespace dwt
