// dwt_noalloc.cu -- dwt_effdim_static: the effective-dimension call of
// dwt_effdim, but with no device allocation of any kind.
//
// Who needs this: dwt_effdim keeps its per-tile class partials in a workspace
// that the plan grows with cudaMalloc on demand.  Some callers cannot allow
// that: an application that reserves its whole device-memory budget up front
// and forbids later allocations (another allocator owns the rest of the
// card), or a latency-critical loop that cannot absorb the implicit
// device-wide synchronisation of cudaMalloc / cudaFree.  This entry point
// keeps the partials in one fixed, file-scope __device__ array instead.
//
// The array lives in the library image: every GPU on which the library is
// loaded holds it (8 MiB) until the process exits.  Every call on a device
// shares that one array, and it keeps whatever the last call left in it.
#include <mutex>

#include "dwt_internal.cuh"

namespace dwt {

int effdim_into_scratch(dwt_plan_s* Pl, const void* coef, int batch, long long ld, dwt_dtype t, double* var, int* dim,
                        double thr, double* scratch, long long scratch_doubles, cudaStream_t st);

// largest scratch one function may need: 2 (s+1) classes x (ceil(N / 8192) + 1) doubles
static constexpr long long kEffdimScratchDoubles = 1ll << 20;   // 8 MiB
static __device__ __align__(256) double g_effdim_scratch[kEffdimScratchDoubles];

static std::mutex g_scratch_mu;
static double* g_scratch_addr[128];

// Device address of the array for the current device, looked up once per device.
static int scratch_address(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
    if (dev < 0 || dev >= 128) {
        set_error("device index %d out of range", dev);
        return DWT_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_effdim_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return DWT_OK;
}

}  // namespace dwt

using namespace dwt;

extern "C" int dwt_effdim_static(dwt_plan_t P, const void* coef, int batch, long long ld, dwt_dtype t, double* var,
                                 int* dim, double thr, void* stream) {
    if (!P || batch < 0 || (batch > 0 && !coef) || ld < P->N || !(thr > 0.0 && thr <= 1.0)) {
        set_error("dwt_effdim_static: bad arguments");
        return DWT_EINVAL;
    }
    const long long need = 2ll * (P->s + 1) * ((P->N + 8191) / 8192 + 1);
    if (need > kEffdimScratchDoubles) {
        set_error("dwt_effdim_static: one function needs %lld scratch doubles, the fixed array holds %lld "
                  "(2 (s+1) (ceil(N/8192)+1) must not exceed it); use dwt_effdim", need, kEffdimScratchDoubles);
        return DWT_EINVAL;
    }
    if (P->tables_status != DWT_OK) {
        set_error("plan has no coset tables (status %d)", P->tables_status);
        return P->tables_status > 0 ? P->tables_status : DWT_EUNSUPPORTED;
    }
    if (P->p == 2 ? t != DWT_F32 : t != DWT_C64) {
        set_error("dwt_effdim_static: coefficients are F32 (p = 2) or C64 (p > 2)");
        return DWT_EUNSUPPORTED;
    }
    if (batch == 0) return DWT_OK;
    double* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    return effdim_into_scratch(P, coef, batch, ld, t, var, dim, thr, scratch, kEffdimScratchDoubles,
                               (cudaStream_t)stream);
}
