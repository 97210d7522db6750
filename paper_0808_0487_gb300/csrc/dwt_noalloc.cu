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
#include <cuda.h>

#include <map>
#include <mutex>

#include "dwt_internal.cuh"

namespace dwt {

int effdim_into_scratch(dwt_plan_s* Pl, const void* coef, int batch, long long ld, dwt_dtype t, double* var, int* dim,
                        double thr, double* scratch, long long scratch_doubles, cudaStream_t st);

// largest scratch one function may need: 2 (s+1) classes x (ceil(N / 8192) + 1) doubles
static constexpr long long kEffdimScratchDoubles = 1ll << 20;   // 8 MiB
static __device__ __align__(256) double g_effdim_scratch[kEffdimScratchDoubles];

// The array's device address belongs to the CUDA context the library's module
// was loaded in: it is looked up once per context (with that context current)
// and cached under the context's unique id, which a later context never
// reuses (so a cudaDeviceReset or a second context on the same device gets its
// own lookup).  Without the driver's context-id call the cache is keyed by
// the device index.
typedef CUresult (*CtxCurrentFn)(CUcontext*);
typedef CUresult (*CtxIdFn)(CUcontext, unsigned long long*);

static std::mutex g_scratch_mu;
static std::map<unsigned long long, double*> g_scratch_addr;
static CtxCurrentFn g_ctx_current = nullptr;
static CtxIdFn g_ctx_id = nullptr;
static bool g_ctx_fns_looked_up = false;

static bool context_key(unsigned long long* key) {
    if (!g_ctx_fns_looked_up) {
        g_ctx_fns_looked_up = true;
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess) {
            g_ctx_current = reinterpret_cast<CtxCurrentFn>(f1);
            g_ctx_id = reinterpret_cast<CtxIdFn>(f2);
        }
        cudaGetLastError();
    }
    if (!g_ctx_current || !g_ctx_id) return false;
    CUcontext ctx = nullptr;
    if (g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return g_ctx_id(ctx, key) == CUDA_SUCCESS;
}

// Device address of the array in the current context.
static int scratch_address(double** out) {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    unsigned long long key = 0;
    bool have_key = context_key(&key);
    if (!have_key) {
        // no context current yet, or no context-id call: the lookup below makes the
        // device's primary context current; then key by context, else by device
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_effdim_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
        have_key = context_key(&key);
        if (!have_key) {
            int dev = 0;
            e = cudaGetDevice(&dev);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
            key = ~0ull - (unsigned long long)dev;
        }
        g_scratch_addr[key] = static_cast<double*>(p);
    }
    auto it = g_scratch_addr.find(key);
    if (it == g_scratch_addr.end()) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_effdim_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress", __FILE__, __LINE__);
        it = g_scratch_addr.emplace(key, static_cast<double*>(p)).first;
    }
    *out = it->second;
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
