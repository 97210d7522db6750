// dwt_api.cu -- the C ABI of libdwt: plan life cycle, argument checks,
// dispatch to the kernels, error strings, launch accounting and the optional
// per-launch event timing.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <unordered_set>
#include <vector>

#include <cmath>

#include "dwt_internal.cuh"

namespace dwt {

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};
static std::atomic<long long> g_allocs{0};

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

int cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    set_error("CUDA error %d (%s) in %s at %s:%d", (int)e, cudaGetErrorString(e), what, file, line);
    return DWT_ECUDA;
}

// ---- optional event timing ------------------------------------------------
struct ProfRec {
    const char* fam;
    cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof_open;   // started, not yet closed (stack per call site)
static std::vector<ProfRec> g_prof_done;
static std::vector<cudaEvent_t> g_ev_pool;

static cudaEvent_t ev_get() {
    if (!g_ev_pool.empty()) {
        cudaEvent_t e = g_ev_pool.back();
        g_ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void launch_begin(const char* fam, cudaStream_t st) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfRec r{fam, ev_get(), ev_get()};
    cudaEventRecord(r.a, st);
    g_prof_open.push_back(r);
}

void launch_end(const char* fam, cudaStream_t st) {
    if (!g_prof_on) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (size_t i = g_prof_open.size(); i-- > 0;) {
        if (g_prof_open[i].fam == fam) {
            ProfRec r = g_prof_open[i];
            g_prof_open.erase(g_prof_open.begin() + (long)i);
            cudaEventRecord(r.b, st);
            g_prof_done.push_back(r);
            return;
        }
    }
}

// ---- per-kernel shared-memory limit ------------------------------------------------
int smem_limit_max_ptr(const void* kern) {
    static std::mutex mu;
    static std::unordered_set<const void*> done;
    std::lock_guard<std::mutex> lk(mu);
    if (done.count(kern)) return DWT_OK;
    int dev = 0, mx = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute", __FILE__, __LINE__);
    done.insert(kern);
    return DWT_OK;
}

// ---- workspace ----------------------------------------------------------------
void count_host_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

// A page-locked staging buffer of the calling host thread, grown on demand and
// kept for the thread's life (uploads of plan-build inputs).  The caller
// synchronises the stream of its copy before the thread uses the buffer again.
namespace {
struct HostStaging {
    unsigned char* p = nullptr;
    size_t n = 0;
    ~HostStaging() {
        if (p) cudaFreeHost(p);
    }
};
thread_local HostStaging g_staging;
}  // namespace

unsigned char* host_staging(size_t bytes) {
    if (g_staging.n >= bytes) return g_staging.p;
    if (g_staging.p) cudaFreeHost(g_staging.p);
    g_staging.p = nullptr;
    g_staging.n = 0;
    const size_t want = std::max(bytes, (size_t)1 << 20);
    count_host_alloc();
    if (cudaMallocHost((void**)&g_staging.p, want) != cudaSuccess) {
        cudaGetLastError();
        g_staging.p = nullptr;
        return nullptr;
    }
    g_staging.n = want;
    return g_staging.p;
}

int dmalloc(void** p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("device allocation of %zu bytes failed (%s)", bytes, cudaGetErrorString(e));
        return DWT_ENOMEM;
    }
    return DWT_OK;
}

void dfree(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

int ensure_workspace(dwt_plan_s* P, size_t bytes, cudaStream_t st) {
    if (bytes <= P->ws_bytes) return DWT_OK;
    // stream-ordered: the old buffer is released after the work queued on st
    dfree(P->d_ws, st);
    P->d_ws = nullptr;
    P->ws_bytes = 0;
    size_t want = bytes < ((size_t)1 << 20) ? ((size_t)1 << 20) : bytes;
    int rc = dmalloc(&P->d_ws, want, st);
    if (rc) return rc;
    P->ws_bytes = want;
    return DWT_OK;
}

// ---- pass decomposition ---------------------------------------------------------
// The transform is the Kronecker power of the p-point DFT over the m digits, so
// digits may be grouped into passes freely.  Pass 0 takes the low digits as one
// contiguous run of p^b elements; later passes take p^b rows spaced p^d0 apart,
// Wc consecutive low indices wide, so that every row is a contiguous segment.
static const size_t kTileBudget = 64 * 1024;   // bytes of shared memory per tile

// widest power-of-2 column count for a pass of R rows starting at row distance S
static int pass_wc(long long R, long long S, long long cap, int wc_max) {
    int wc = 1;
    while (wc * 2 <= wc_max && wc * 2 <= S && R * wc * 2 <= cap) wc *= 2;
    return wc;
}

struct PassLimits {
    long long cap;   // elements per tile
    int wc_min, wc_max, blo, bhi;
};
static PassLimits pass_limits(int p, int elem) {
    PassLimits L;
    L.cap = (long long)(kTileBudget / (size_t)elem);
    L.wc_min = std::max(1, 64 / elem);    // 64-byte rows at least in a high pass
    L.wc_max = std::max(1, 256 / elem);   // 256-byte rows at most
    L.blo = 0;
    while (dwt::ipow_ll(p, L.blo + 1) <= L.cap) ++L.blo;
    L.bhi = 0;
    while (dwt::ipow_ll(p, L.bhi + 1) * L.wc_min <= L.cap) ++L.bhi;
    return L;
}

// Geometry of the passes of a digit split b[0..q): pass 0 the low b[0] digits,
// then the others upward.  Each high pass takes the widest rows its tile
// allows, divided by wc_div, and halves them further (down to 64 bytes) while
// it has fewer than min_tiles tiles per function.
void pass_geometry(int p, int m, int elem, const int* b, int q, long long min_tiles, int wc_div, PassPlan& pp) {
    const PassLimits L = pass_limits(p, elem);
    const long long N = dwt::ipow_ll(p, m);
    pp.q = q;
    int d = 0;
    for (int t = 0; t < q; ++t) {
        PassGeom& g = pp.g[t];
        g.d0 = d;
        g.b = b[t];
        d += b[t];
        g.S = dwt::ipow_ll(p, g.d0);
        g.R = (int)dwt::ipow_ll(p, g.b);
        g.Wc = g.d0 > 0 ? pass_wc(g.R, g.S, L.cap, L.wc_max) : 1;
        for (int k = 1; k < wc_div && g.Wc > L.wc_min; k *= 2) g.Wc /= 2;
        while (g.Wc > L.wc_min && ((g.S + g.Wc - 1) / g.Wc) * (N / (g.S * g.R)) < min_tiles) g.Wc /= 2;
        g.wlog = 0;
        while ((1 << g.wlog) < g.Wc) ++g.wlog;
        g.nlo = (g.S + g.Wc - 1) / g.Wc;
        g.ntile = g.nlo * (N / (g.S * g.R));
    }
}

// Passes over the digits d0 .. d0+nd-1 only (the stages of a digit range):
// from the lowest digit up, each pass as many digits as the tile allows (the
// low-pass limit when the range starts at digit 0, the high-pass limit above).
void pass_plan_range(int p, int m, int elem, int d0, int nd, long long min_tiles, PassPlan& pp) {
    const PassLimits L = pass_limits(p, elem);
    const long long N = dwt::ipow_ll(p, m);
    pp.q = 0;
    int d = d0;
    while (d < d0 + nd && pp.q < 32) {
        const int lim = d == 0 ? L.blo : L.bhi;
        const int b = std::max(1, std::min(lim, d0 + nd - d));
        PassGeom& g = pp.g[pp.q++];
        g.d0 = d;
        g.b = b;
        g.S = dwt::ipow_ll(p, d);
        g.R = (int)dwt::ipow_ll(p, b);
        g.Wc = d > 0 ? pass_wc(g.R, g.S, L.cap, L.wc_max) : 1;
        while (g.Wc > L.wc_min && ((g.S + g.Wc - 1) / g.Wc) * (N / (g.S * g.R)) < min_tiles) g.Wc /= 2;
        g.wlog = 0;
        while ((1 << g.wlog) < g.Wc) ++g.wlog;
        g.nlo = (g.S + g.Wc - 1) / g.Wc;
        g.ntile = g.nlo * (N / (g.S * g.R));
        d += b;
    }
}

// Candidate digit splits within the tile budget: with the fewest passes, every
// low-pass length that leaves the rest to the high passes (shared evenly), and
// one more pass shared evenly.  The heuristic's split is among them.
void pass_splits(int p, int m, int elem, std::vector<std::vector<int>>& out) {
    const PassLimits L = pass_limits(p, elem);
    out.clear();
    if (m <= L.blo) {
        out.push_back({m});
        if (m >= 2) {
            const int lo = (m + 1) / 2;
            if (m - lo <= L.bhi) out.push_back({lo, m - lo});
        }
        return;
    }
    const int nh = (m - L.blo + L.bhi - 1) / L.bhi;
    for (int lo = L.blo; lo >= std::max(1, m - nh * L.bhi); --lo) {
        const int rest = m - lo;
        if (rest < nh) continue;
        std::vector<int> bt{lo};
        for (int t = 0; t < nh; ++t) bt.push_back(rest / nh + (t < rest % nh ? 1 : 0));
        out.push_back(bt);
    }
    // one more pass, all passes as even as the limits allow
    const int q = nh + 2;
    std::vector<int> bt(q);
    for (int t = 0; t < q; ++t) bt[t] = m / q + (t < m % q ? 1 : 0);
    std::sort(bt.begin(), bt.end(), [](int a, int c) { return a > c; });   // the longest first (the low pass)
    bool ok = bt[0] <= L.blo;
    for (int t = 1; t < q; ++t) ok = ok && bt[t] <= L.bhi && bt[t] >= 1;
    if (ok) out.push_back(bt);
}

// Fewest passes first.  Among the splits with that many passes, the one whose
// narrowest high pass has the widest rows (wide rows keep the strided passes
// coalesced), then the one with the longest contiguous low pass.  A high pass
// then halves its rows (down to 64 bytes) while it has fewer than min_tiles
// tiles per function.
static void make_pass_plan(int p, int m, int elem, long long min_tiles, dwt::PassPlan& pp) {
    const PassLimits L = pass_limits(p, elem);
    int b[32];
    int q = 0;
    if (m <= L.blo) {
        b[0] = m;
        q = 1;
    } else {
        const int nh = (m - L.blo + L.bhi - 1) / L.bhi;
        int best_wc = -1;
        for (int lo = L.blo; lo >= std::max(1, m - nh * L.bhi); --lo) {
            const int rest = m - lo;
            if (rest < nh) continue;
            int bt[32], wc_lo = 1 << 30, d = lo;
            bt[0] = lo;
            for (int t = 0; t < nh; ++t) {
                bt[t + 1] = rest / nh + (t < rest % nh ? 1 : 0);
                const int wc = pass_wc(dwt::ipow_ll(p, bt[t + 1]), dwt::ipow_ll(p, d), L.cap, L.wc_max);
                wc_lo = std::min(wc_lo, wc);
                d += bt[t + 1];
            }
            if (wc_lo > best_wc) {
                best_wc = wc_lo;
                for (int t = 0; t <= nh; ++t) b[t] = bt[t];
                q = nh + 1;
            }
        }
    }
    pass_geometry(p, m, elem, b, q, min_tiles, 1, pp);
}

const PassPlan& pass_plan(dwt_plan_s* P, int elem_bytes) {
    int idx = elem_bytes == 4 ? 0 : elem_bytes == 8 ? 1 : 2;
    return P->passes[idx];
}

static bool is_prime_small(int p) {
    return p == 2 || p == 3 || p == 5 || p == 7 || p == 11 || p == 13 || p == 17 || p == 19 || p == 23 ||
           p == 29 || p == 31;
}

}  // namespace dwt

using namespace dwt;

extern "C" {

const char* dwt_strerror(int status) {
    switch (status) {
        case DWT_OK: return "ok";
        case DWT_EINVAL: return "invalid argument";
        case DWT_ESPAN: return "rows of the generating matrices do not span F_p^m";
        case DWT_ENOMEM: return "out of memory";
        case DWT_ECUDA: return "CUDA error";
        case DWT_ETIMEOUT: return "device-side wait timed out";
        case DWT_EBUSY: return "queue full";
        case DWT_EUNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

const char* dwt_last_error(void) { return g_err; }

long long dwt_launch_count(void) { return g_launches.load(); }

long long dwt_alloc_count(void) { return g_allocs.load(); }

int dwt_profile_enable(int on) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = on != 0;
    return DWT_OK;
}

int dwt_profile_reset(void) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g_prof_done) {
        g_ev_pool.push_back(r.a);
        g_ev_pool.push_back(r.b);
    }
    g_prof_done.clear();
    return DWT_OK;
}

int dwt_profile_query(const char* name, long long* launches, double* total_ms) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    long long n = 0;
    double tot = 0.0;
    for (auto& r : g_prof_done) {
        if (strcmp(r.fam, name) != 0) continue;
        DWT_CK(cudaEventSynchronize(r.b));
        float ms = 0.f;
        DWT_CK(cudaEventElapsedTime(&ms, r.a, r.b));
        tot += ms;
        ++n;
    }
    if (launches) *launches = n;
    if (total_ms) *total_ms = tot;
    return DWT_OK;
}

int dwt_plan_create(int p, int m, int s, const uint8_t* C, unsigned flags, void* stream, dwt_plan_t* out) {
    if (!out) {
        set_error("plan output pointer is NULL");
        return DWT_EINVAL;
    }
    *out = nullptr;
    if (!is_prime_small(p)) {
        set_error("p = %d: supported primes are those below 32", p);
        return DWT_EINVAL;
    }
    if (m < 1 || s < 1 || s > 255 || !C) {
        set_error("bad sizes m = %d, s = %d (or C is NULL)", m, s);
        return DWT_EINVAL;
    }
    if (ipow_ll(p, m) > (1ll << 31)) {
        set_error("p^m = %d^%d exceeds 2^31", p, m);
        return DWT_EINVAL;
    }
    if (flags & ~(DWT_PLAN_TRANSFORM_ONLY | DWT_PLAN_KEEP_INDEX_MAP | DWT_PLAN_TUNE)) {
        set_error("unknown plan flags 0x%x", flags);
        return DWT_EINVAL;
    }
    for (size_t t = 0; t < (size_t)s * m * m; ++t)
        if (C[t] >= p) {
            set_error("entry %zu of C is %d >= p", t, (int)C[t]);
            return DWT_EINVAL;
        }
    cudaStream_t st = (cudaStream_t)stream;
    dwt_plan_s* P = new dwt_plan_s();
    P->p = p;
    P->m = m;
    P->s = s;
    P->N = ipow_ll(p, m);
    P->flags = flags;
    P->C.assign(C, C + (size_t)s * m * m);
    {
        // high passes of small transforms take narrower rows, for at least two tiles per SM
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                      cudaSuccess || sms < 1) {
            cudaGetLastError();
            sms = 1;
        }
        make_pass_plan(p, m, 4, 2ll * sms, P->passes[0]);
        make_pass_plan(p, m, 8, 2ll * sms, P->passes[1]);
        make_pass_plan(p, m, 16, 2ll * sms, P->passes[2]);
        P->min_tiles = 2ll * sms;
    }
    // row coset labels and column point contributions
    std::vector<uint32_t> R((size_t)s * m), col((size_t)s * m);
    for (int j = 0; j < s; ++j)
        for (int i = 0; i < m; ++i) {
            uint64_t r = 0, pw = 1;
            for (int c = 0; c < m; ++c, pw *= (uint64_t)p) r += (uint64_t)C[((size_t)j * m + i) * m + c] * pw;
            R[(size_t)j * m + i] = (uint32_t)r;
        }
    for (int j = 0; j < s; ++j)
        for (int c = 0; c < m; ++c) {
            uint64_t v = 0;
            for (int i = 0; i < m; ++i) v = v * (uint64_t)p + C[((size_t)j * m + i) * m + c];
            col[(size_t)j * m + c] = (uint32_t)v;
        }
    int rc = DWT_OK;
    P->st_create = st;
    P->R_host = R;
    auto fail = [&](int code) {
        dwt_plan_destroy(P);
        return code;
    };
    // R, col and C in one device block, uploaded by one copy (d_R owns it)
    const size_t nR = R.size() * 4, nC = P->C.size();
    std::vector<unsigned char> blob(2 * nR + nC);
    memcpy(blob.data(), R.data(), nR);
    memcpy(blob.data() + nR, col.data(), nR);
    memcpy(blob.data() + 2 * nR, P->C.data(), nC);
    if (dmalloc((void**)&P->d_R, blob.size(), st)) {
        return fail(DWT_ENOMEM);
    }
    P->d_col = P->d_R + R.size();
    P->d_C = reinterpret_cast<uint8_t*>(P->d_R) + 2 * nR;
    if (cudaMemcpyAsync(P->d_R, blob.data(), blob.size(), cudaMemcpyHostToDevice, st) != cudaSuccess) {
        set_error("plan upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(DWT_ECUDA);
    }
    if (flags & DWT_PLAN_TUNE) {
        const int trc = tune_passes(P, P->min_tiles, st);
        if (trc) return fail(trc);
    }
    if (!(flags & DWT_PLAN_TRANSFORM_ONLY)) {
        rc = build_coset_tables(P, st);
        if (rc == DWT_ESPAN || rc == DWT_EUNSUPPORTED) {
            P->tables_status = rc;
        } else if (rc != DWT_OK) {
            return fail(rc);
        } else {
            P->tables_status = DWT_OK;
            rc = p2_build_tiled_tables(P, st);
            if (!rc) rc = p2i_build_tables(P, st);
            if (rc) return fail(rc);
        }
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cuda_fail(e, "plan build", __FILE__, __LINE__);
        return fail(DWT_ECUDA);
    }
    *out = P;
    return rc;
}

int dwt_plan(int p, int m, int s, const uint8_t* C, unsigned flags, void* stream, dwt_plan_t* out) {
    return dwt_plan_create(p, m, s, C, flags, stream, out);
}

int dwt_pass_plan_for(int p, int m, int elem_bytes, long long min_tiles, int* q, int* digits, int* wc) {
    if (!is_prime_small(p) || m < 1 || ipow_ll(p, m) > (1ll << 31) || !q || !digits || !wc ||
        (elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16) || min_tiles < 0) {
        set_error("dwt_pass_plan_for: bad arguments");
        return DWT_EINVAL;
    }
    PassPlan pp;
    make_pass_plan(p, m, elem_bytes, min_tiles, pp);
    *q = pp.q;
    for (int t = 0; t < pp.q; ++t) {
        digits[t] = pp.g[t].b;
        wc[t] = pp.g[t].Wc;
    }
    return DWT_OK;
}

int dwt_plan_passes(dwt_plan_t P, int elem_bytes, int* q, int* digits, int* wc) {
    if (!P || !q || !digits || !wc || (elem_bytes != 4 && elem_bytes != 8 && elem_bytes != 16)) {
        set_error("dwt_plan_passes: bad arguments");
        return DWT_EINVAL;
    }
    const PassPlan& pp = pass_plan(P, elem_bytes);
    *q = pp.q;
    for (int t = 0; t < pp.q; ++t) {
        digits[t] = pp.g[t].b;
        wc[t] = pp.g[t].Wc;
    }
    return DWT_OK;
}

int dwt_plan_tuned(dwt_plan_t P, int* lo_digits, int* tc, long long* group_bytes) {
    if (!P) {
        set_error("dwt_plan_tuned: NULL plan");
        return DWT_EINVAL;
    }
    if (lo_digits) *lo_digits = P->tuned_lo;
    if (tc) *tc = P->tuned_tc;
    if (group_bytes) *group_bytes = P->tuned_group_bytes;
    return DWT_OK;
}

int dwt_plan_destroy(dwt_plan_t P) {
    if (!P) return DWT_OK;
    cudaDeviceSynchronize();
    host_stage_free(P, nullptr, true);
    spline_free(P, nullptr, true);
    cudaFree(P->d_R);   // also holds d_col and d_C
    cudaFree(P->d_W);
    cudaFree(P->d_cls);
    cudaFree(P->d_Wt);
    cudaFree(P->d_clst);
    cudaFree(P->d_tq);
    cudaFree(P->d_tw);
    cudaFree(P->d_tkt);
    cudaFree(P->d_tks);
    cudaFree(P->d_T);
    cudaFree(P->d_D);
    cudaFree(P->d_ws);
    delete P;
    return DWT_OK;
}

int dwt_plan_destroy_async(dwt_plan_t P, void* stream) {
    if (!P) return DWT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    host_stage_free(P, st, false);
    spline_free(P, st, false);
    dfree(P->d_R, st);   // also holds d_col and d_C
    dfree(P->d_W, st);
    dfree(P->d_cls, st);
    dfree(P->d_Wt, st);
    dfree(P->d_clst, st);
    dfree(P->d_tq, st);
    dfree(P->d_tw, st);
    dfree(P->d_tkt, st);
    dfree(P->d_tks, st);
    dfree(P->d_T, st);
    dfree(P->d_D, st);
    dfree(P->d_ws, st);
    delete P;
    return DWT_OK;
}

int dwt_plan_info(dwt_plan_t P, int* p, int* m, int* s, long long* N, int* tables_status) {
    if (!P) {
        set_error("NULL plan");
        return DWT_EINVAL;
    }
    if (p) *p = P->p;
    if (m) *m = P->m;
    if (s) *s = P->s;
    if (N) *N = P->N;
    if (tables_status) *tables_status = P->tables_status;
    return DWT_OK;
}

int dwt_plan_tables(dwt_plan_t P, const float** W, const uint8_t** cls) {
    if (!P) {
        set_error("NULL plan");
        return DWT_EINVAL;
    }
    if (P->tables_status != DWT_OK) {
        set_error("plan has no coset tables (status %d)", P->tables_status);
        return P->tables_status < 0 ? DWT_EUNSUPPORTED : P->tables_status;
    }
    if (W) *W = P->d_W;
    if (cls) *cls = P->d_cls;
    return DWT_OK;
}

int dwt_points(dwt_plan_t P, uint32_t* Y, long long ldY, void* stream) {
    if (!P || !Y || ldY < P->N) {
        set_error("dwt_points: bad arguments");
        return DWT_EINVAL;
    }
    return run_points(P, Y, ldY, (cudaStream_t)stream);
}

int dwt_wavenumber_to_index(dwt_plan_t P, const uint32_t* k, uint32_t* H, long long cnt, void* stream) {
    if (!P || cnt < 0 || (cnt > 0 && (!k || !H))) {
        set_error("dwt_wavenumber_to_index: bad arguments");
        return DWT_EINVAL;
    }
    if (cnt == 0) return DWT_OK;
    return run_k_to_h(P, k, H, cnt, (cudaStream_t)stream);
}

int dwt_index_to_wavenumber(dwt_plan_t P, const uint32_t* H, uint32_t* k, long long cnt, void* stream) {
    if (!P || cnt < 0 || (cnt > 0 && (!k || !H))) {
        set_error("dwt_index_to_wavenumber: bad arguments");
        return DWT_EINVAL;
    }
    if (!(P->flags & DWT_PLAN_KEEP_INDEX_MAP) || P->tables_status != DWT_OK) {
        set_error("plan was not built with DWT_PLAN_KEEP_INDEX_MAP or has no coset tables");
        return P->tables_status > 0 ? P->tables_status : DWT_EUNSUPPORTED;
    }
    if (cnt == 0) return DWT_OK;
    return run_h_to_k(P, H, k, cnt, (cudaStream_t)stream);
}

static int check_transform_types(dwt_plan_s* P, dwt_dtype in_t, dwt_dtype out_t, int sgn) {
    if (P->p == 2) {
        if (in_t != out_t || !(in_t == DWT_F32 || in_t == DWT_F64 || in_t == DWT_I32)) {
            set_error("p = 2 transforms take F32->F32, F64->F64 or I32->I32");
            return DWT_EUNSUPPORTED;
        }
        return DWT_OK;
    }
    bool ok32 = out_t == DWT_C64 && (in_t == DWT_C64 || (sgn < 0 && in_t == DWT_F32));
    bool ok64 = out_t == DWT_C128 && (in_t == DWT_C128 || (sgn < 0 && in_t == DWT_F64));
    if (!ok32 && !ok64) {
        set_error("p > 2 transforms produce complex output (C64 / C128); real input only for the forward");
        return DWT_EUNSUPPORTED;
    }
    return DWT_OK;
}

static int transform_common(dwt_plan_t P, const void* in, void* out, int batch, long long ld_in, long long ld_out,
                            dwt_dtype in_t, dwt_dtype out_t, dwt_algo algo, void* stream, int sgn) {
    if (!P || batch < 0 || (batch > 0 && (!in || !out)) || ld_in < P->N || ld_out < P->N) {
        set_error("transform: bad arguments (batch %d, ld_in %lld, ld_out %lld, N %lld)", batch, ld_in, ld_out, P ? P->N : 0);
        return DWT_EINVAL;
    }
    int rc = check_transform_types(P, in_t, out_t, sgn);
    if (rc) return rc;
    if (batch == 0) return DWT_OK;
    if (algo == DWT_ALGO_TC_SPLIT_BF16) {
        if (P->p != 2 || in_t != DWT_F32) {
            set_error("the split-BF16 tensor-core form needs p = 2 and F32 data");
            return DWT_EUNSUPPORTED;
        }
        return run_tc_transform(P, (const float*)in, (float*)out, batch, ld_in, ld_out, sgn, (cudaStream_t)stream);
    }
    if (algo != DWT_ALGO_AUTO && algo != DWT_ALGO_BUTTERFLY) {
        set_error("unknown algo %d", (int)algo);
        return DWT_EINVAL;
    }
    // a tuned plan's measured choice for DWT_ALGO_AUTO
    if (algo == DWT_ALGO_AUTO && P->tuned_tc && P->p == 2 && in_t == DWT_F32 && tc_ok(P->m))
        return run_tc_transform(P, (const float*)in, (float*)out, batch, ld_in, ld_out, sgn, (cudaStream_t)stream);
    return run_transform(P, in, out, batch, ld_in, ld_out, in_t, out_t, sgn, (cudaStream_t)stream);
}

int dwt_forward(dwt_plan_t P, const void* in, void* out, int batch, long long ld_in, long long ld_out, dwt_dtype in_t,
                dwt_dtype out_t, dwt_algo algo, void* stream) {
    return transform_common(P, in, out, batch, ld_in, ld_out, in_t, out_t, algo, stream, -1);
}

int dwt_inverse(dwt_plan_t P, const void* in, void* out, int batch, long long ld_in, long long ld_out, dwt_dtype in_t,
                dwt_dtype out_t, dwt_algo algo, void* stream) {
    return transform_common(P, in, out, batch, ld_in, ld_out, in_t, out_t, algo, stream, +1);
}

static int grouped_common(const dwt_job* jobs, int njobs, dwt_dtype in_t, dwt_dtype out_t, void* stream, int sgn) {
    if (!jobs || njobs < 1) {
        set_error("grouped transform: no jobs");
        return DWT_EINVAL;
    }
    std::vector<GroupJob> js;
    js.reserve((size_t)njobs);
    for (int i = 0; i < njobs; ++i) {
        const dwt_job& j = jobs[i];
        dwt_plan_s* P = j.plan;
        if (!P || j.batch < 0 || (j.batch > 0 && (!j.in || !j.out)) || j.ld_in < P->N || j.ld_out < P->N) {
            set_error("grouped transform: bad job %d", i);
            return DWT_EINVAL;
        }
        if (P->p != jobs[0].plan->p) {
            set_error("grouped transform: job %d has p = %d, job 0 p = %d", i, P->p, jobs[0].plan->p);
            return DWT_EINVAL;
        }
        const int rc = check_transform_types(P, in_t, out_t, sgn);
        if (rc) return rc;
        js.push_back(GroupJob{P, j.in, j.out, j.batch, j.ld_in, j.ld_out});
    }
    return run_transform_grouped(js, in_t, out_t, sgn, (cudaStream_t)stream);
}

int dwt_forward_grouped(const dwt_job* jobs, int njobs, dwt_dtype in_t, dwt_dtype out_t, void* stream) {
    return grouped_common(jobs, njobs, in_t, out_t, stream, -1);
}

int dwt_inverse_grouped(const dwt_job* jobs, int njobs, dwt_dtype in_t, dwt_dtype out_t, void* stream) {
    return grouped_common(jobs, njobs, in_t, out_t, stream, +1);
}

static int digits_common(dwt_plan_t P, const void* in, void* out, int batch, long long ld_in, long long ld_out,
                         dwt_dtype in_t, dwt_dtype out_t, int d0, int nd, void* stream, int sgn) {
    if (!P || batch < 0 || (batch > 0 && (!in || !out)) || ld_in < P->N || ld_out < P->N || d0 < 0 || nd < 1 ||
        d0 + nd > P->m) {
        set_error("digit stages: bad arguments (batch %d, ld_in %lld, ld_out %lld, digits %d + %d of %d)", batch, ld_in,
                  ld_out, d0, nd, P ? P->m : 0);
        return DWT_EINVAL;
    }
    int rc = check_transform_types(P, in_t, out_t, sgn);
    if (rc) return rc;
    if (batch == 0) return DWT_OK;
    return run_transform_digits(P, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, sgn, (cudaStream_t)stream);
}

int dwt_forward_digits(dwt_plan_t P, const void* in, void* out, int batch, long long ld_in, long long ld_out,
                       dwt_dtype in_t, dwt_dtype out_t, int d0, int nd, void* stream) {
    return digits_common(P, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, stream, -1);
}

int dwt_inverse_digits(dwt_plan_t P, const void* in, void* out, int batch, long long ld_in, long long ld_out,
                       dwt_dtype in_t, dwt_dtype out_t, int d0, int nd, void* stream) {
    return digits_common(P, in, out, batch, ld_in, ld_out, in_t, out_t, d0, nd, stream, +1);
}

int dwt_interpolate(dwt_plan_t P, const void* f, void* c, void* coef, int batch, long long ld, dwt_dtype f_t,
                    dwt_weight weight, dwt_algo algo, double* var, int* dim, double thr, void* stream) {
    if (!P || batch < 0 || (batch > 0 && (!f || !c)) || ld < P->N || !(thr > 0.0 && thr <= 1.0)) {
        set_error("dwt_interpolate: bad arguments");
        return DWT_EINVAL;
    }
    if (weight != DWT_WEIGHT_NONE && weight != DWT_WEIGHT_INV_SQ_WAVENUMBER) {
        set_error("unknown weight %d", (int)weight);
        return DWT_EINVAL;
    }
    if (P->tables_status != DWT_OK) {
        set_error("plan has no coset tables (status %d)", P->tables_status);
        return P->tables_status > 0 ? P->tables_status : DWT_EUNSUPPORTED;
    }
    if (P->p == 2 ? f_t != DWT_F32 : (f_t != DWT_F32 && f_t != DWT_C64)) {
        set_error("dwt_interpolate: p = 2 takes F32; p > 2 takes F32 (real) or C64");
        return DWT_EUNSUPPORTED;
    }
    if (algo != DWT_ALGO_AUTO && algo != DWT_ALGO_BUTTERFLY && algo != DWT_ALGO_TC_SPLIT_BF16) {
        set_error("unknown algo %d", (int)algo);
        return DWT_EINVAL;
    }
    if (batch == 0) return DWT_OK;
    return run_interpolate(P, f, c, coef, batch, ld, f_t, weight, algo, var, dim, thr, (cudaStream_t)stream);
}

int dwt_interpolate_host(dwt_plan_t P, const void* f, void* c, int batch, long long ld, dwt_dtype f_t,
                         dwt_weight weight, double* var, int* dim, double thr, void* stream) {
    if (!P || batch < 0 || (batch > 0 && (!f || !c)) || ld < P->N || !(thr > 0.0 && thr <= 1.0)) {
        set_error("dwt_interpolate_host: bad arguments");
        return DWT_EINVAL;
    }
    if (weight != DWT_WEIGHT_NONE && weight != DWT_WEIGHT_INV_SQ_WAVENUMBER) {
        set_error("unknown weight %d", (int)weight);
        return DWT_EINVAL;
    }
    if (P->tables_status != DWT_OK) {
        set_error("plan has no coset tables (status %d)", P->tables_status);
        return P->tables_status > 0 ? P->tables_status : DWT_EUNSUPPORTED;
    }
    if (P->p == 2 ? f_t != DWT_F32 : (f_t != DWT_F32 && f_t != DWT_C64)) {
        set_error("dwt_interpolate_host: p = 2 takes F32; p > 2 takes F32 (real) or C64");
        return DWT_EUNSUPPORTED;
    }
    if (batch == 0) return DWT_OK;
    return run_interpolate_host(P, f, c, batch, ld, f_t, weight, var, dim, thr, (cudaStream_t)stream);
}

int dwt_selftest_bounded_wait(void* stream) { return run_wait_probe((cudaStream_t)stream); }

int dwt_spline_prepare(dwt_plan_t P, double alpha, const double* gamma, void* stream) {
    if (!P || !gamma || !(alpha > 1.0) || !std::isfinite(alpha)) {
        set_error("dwt_spline_prepare: bad arguments (alpha > 1 and gamma[s] required)");
        return DWT_EINVAL;
    }
    for (int j = 0; j < P->s; ++j)
        if (!(gamma[j] >= 0.0) || !std::isfinite(gamma[j])) {
            set_error("dwt_spline_prepare: gamma[%d] must be finite and >= 0", j);
            return DWT_EINVAL;
        }
    return run_spline_prepare(P, alpha, gamma, (cudaStream_t)stream);
}

int dwt_spline_values_shifted(dwt_plan_t P, const void* c, const uint32_t* delta, int M, void* values, int batch,
                              long long ld, const double* f_shift, double* sse, void* stream) {
    if (!P || !delta || batch < 0 || (batch > 0 && (!c || !values)) || ld < P->N) {
        set_error("dwt_spline_values_shifted: bad arguments");
        return DWT_EINVAL;
    }
    if (batch == 0) return DWT_OK;
    return run_spline_shifted(P, c, delta, M, values, batch, ld, f_shift, sse, (cudaStream_t)stream);
}

int dwt_spline_eval(dwt_plan_t P, const void* c, int batch, long long ld, const uint32_t* X, int Q, int M,
                    double* values, long long ldv, void* stream) {
    if (!P || batch < 0 || Q < 0 || ld < P->N || ldv < Q || (batch > 0 && Q > 0 && (!c || !X || !values))) {
        set_error("dwt_spline_eval: bad arguments");
        return DWT_EINVAL;
    }
    if (batch == 0 || Q == 0) return DWT_OK;
    return run_spline_eval(P, c, batch, ld, X, Q, M, values, ldv, (cudaStream_t)stream);
}

int dwt_spline(dwt_plan_t P, const double* f, void* c, int batch, long long ld, double* var_trc, double* var_sup,
               int* dim, double thr, void* stream) {
    if (!P || batch < 0 || (batch > 0 && !f) || ld < P->N || !(thr > 0.0 && thr <= 1.0)) {
        set_error("dwt_spline: bad arguments");
        return DWT_EINVAL;
    }
    if (batch == 0) return DWT_OK;
    return run_spline(P, f, c, batch, ld, var_trc, var_sup, dim, thr, (cudaStream_t)stream);
}

static int effdim_check(dwt_plan_t P, const void* coef, int batch, long long ld, dwt_dtype t, double thr,
                        const char* who) {
    if (!P || batch < 0 || (batch > 0 && !coef) || ld < P->N || !(thr > 0.0 && thr <= 1.0)) {
        set_error("%s: bad arguments", who);
        return DWT_EINVAL;
    }
    if (P->tables_status != DWT_OK) {
        set_error("plan has no coset tables (status %d)", P->tables_status);
        return P->tables_status > 0 ? P->tables_status : DWT_EUNSUPPORTED;
    }
    if (P->p == 2 ? t != DWT_F32 : t != DWT_C64) {
        set_error("%s: coefficients are F32 (p = 2) or C64 (p > 2)", who);
        return DWT_EUNSUPPORTED;
    }
    return DWT_OK;
}

int dwt_effdim(dwt_plan_t P, const void* coef, int batch, long long ld, dwt_dtype t, double* var_trc, double* var_sup,
               int* d_trc, int* d_sup, double thr, void* stream) {
    int rc = effdim_check(P, coef, batch, ld, t, thr, "dwt_effdim");
    if (rc || batch == 0) return rc;
    EffOut o;
    o.vt = var_trc;
    o.vs = var_sup;
    o.vstride = P->s + 1;
    o.dt = d_trc;
    o.ds = d_sup;
    o.dstride = 1;
    return run_effdim(P, coef, batch, ld, t, o, thr, (cudaStream_t)stream);
}

int dwt_effdim_packed(dwt_plan_t P, const void* coef, int batch, long long ld, dwt_dtype t, double* var, int* dim,
                      double thr, void* stream) {
    int rc = effdim_check(P, coef, batch, ld, t, thr, "dwt_effdim_packed");
    if (rc || batch == 0) return rc;
    return run_effdim(P, coef, batch, ld, t, eff_packed(var, dim, P->s + 1), thr, (cudaStream_t)stream);
}

int dwt_eval_product(dwt_plan_t P, const double* coef, void* f, int batch, long long ld, dwt_dtype t, void* stream) {
    if (!P || batch < 0 || (batch > 0 && (!coef || !f)) || ld < P->N || (t != DWT_F32 && t != DWT_F64)) {
        set_error("dwt_eval_product: bad arguments");
        return DWT_EINVAL;
    }
    if (batch == 0) return DWT_OK;
    return run_eval_product(P, coef, f, batch, ld, t, (cudaStream_t)stream);
}

int dwt_eval_exp(dwt_plan_t P, void* f, int batch, long long ld, dwt_dtype t, void* stream) {
    if (!P || batch < 0 || (batch > 0 && !f) || ld < P->N || (t != DWT_F32 && t != DWT_F64)) {
        set_error("dwt_eval_exp: bad arguments");
        return DWT_EINVAL;
    }
    if (batch == 0) return DWT_OK;
    return run_eval_exp(P, f, batch, ld, t, (cudaStream_t)stream);
}

}  // extern "C"
