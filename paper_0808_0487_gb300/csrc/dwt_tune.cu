// dwt_tune.cu -- measured choices of a plan (DWT_PLAN_TUNE).
//
// Any grouping of the m digits into passes computes the same transform
// (Sec. 2.2: the digit sums commute); what differs is the time.  With
// DWT_PLAN_TUNE the plan measures, on scratch functions of its size, in the
// FP32 form (real to complex for p > 2):
//  - the digit split of the generic passes: every candidate split, each with
//    the heuristic row width and with half of it;
//  - the functions per group of the generic passes (16, 48, 128 MB of
//    functions between the passes of a group, L2-resident, or 1 GB: every
//    pass over the whole batch in one launch);
//  - p = 2, 16 <= m <= 19: the digits of the register-tile low pass (the high
//    pass takes the rest);
//  - p = 2 where the split-BF16 tensor-core form exists: whether
//    DWT_ALGO_AUTO runs it instead of the butterflies (its results differ from
//    the butterflies' by rounding, within the same tolerance);
// and keeps the fastest of each.  Results are cached per process and, when
// the environment variable DWT_TUNE_CACHE names a file, in that file (one JSON
// object per line: device, p, m, element size, digits and row widths of the
// passes, low-pass digits, tensor-core choice, group bytes), so a shape is
// measured once per device.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "dwt_internal.cuh"

namespace dwt {

namespace {

struct TunedSplit {
    std::vector<int> b, wc;   // empty: no generic split was measured
    int lo = 0, tc = 0;
    long long group = 0;
};

std::mutex g_mu;
std::map<std::string, TunedSplit> g_cache;
bool g_file_read = false;

std::string cache_key(const std::string& dev, int p, int m, int elem) {
    char buf[64];
    snprintf(buf, sizeof buf, "|%d|%d|%d", p, m, elem);
    return dev + buf;
}

// integers of the JSON array that follows "name": [ in line
bool json_ints(const char* line, const char* name, std::vector<int>& out) {
    const char* k = strstr(line, name);
    if (!k) return false;
    const char* a = strchr(k, '[');
    const char* z = a ? strchr(a, ']') : nullptr;
    if (!a || !z) return false;
    out.clear();
    for (const char* c = a + 1; c < z;) {
        char* e = nullptr;
        const long v = strtol(c, &e, 10);
        if (e == c) {
            ++c;
            continue;
        }
        out.push_back((int)v);
        c = e;
    }
    return true;
}

bool json_int(const char* line, const char* name, int* v) {
    const char* k = strstr(line, name);
    if (!k) return false;
    k = strchr(k, ':');
    if (!k) return false;
    *v = (int)strtol(k + 1, nullptr, 10);
    return true;
}

void read_cache_file() {
    const char* path = getenv("DWT_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* fh = fopen(path, "r");
    if (!fh) return;
    char line[1024];
    while (fgets(line, sizeof line, fh)) {
        const char* d = strstr(line, "\"device\": \"");
        if (!d) continue;
        d += strlen("\"device\": \"");
        const char* de = strchr(d, '"');
        if (!de) continue;
        int p = 0, m = 0, elem = 0, gmb = 0;
        TunedSplit ts;
        if (!json_int(line, "\"p\"", &p) || !json_int(line, "\"m\"", &m) || !json_int(line, "\"elem\"", &elem) ||
            !json_ints(line, "\"digits\"", ts.b) || !json_ints(line, "\"wc\"", ts.wc) || ts.b.size() != ts.wc.size())
            continue;
        json_int(line, "\"lo\"", &ts.lo);
        json_int(line, "\"tc\"", &ts.tc);
        if (json_int(line, "\"group_mb\"", &gmb)) ts.group = (long long)gmb << 20;
        g_cache[cache_key(std::string(d, de), p, m, elem)] = ts;
    }
    fclose(fh);
}

void append_cache_file(const std::string& dev, int p, int m, int elem, const TunedSplit& ts) {
    const char* path = getenv("DWT_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* fh = fopen(path, "a");
    if (!fh) return;
    fprintf(fh, "{\"device\": \"%s\", \"p\": %d, \"m\": %d, \"elem\": %d, \"digits\": [", dev.c_str(), p, m, elem);
    for (size_t i = 0; i < ts.b.size(); ++i) fprintf(fh, "%s%d", i ? ", " : "", ts.b[i]);
    fprintf(fh, "], \"wc\": [");
    for (size_t i = 0; i < ts.wc.size(); ++i) fprintf(fh, "%s%d", i ? ", " : "", ts.wc[i]);
    fprintf(fh, "], \"lo\": %d, \"tc\": %d, \"group_mb\": %lld}\n", ts.lo, ts.tc, ts.group >> 20);
    fclose(fh);
}

// a plan from a cached split: the digits, and row widths as measured
bool apply_split(int p, int m, int elem, const TunedSplit& ts, PassPlan& pp) {
    int sum = 0;
    for (int v : ts.b) {
        if (v < 1) return false;
        sum += v;
    }
    if (sum != m || ts.b.empty() || ts.b.size() > 32) return false;
    pass_geometry(p, m, elem, ts.b.data(), (int)ts.b.size(), 0, 1, pp);
    const long long N = ipow_ll(p, m);
    for (int t = 0; t < pp.q; ++t) {
        PassGeom& g = pp.g[t];
        const int wc = ts.wc[t];
        if (wc < 1 || (wc & (wc - 1)) || (long long)g.R * wc * elem > 64 * 1024 || (t == 0 && wc != 1)) return false;
        g.Wc = wc;
        g.wlog = 0;
        while ((1 << g.wlog) < g.Wc) ++g.wlog;
        g.nlo = (g.S + g.Wc - 1) / g.Wc;
        g.ntile = g.nlo * (N / (g.S * g.R));
    }
    return true;
}

}  // namespace

// best of 3 timed runs (after one untimed) of fn on st; < 0 on failure
template <typename F>
static float time_best(F fn, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, int* rc) {
    float best = -1.f;
    for (int rep = 0; rep < 4 && !*rc; ++rep) {
        cudaEventRecord(e0, st);
        *rc = fn();
        cudaEventRecord(e1, st);
        if (*rc) break;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            *rc = cuda_fail(cudaGetLastError(), "tuning run", __FILE__, __LINE__);
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best < 0.f || ms < best)) best = ms;
    }
    return best;
}

static void apply_choices(dwt_plan_s* P, const TunedSplit& ts) {
    P->tuned_lo = ts.lo;
    P->tuned_tc = ts.tc;
    P->tuned_group_bytes = ts.group;
}

int tune_passes(dwt_plan_s* P, long long min_tiles, cudaStream_t st) {
    const int p = P->p, m = P->m;
    const long long N = P->N;
    // the FP32 form: real -> complex for p > 2; for p = 2 the generic passes
    // outside the register-tile range
    const bool generic = !(p == 2 && p2_fast_ok(m));
    const int elem = p == 2 ? 4 : 8;
    const int idx = p == 2 ? 0 : 1;
    const size_t per_fn = (size_t)N * (4 + (size_t)elem);
    if (per_fn > ((size_t)1 << 30)) return DWT_OK;   // above 1 GiB of scratch the heuristics stay
    int dev = 0;
    cudaDeviceProp prop;
    DWT_CK(cudaGetDevice(&dev));
    DWT_CK(cudaGetDeviceProperties(&prop, dev));
    char devbuf[300];
    snprintf(devbuf, sizeof devbuf, "%s/%d", prop.name, prop.multiProcessorCount);
    const std::string devname(devbuf);
    const std::string key = cache_key(devname, p, m, elem);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_file_read) {
            read_cache_file();
            g_file_read = true;
        }
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            PassPlan pp;
            if (!generic || it->second.b.empty()) {
                apply_choices(P, it->second);
                return DWT_OK;
            }
            if (apply_split(p, m, elem, it->second, pp)) {
                P->passes[idx] = pp;
                apply_choices(P, it->second);
                return DWT_OK;
            }
        }
    }
    // scratch: up to 256 MB of functions (at least one)
    const int nbatch = (int)std::max<size_t>(1, std::min<size_t>(64, ((size_t)256 << 20) / per_fn));
    void* in = nullptr;
    void* out = nullptr;
    int rc = dmalloc(&in, (size_t)nbatch * N * 4, st);
    if (!rc) rc = dmalloc(&out, (size_t)nbatch * N * elem, st);
    if (rc) {   // no room for the scratch: the heuristics stay
        dfree(in, st);
        return DWT_OK;
    }
    DWT_CK(cudaMemsetAsync(in, 0, (size_t)nbatch * N * 4, st));
    cudaEvent_t e0, e1;
    DWT_CK(cudaEventCreate(&e0));
    DWT_CK(cudaEventCreate(&e1));
    const dwt_dtype ot = p == 2 ? DWT_F32 : DWT_C64;
    TunedSplit ts;
    const PassPlan keep = P->passes[idx];
    if (generic) {
        // the digit split: every split, with the heuristic row widths and with half
        std::vector<std::vector<int>> splits;
        pass_splits(p, m, elem, splits);
        std::vector<PassPlan> cands;
        cands.push_back(P->passes[idx]);   // the heuristic plan first
        for (const auto& b : splits)
            for (int div : {1, 2}) {
                PassPlan pp;
                pass_geometry(p, m, elem, b.data(), (int)b.size(), min_tiles, div, pp);
                bool dup = false;
                for (const PassPlan& c : cands) {
                    bool same = c.q == pp.q;
                    for (int t = 0; same && t < pp.q; ++t) same = c.g[t].b == pp.g[t].b && c.g[t].Wc == pp.g[t].Wc;
                    dup = dup || same;
                }
                if (!dup) cands.push_back(pp);
            }
        int best = 0;
        float best_ms = -1.f;
        for (size_t c = 0; c < cands.size() && !rc; ++c) {
            P->passes[idx] = cands[c];
            const float ms = time_best([&] { return run_transform(P, in, out, 1, N, N, DWT_F32, ot, -1, st); }, st,
                                       e0, e1, &rc);
            if (!rc && ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
                best_ms = ms;
                best = (int)c;
            }
        }
        P->passes[idx] = rc ? keep : cands[best];
        for (int t = 0; !rc && t < cands[best].q; ++t) {
            ts.b.push_back(cands[best].g[t].b);
            ts.wc.push_back(cands[best].g[t].Wc);
        }
        // functions per L2-resident group, on the whole scratch batch
        if (!rc && nbatch > 1) {
            const long long fbytes = N * (long long)elem;
            long long best_g = 0;
            float gbest = -1.f;
            int last_G = -1;
            for (long long mb : {48ll, 16ll, 128ll, 1024ll}) {
                const long long bytes = mb << 20;
                const int G = (int)std::max(1ll, bytes / fbytes);
                if (G == last_G || (G >= nbatch && last_G >= nbatch)) continue;
                last_G = G;
                P->tuned_group_bytes = bytes;
                const float ms = time_best(
                    [&] { return run_transform(P, in, out, nbatch, N, N, DWT_F32, ot, -1, st); }, st, e0, e1, &rc);
                if (rc) break;
                if (ms >= 0.f && (gbest < 0.f || ms < gbest * 0.97f)) {   // 3% better than the first to move
                    gbest = ms;
                    best_g = bytes;
                }
            }
            P->tuned_group_bytes = 0;
            if (!rc && best_g != (48ll << 20)) ts.group = best_g;
        }
    }
    if (!rc && p == 2 && m >= 16 && m <= 19) {
        // low-pass digits of the register-tile pair
        float best_ms = -1.f;
        for (int L = std::max(12, m - 10); L <= std::min(14, m - 4) && !rc; ++L) {
            P->tuned_lo = L;
            const float ms = time_best(
                [&] { return run_transform(P, in, out, nbatch, N, N, DWT_F32, DWT_F32, -1, st); }, st, e0, e1, &rc);
            if (!rc && ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
                best_ms = ms;
                ts.lo = L;
            }
        }
        P->tuned_lo = 0;
    }
    if (!rc && p == 2 && tc_ok(m)) {
        // tensor-core form against the butterflies for DWT_ALGO_AUTO
        // (both timed to the end of a synchronisation: the tensor-core call reads its wait flag)
        const float b_ms = time_best(
            [&] {
                const int r = run_transform(P, in, out, nbatch, N, N, DWT_F32, DWT_F32, -1, st);
                return r ? r : (cudaStreamSynchronize(st) == cudaSuccess ? DWT_OK : DWT_ECUDA);
            },
            st, e0, e1, &rc);
        int trc = 0;
        const float t_ms = rc ? -1.f
                              : time_best([&] { return run_tc_transform(P, (const float*)in, (float*)out, nbatch, N,
                                                                         N, -1, st); },
                                          st, e0, e1, &trc);
        if (!rc && !trc && t_ms >= 0.f && b_ms >= 0.f && t_ms < b_ms) ts.tc = 1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(in, st);
    dfree(out, st);
    if (rc) {
        P->passes[idx] = keep;
        return rc;
    }
    apply_choices(P, ts);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_cache.count(key)) {
        g_cache[key] = ts;
        append_cache_file(devname, p, m, elem, ts);
    }
    return DWT_OK;
}

}  // namespace dwt
