// dwt_server.cu -- continuous-batching request engine over the transform
// pipeline.
//
// A request is one complete job of the method: a digital net P(C) of its own
// (p, m, s, C), a product test function sampled on it, and the interpolation
// path forward transform -> weighting -> class variances / effective
// dimensions -> inverse transform (Algorithms 1 and 2, Sec. 3, Sec. 4).
//
// Requests wait in a FIFO queue.  A pool of worker threads, one CUDA stream
// each ("slots"), admits the head of the queue as soon as a slot is idle and
// its device-memory footprint fits the budget left; the admitted request then
// builds its plan, evaluates its function, runs dwt_interpolate and copies its
// results back, all on its own stream.  Every allocation on that path is
// stream-ordered, so requests in different slots overlap on the GPU and never
// wait for each other's memory operations.  Results are kept by ticket until
// polled; timestamps give queueing and service latency.
#include <stdio.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dwt_internal.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    unsigned long long ticket;
    int p, m, s, weight;
    double thr;
    std::vector<uint8_t> C;
    std::vector<double> coef;
    float* c_out;
    size_t footprint;
    double t_submit;
};

}  // namespace

struct dwt_server_s {
    size_t budget = 0, used = 0;
    int slots = 1;
    size_t max_queue = 1024;
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req> queue;
    std::unordered_map<unsigned long long, dwt_result> done;
    std::unordered_map<unsigned long long, int> live;   // submitted, not yet polled
    std::vector<std::thread> workers;
    bool stop = false;
    unsigned long long next_ticket = 1;
    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace dwt {

// device bytes one request holds at its peak (plan build + buffers)
static size_t request_footprint(int p, int m, int s) {
    const size_t N = (size_t)ipow_ll(p, m);
    // plan build per label: the tiled tree forms (k_j per coordinate, records
    // or levels, T, W, cls) or the per-digit programme's tables, state, W and
    // cls, whichever is larger
    const size_t plan_build = p == 2 ? std::max<size_t>((size_t)(4 * s + 10), (size_t)(2 * s + 1 + m + 2) + 12)
                                     : std::max<size_t>((size_t)(4 * s + 10), (size_t)(2 * s + 1 + m + 2) + 12);
    const size_t tiled = (p == 2 && m >= 16) ? 6 : 0;
    const size_t data = 4 + (p == 2 ? 4 : 8);                    // f (real) and c
    return N * (plan_build + tiled + data) + ((size_t)1 << 20);
}

static void run_request(dwt_server_s* S, Req& r, cudaStream_t st, double* var_h, int* dim_h, dwt_result& res) {
    res.status = DWT_OK;
    res.s = r.s;
    const double t_admit = S->now();
    res.t_admit = t_admit;
    dwt_plan_t plan = nullptr;
    int rc = dwt_plan_create(r.p, r.m, r.s, r.C.data(), 0, st, &plan);
    res.t_plan = S->now();
    if (rc != DWT_OK) {
        snprintf(res.message, sizeof res.message, "plan: %s", dwt_last_error());
        if (plan) dwt_plan_destroy_async(plan, st);
        res.status = rc;
        return;
    }
    const long long N = plan->N;
    const int nb = r.s + 1;
    float *f = nullptr, *c = nullptr;
    double *coef = nullptr, *var = nullptr;
    int* dim = nullptr;
    const size_t cbytes = (size_t)N * (r.p == 2 ? 4 : 8);
    if (dmalloc((void**)&f, (size_t)N * 4, st) || dmalloc((void**)&c, cbytes, st) ||
        dmalloc((void**)&coef, (size_t)r.s * 8, st) || dmalloc((void**)&var, (size_t)2 * nb * 8, st) ||
        dmalloc((void**)&dim, 2 * sizeof(int), st)) {
        rc = DWT_ENOMEM;
    }
    if (!rc && cudaMemcpyAsync(coef, r.coef.data(), (size_t)r.s * 8, cudaMemcpyHostToDevice, st) != cudaSuccess)
        rc = DWT_ECUDA;
    if (!rc) rc = dwt_eval_product(plan, coef, f, 1, N, DWT_F32, st);
    if (!rc)
        rc = dwt_interpolate(plan, f, c, nullptr, 1, N, DWT_F32, (dwt_weight)r.weight, DWT_ALGO_AUTO, var, dim, r.thr,
                             st);
    if (!rc && (cudaMemcpyAsync(var_h, var, (size_t)2 * nb * 8, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaMemcpyAsync(dim_h, dim, 2 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess))
        rc = DWT_ECUDA;
    if (!rc && r.c_out && cudaMemcpyAsync(r.c_out, c, cbytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        rc = DWT_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess && !rc) rc = DWT_ECUDA;
    res.t_done = S->now();
    if (!rc) {
        for (int d = 0; d < nb; ++d) {
            res.var_trc[d] = var_h[d];
            res.var_sup[d] = var_h[nb + d];
        }
        res.d_trc = dim_h[0];
        res.d_sup = dim_h[1];
    }
    res.status = rc;
    if (rc) snprintf(res.message, sizeof res.message, "%s", dwt_last_error());
    dfree(f, st);
    dfree(c, st);
    dfree(coef, st);
    dfree(var, st);
    dfree(dim, st);
    dwt_plan_destroy_async(plan, st);
}

static void worker_main(dwt_server_s* S) {
    cudaSetDevice(S->device);
    cudaStream_t st = nullptr;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    double* var_h = nullptr;
    int* dim_h = nullptr;
    count_host_alloc();
    count_host_alloc();
    cudaMallocHost(&var_h, 2 * 256 * sizeof(double));
    cudaMallocHost(&dim_h, 2 * sizeof(int));
    for (;;) {
        Req r;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait(lk, [&] {
                if (S->queue.empty()) return S->stop;
                const Req& h = S->queue.front();
                return S->used == 0 || S->used + h.footprint <= S->budget;
            });
            if (S->queue.empty()) break;
            r = std::move(S->queue.front());
            S->queue.pop_front();
            S->used += r.footprint;
        }
        S->cv_work.notify_all();   // the next head may fit as well
        dwt_result res{};
        res.t_submit = r.t_submit;
        run_request(S, r, st, var_h, dim_h, res);
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->used -= r.footprint;
            S->done[r.ticket] = res;
        }
        S->cv_done.notify_all();
        S->cv_work.notify_all();
    }
    cudaStreamSynchronize(st);
    cudaFreeHost(var_h);
    cudaFreeHost(dim_h);
    cudaStreamDestroy(st);
}

}  // namespace dwt

using namespace dwt;

extern "C" {

int dwt_server_create(size_t hbm_budget_bytes, int slots, int max_queue, dwt_server_t* out) {
    if (!out || slots < 1 || slots > 64 || max_queue < 1) {
        set_error("dwt_server_create: bad arguments");
        return DWT_EINVAL;
    }
    dwt_server_s* S = new dwt_server_s();
    cudaGetDevice(&S->device);
    if (hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        hbm_budget_bytes = fr / 2;
    }
    // keep freed blocks in the stream-ordered pool instead of returning them to
    // the driver at every synchronisation, and never let one slot's allocation
    // wait for another slot's stream to reach a free (settings of this
    // process's pool only)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, S->device) == cudaSuccess) {
        unsigned long long thr = hbm_budget_bytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        int no = 0;
        cudaMemPoolSetAttribute(pool, cudaMemPoolReuseAllowInternalDependencies, &no);
    }
    S->budget = hbm_budget_bytes;
    S->slots = slots;
    S->max_queue = (size_t)max_queue;
    S->t0 = Clock::now();
    for (int i = 0; i < slots; ++i) S->workers.emplace_back(worker_main, S);
    *out = S;
    return DWT_OK;
}

int dwt_server_submit(dwt_server_t S, const dwt_request* q, unsigned long long* ticket) {
    if (!S || !q || !ticket || !q->C || !q->coef) {
        set_error("dwt_server_submit: bad arguments");
        return DWT_EINVAL;
    }
    if (!(q->p == 2 || q->p == 3 || q->p == 5 || q->p == 7 || q->p == 11 || q->p == 13 || q->p == 17 ||
          q->p == 19 || q->p == 23 || q->p == 29 || q->p == 31) || q->m < 1 || q->s < 1 ||
        q->s > 255 ||
        ipow_ll(q->p, q->m) > (1ll << 31) || !(q->threshold > 0.0 && q->threshold <= 1.0)) {
        set_error("dwt_server_submit: bad request shape");
        return DWT_EINVAL;
    }
    Req r;
    r.p = q->p;
    r.m = q->m;
    r.s = q->s;
    r.weight = q->weight;
    r.thr = q->threshold;
    r.C.assign(q->C, q->C + (size_t)q->s * q->m * q->m);
    r.coef.assign(q->coef, q->coef + q->s);
    r.c_out = q->c_out;
    r.footprint = request_footprint(q->p, q->m, q->s);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->queue.size() >= S->max_queue) {
            set_error("queue full");
            return DWT_EBUSY;
        }
        if (r.footprint > S->budget) {
            set_error("request needs %zu bytes, budget is %zu", r.footprint, S->budget);
            return DWT_ENOMEM;
        }
        r.ticket = S->next_ticket++;
        r.t_submit = S->now();
        *ticket = r.ticket;
        S->live[r.ticket] = 1;
        S->queue.push_back(std::move(r));
    }
    S->cv_work.notify_one();
    return DWT_OK;
}

int dwt_server_poll(dwt_server_t S, unsigned long long ticket, dwt_result* res) {
    if (!S || !res) return DWT_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->done.find(ticket);
    if (it == S->done.end()) {
        if (S->live.count(ticket)) return DWT_EBUSY;
        set_error("unknown ticket %llu", ticket);
        return DWT_EINVAL;
    }
    *res = it->second;
    S->done.erase(it);
    S->live.erase(ticket);
    return DWT_OK;
}

int dwt_server_wait(dwt_server_t S, unsigned long long ticket, double timeout_s, dwt_result* res) {
    if (!S || !res) return DWT_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    if (!S->live.count(ticket)) {
        set_error("unknown ticket %llu", ticket);
        return DWT_EINVAL;
    }
    const bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                        [&] { return S->done.count(ticket) > 0; });
    if (!ok) {
        set_error("ticket %llu not done after %.3f s", ticket, timeout_s);
        return DWT_ETIMEOUT;
    }
    *res = S->done[ticket];
    S->done.erase(ticket);
    S->live.erase(ticket);
    return DWT_OK;
}

int dwt_server_stats(dwt_server_t S, long long* queued, size_t* bytes_in_use, double* now_s) {
    if (!S) return DWT_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (queued) *queued = (long long)S->queue.size();
    if (bytes_in_use) *bytes_in_use = S->used;
    if (now_s) *now_s = S->now();
    return DWT_OK;
}

int dwt_server_destroy(dwt_server_t S) {
    if (!S) return DWT_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    for (auto& t : S->workers) t.join();
    delete S;
    return DWT_OK;
}

}  // extern "C"
