// dwt_host.cu -- dwt_interpolate_host: the interpolation path (Sec. 3.2-3.3,
// Sec. 4) on host-resident data, with the host<->device copies overlapped
// with the transforms.
//
// The batch is cut into chunks of whole functions.  Three device slots rotate
// through three streams: the copy-in stream moves chunk k's samples into slot
// k % 3, the caller's stream runs the interpolation of that slot, and the
// copy-out stream returns chunk k's result while chunk k+1 is transformed and
// chunk k+2 is copied in.  Events order each slot's reuse after its previous
// copy-out.  The slots, streams and events belong to the plan and are created
// by the first call.
#include <string.h>

#include <algorithm>

#include "dwt_internal.cuh"

namespace dwt {

static constexpr int kSlots = 3;
static constexpr size_t kChunkBytes = (size_t)64 << 20;   // samples moved per chunk (at least one function)

struct HostStage {
    size_t fbytes = 0, cbytes = 0;   // bytes of one function's samples and results
    int chunk = 0;                   // functions per chunk
    void* f[kSlots] = {};
    void* c[kSlots] = {};
    double* var = nullptr;
    int* dim = nullptr;
    int cap = 0;                     // functions var / dim can hold
    cudaStream_t s_in = nullptr, s_out = nullptr;
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;
    cudaEvent_t ev_in[kSlots] = {}, ev_done[kSlots] = {}, ev_free[kSlots] = {};
};

void host_stage_free(dwt_plan_s* P, cudaStream_t st, bool sync) {
    HostStage* H = P->host;
    if (!H) return;
    if (sync) {
        if (H->s_in) cudaStreamSynchronize(H->s_in);
        if (H->s_out) cudaStreamSynchronize(H->s_out);
    } else if (H->ev_end) {
        cudaStreamWaitEvent(st, H->ev_end, 0);
    }
    for (int i = 0; i < kSlots; ++i) {
        if (sync) {
            cudaFree(H->f[i]);
            cudaFree(H->c[i]);
        } else {
            dfree(H->f[i], st);
            dfree(H->c[i], st);
        }
    }
    if (sync) {
        cudaFree(H->var);
        cudaFree(H->dim);
    } else {
        dfree(H->var, st);
        dfree(H->dim, st);
    }
    cudaEvent_t* evs[] = {&H->ev_start, &H->ev_end};
    for (cudaEvent_t* e : evs)
        if (*e) cudaEventDestroy(*e);
    for (int i = 0; i < kSlots; ++i) {
        if (H->ev_in[i]) cudaEventDestroy(H->ev_in[i]);
        if (H->ev_done[i]) cudaEventDestroy(H->ev_done[i]);
        if (H->ev_free[i]) cudaEventDestroy(H->ev_free[i]);
    }
    if (H->s_in) cudaStreamDestroy(H->s_in);
    if (H->s_out) cudaStreamDestroy(H->s_out);
    delete H;
    P->host = nullptr;
}

// slots for functions of fbytes / cbytes bytes; grown when a call needs more
static int host_stage_get(dwt_plan_s* P, size_t fbytes, size_t cbytes, int batch, cudaStream_t st, HostStage** out) {
    HostStage* H = P->host;
    if (H && (H->fbytes != fbytes || H->cbytes != cbytes)) {
        host_stage_free(P, st, false);
        H = nullptr;
    }
    if (!H) {
        H = new HostStage();
        P->host = H;
        H->fbytes = fbytes;
        H->cbytes = cbytes;
        H->chunk = (int)std::max<size_t>(1, kChunkBytes / fbytes);
        DWT_CK(cudaStreamCreateWithFlags(&H->s_in, cudaStreamNonBlocking));
        DWT_CK(cudaStreamCreateWithFlags(&H->s_out, cudaStreamNonBlocking));
        DWT_CK(cudaEventCreateWithFlags(&H->ev_start, cudaEventDisableTiming));
        DWT_CK(cudaEventCreateWithFlags(&H->ev_end, cudaEventDisableTiming));
        for (int i = 0; i < kSlots; ++i) {
            DWT_CK(cudaEventCreateWithFlags(&H->ev_in[i], cudaEventDisableTiming));
            DWT_CK(cudaEventCreateWithFlags(&H->ev_done[i], cudaEventDisableTiming));
            DWT_CK(cudaEventCreateWithFlags(&H->ev_free[i], cudaEventDisableTiming));
            if (dmalloc(&H->f[i], fbytes * H->chunk, st) || dmalloc(&H->c[i], cbytes * H->chunk, st))
                return DWT_ENOMEM;
        }
    }
    if (batch > H->cap) {
        dfree(H->var, st);
        dfree(H->dim, st);
        H->var = nullptr;
        H->dim = nullptr;
        H->cap = 0;
        if (dmalloc((void**)&H->var, (size_t)batch * 2 * (P->s + 1) * sizeof(double), st) ||
            dmalloc((void**)&H->dim, (size_t)batch * 2 * sizeof(int), st))
            return DWT_ENOMEM;
        H->cap = batch;
    }
    *out = H;
    return DWT_OK;
}

int run_interpolate_host(dwt_plan_s* P, const void* f_host, void* c_host, int batch, long long ld, dwt_dtype f_t,
                         dwt_weight weight, double* var_host, int* dim_host, double thr, cudaStream_t st) {
    const size_t fe = f_t == DWT_C64 ? 8 : 4;
    const size_t ce = P->p == 2 ? 4 : 8;
    const size_t fbytes = (size_t)P->N * fe, cbytes = (size_t)P->N * ce;
    HostStage* H = nullptr;
    int rc = host_stage_get(P, fbytes, cbytes, batch, st, &H);
    if (rc) return rc;
    const int nb2 = 2 * (P->s + 1);
    // the side streams start after everything already queued on the caller's
    // stream (including an earlier call that used the same slots)
    DWT_CK(cudaEventRecord(H->ev_start, st));
    DWT_CK(cudaStreamWaitEvent(H->s_in, H->ev_start, 0));
    DWT_CK(cudaStreamWaitEvent(H->s_out, H->ev_start, 0));
    const int nchunk = (batch + H->chunk - 1) / H->chunk;
    for (int k = 0; k < nchunk; ++k) {
        const int b = k % kSlots;
        const int f0 = k * H->chunk, nf = std::min(H->chunk, batch - f0);
        // copy in (after the slot's previous result has left)
        if (k >= kSlots) DWT_CK(cudaStreamWaitEvent(H->s_in, H->ev_free[b], 0));
        DWT_CK(cudaMemcpy2DAsync(H->f[b], fbytes, (const char*)f_host + (size_t)f0 * ld * fe, (size_t)ld * fe, fbytes,
                                 (size_t)nf, cudaMemcpyHostToDevice, H->s_in));
        DWT_CK(cudaEventRecord(H->ev_in[b], H->s_in));
        // transform on the caller's stream
        DWT_CK(cudaStreamWaitEvent(st, H->ev_in[b], 0));
        rc = run_interpolate(P, H->f[b], H->c[b], nullptr, nf, P->N, f_t, weight, DWT_ALGO_AUTO, H->var + (size_t)f0 * nb2,
                             H->dim + (size_t)f0 * 2, thr, st);
        if (rc) return rc;
        DWT_CK(cudaEventRecord(H->ev_done[b], st));
        // copy out
        DWT_CK(cudaStreamWaitEvent(H->s_out, H->ev_done[b], 0));
        DWT_CK(cudaMemcpy2DAsync((char*)c_host + (size_t)f0 * ld * ce, (size_t)ld * ce, H->c[b], cbytes, cbytes,
                                 (size_t)nf, cudaMemcpyDeviceToHost, H->s_out));
        DWT_CK(cudaEventRecord(H->ev_free[b], H->s_out));
    }
    // variances and dimensions, then the caller's stream waits for the last copy out
    if (var_host)
        DWT_CK(cudaMemcpyAsync(var_host, H->var, (size_t)batch * nb2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (dim_host)
        DWT_CK(cudaMemcpyAsync(dim_host, H->dim, (size_t)batch * 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    DWT_CK(cudaEventRecord(H->ev_end, H->s_out));
    DWT_CK(cudaStreamWaitEvent(st, H->ev_end, 0));
    return DWT_OK;
}

}  // namespace dwt
