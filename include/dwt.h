/*
 * dwt.h -- C ABI of libdwt, a GB300 (sm_103a) library for the multivariate
 * fast discrete Walsh transform over digital (t,m,s)-nets and its inverse,
 * after K.-I. Liu, J. Dick and F. J. Hickernell, "A Multivariate Fast Discrete
 * Walsh Transform with an Application to Function Interpolation".
 *
 * Notation: p prime, m digits, s dimension, N = p^m.  Data f_n are indexed by
 * n = n_0 + n_1 p + ... + n_{m-1} p^{m-1} (the net point x_n of Def. 1.1);
 * coefficients are indexed by the coset label H = h_0 + h_1 p + ... with
 * (h_0..h_{m-1}) = C . k (Sec. 2.1), k being the representative of that coset
 * in K(C): least nu(k), ties broken by the lexicographically smallest
 * (k_1, ..., k_s) compared as integers.
 *
 * Conventions for every call:
 *  - Pointers named "device" are CUDA device (or managed) memory owned by the
 *    caller; the library never frees them.  Host pointers are plain memory.
 *  - Array arguments are row-major; "ld" is the distance in ELEMENTS between
 *    consecutive functions of a batch (ld >= N; 16-byte alignment of every
 *    function start gives the fastest path, any ld works).
 *  - Complex data (DWT_C64, DWT_C128) is interleaved (re, im).
 *  - Calls are asynchronous on "stream" (a cudaStream_t, NULL = legacy
 *    default stream) unless stated otherwise.  dwt_plan (dwt_plan_create) synchronises.
 *  - CUDA graphs: dwt_forward, dwt_inverse, dwt_interpolate (FP32 algorithm)
 *    and dwt_effdim only enqueue kernels on "stream"; once an ordinary call
 *    of the same shape has grown the plan's workspace they neither allocate
 *    nor synchronise, so such a call can be captured into a graph (stream
 *    capture) and replayed, with the same results.  The tensor-core
 *    algorithm, the spline calls, the host-buffer call and the serving engine
 *    allocate or synchronise and are not for capture.
 *  - Status codes are returned, never thrown.  After a failed call the outputs
 *    are unspecified and the plan stays usable, except after DWT_ECUDA, which
 *    reports a sticky CUDA error.  dwt_last_error() gives a message for the
 *    last failure of the calling thread.
 *  - The library runs every step of every call in its own CUDA kernels; it has
 *    no CPU fallback.
 */
#ifndef DWT_H
#define DWT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define DWT_OK 0
#define DWT_EINVAL 1        /* bad argument: p not prime, p^m > 2^31, entry of C >= p, s < 1, ... */
#define DWT_ESPAN 2         /* rows of C_1..C_s do not span F_p^m: some coset is empty, K(C) undefined */
#define DWT_ENOMEM 3        /* device or host allocation failed */
#define DWT_ECUDA 4         /* a CUDA call failed (message in dwt_last_error) */
#define DWT_ETIMEOUT 5      /* a bounded device-side wait expired */
#define DWT_EBUSY 6         /* serving queue full */
#define DWT_EUNSUPPORTED 7  /* valid request the library does not serve (e.g. I32 with p != 2) */

typedef enum { DWT_F32 = 0, DWT_F64 = 1, DWT_I32 = 2, DWT_C64 = 3, DWT_C128 = 4 } dwt_dtype;
typedef enum { DWT_ALGO_AUTO = 0, DWT_ALGO_BUTTERFLY = 1, DWT_ALGO_TC_SPLIT_BF16 = 2 } dwt_algo;
typedef enum { DWT_WEIGHT_NONE = 0, DWT_WEIGHT_INV_SQ_WAVENUMBER = 1 } dwt_weight;

/* plan flags */
#define DWT_PLAN_TRANSFORM_ONLY 1u  /* build no K(C) tables: forward/inverse/points/k->H only */
#define DWT_PLAN_KEEP_INDEX_MAP 2u  /* keep the coset tables needed by dwt_index_to_wavenumber */
#define DWT_PLAN_TUNE 4u            /* measure the plan's launch choices (see dwt_plan), keep the fastest */

typedef struct dwt_plan_s *dwt_plan_t;

/*
 * dwt_plan: build a plan for the digital net P(C) of Def. 1.1 (eq. defy).
 *   p: prime, 2 <= p <= 31;  m >= 1 with p^m <= 2^31;  1 <= s <= 255.
 *   C: HOST array uint8 [s][m][m], C[j][i][c] in 0..p-1.  Row i of C_j gives
 *      the point digit y_{j,n,i+1}; column c multiplies the index digit n_c.
 *   flags: DWT_PLAN_* bits.
 * Unless DWT_PLAN_TRANSFORM_ONLY is set, the plan computes on the device the
 * coset representatives k(H) of K(C) (Sec. 2.1) and keeps two tables per H:
 * the weight W[H] = prod_j (1 + k_j(H))^-2 as FP32, rounded as
 * RN_f32(1 / RN_f32(prod_j (1+k_j)^2)) from the exact integer product, and the
 * class (max{j : k_j != 0} counted from 1, #{j : k_j != 0}).
 * Returns DWT_ESPAN (plan still created, transform calls allowed) when the
 * rows of C do not span F_p^m, DWT_EUNSUPPORTED (plan still created) when a
 * least nu reaches 255 or a weight denominator exceeds 64 bits.  On any other
 * failure *plan is NULL.  Synchronises "stream".
 * DWT_PLAN_TUNE: the digits of the transform may be grouped into passes in
 * any way (Sec. 2.2); with this flag the plan times, on scratch functions of N
 * points in the FP32 form (real in, complex out for p > 2), for
 * N (4 + element size) <= 1 GiB, and keeps the fastest of:
 *   - the grouping of the generic passes (used for p > 2, and for p = 2
 *     outside 12 <= m <= 14, 16 <= m <= 24) and the functions per group of
 *     those passes (16, 48 or 128 MB of functions kept in L2 between the
 *     passes of a group, or 1 GB: each pass over the whole batch at once);
 *   - p = 2, 16 <= m <= 19: the digits of the register-tile low pass;
 *   - p = 2, m = 14 or 18 <= m <= 24: whether DWT_ALGO_AUTO runs the
 *     split-BF16 tensor-core form (results then differ from the butterflies'
 *     by rounding, within the same tolerance).
 * dwt_plan_tuned reports the choices.  Results are kept per process and per
 * device, and appended to the file named by the environment variable
 * DWT_TUNE_CACHE when it is set (one JSON object per line), from which later
 * processes read them instead of measuring again.
 */
int dwt_plan(int p, int m, int s, const uint8_t *C, unsigned flags, void *stream, dwt_plan_t *plan);
/* The same call under its earlier name (identical arguments and behaviour). */
int dwt_plan_create(int p, int m, int s, const uint8_t *C, unsigned flags, void *stream, dwt_plan_t *plan);

/* Free a plan and its device tables (synchronises the device). NULL is ignored. */
int dwt_plan_destroy(dwt_plan_t plan);

/* Free a plan without synchronising: its device memory is released in stream
 * order on "stream" (cudaFreeAsync).  The caller guarantees that all work that
 * uses the plan is ordered before that point on "stream".  Plans are built
 * with stream-ordered allocations, so concurrent streams that build, use and
 * free their own plans never wait for one another. */
int dwt_plan_destroy_async(dwt_plan_t plan, void *stream);

/* Plan facts: p, m, s, N, and the status of its coset tables (DWT_OK,
 * DWT_ESPAN, DWT_EUNSUPPORTED, or -1 when built with TRANSFORM_ONLY). Any
 * output pointer may be NULL. */
int dwt_plan_info(dwt_plan_t plan, int *p, int *m, int *s, long long *N, int *tables_status);

/* The digit split of the generic passes for elements of elem_bytes (4: FP32
 * or int32, 8: complex FP32 or FP64, 16: complex FP64): *q passes, digits[t]
 * digits and wc[t] columns (consecutive low indices per row) in pass t, from
 * the lowest digits up.  digits and wc: host int [32]. */
int dwt_plan_passes(dwt_plan_t plan, int elem_bytes, int *q, int *digits, int *wc);

/* The measured choices of a DWT_PLAN_TUNE plan (0 where the heuristic stays):
 * *lo_digits = digits of the p = 2 register-tile low pass, *tc = 1 when
 * DWT_ALGO_AUTO runs the tensor-core form, *group_bytes = bytes of functions
 * per L2-resident group of the generic passes.  Any pointer may be NULL. */
int dwt_plan_tuned(dwt_plan_t plan, int *lo_digits, int *tc, long long *group_bytes);

/* The heuristic split that dwt_plan_create gives a plan (before any tuning),
 * computed on the host without a device: fewest passes within the 64 KB tile
 * budget, then the widest rows of the narrowest high pass, then the longest
 * low pass; high-pass rows halve (down to 64 bytes) while a function has
 * fewer than min_tiles tiles (a plan uses two per SM).  Outputs as above. */
int dwt_pass_plan_for(int p, int m, int elem_bytes, long long min_tiles, int *q, int *digits, int *wc);

/* Device pointers to the plan's tables: W[N] (float) and cls[N][2] (uint8, max
 * support then support size).  Owned by the plan; valid until destroy. */
int dwt_plan_tables(dwt_plan_t plan, const float **W, const uint8_t **cls);

/*
 * Net points of Def. 1.1: Y[j*ldY + n] = sum_{i=1}^m y_{j,n,i} p^{m-i}
 * (uint32, device [s][ldY], ldY >= N), so x_{j,n} = Y / p^m exactly.
 */
int dwt_points(dwt_plan_t plan, uint32_t *Y, long long ldY, void *stream);

/*
 * Coset label of wavenumber vectors (Sec. 2.1): H = C . k = sum_j C_j^T k_j^{(m)}
 * over F_p, digits of k_j at positions >= m dropped.
 *   k: device uint32 [cnt][s];  H: device uint32 [cnt].
 */
int dwt_wavenumber_to_index(dwt_plan_t plan, const uint32_t *k, uint32_t *H, long long cnt, void *stream);

/*
 * Representative k(H) in K(C) of each coset label (Sec. 2.1).
 *   H: device uint32 [cnt], each < N;  k: device uint32 [cnt][s].
 * Needs a plan built with DWT_PLAN_KEEP_INDEX_MAP (else DWT_EUNSUPPORTED).
 */
int dwt_index_to_wavenumber(dwt_plan_t plan, const uint32_t *H, uint32_t *k, long long cnt, void *stream);

/*
 * Forward transform, Algorithm 1 with eq. (fdwt):
 *   out[H] = f~(H) = p^{-m} sum_n in[n] omega^{-(n . h)},  omega = e^{2 pi i / p},
 * for each of "batch" functions (in at in + b*ld_in, out at out + b*ld_out).
 * Output in natural H order; in == out (same ld) is allowed when the element
 * sizes agree.  Types:
 *   p = 2: in_t = out_t = DWT_F32 or DWT_F64; or DWT_I32 -> DWT_I32, which
 *          returns G^{(m)} without the factor 2^{-m} (exact; the caller keeps
 *          N * max|in| < 2^31).
 *   p > 2: in_t DWT_F32 (real) or DWT_C64 -> out_t DWT_C64; in_t DWT_F64 or
 *          DWT_C128 -> out_t DWT_C128.
 * algo: DWT_ALGO_TC_SPLIT_BF16 (p = 2, F32 only) runs the Hadamard stages as
 * tensor-core tile products on hi/lo BF16 splits with FP32 accumulation.
 */
int dwt_forward(dwt_plan_t plan, const void *in, void *out, int batch, long long ld_in, long long ld_out,
                dwt_dtype in_t, dwt_dtype out_t, dwt_algo algo, void *stream);

/*
 * Inverse transform, Algorithm 2 (Lemma 3.1):
 *   out[n] = c_n = sum_H in[H] omega^{+(h . n)}   (no factor),
 * so dwt_inverse(dwt_forward(f)) = f.  Types as for dwt_forward, except that
 * for p > 2 the input is complex (DWT_C64 or DWT_C128) and so is the output;
 * for DWT_I32 the result is D^{(m)} (forward then inverse gives N * f).
 */
int dwt_inverse(dwt_plan_t plan, const void *in, void *out, int batch, long long ld_in, long long ld_out,
                dwt_dtype in_t, dwt_dtype out_t, dwt_algo algo, void *stream);

/*
 * Grouped transforms: the dwt_forward (dwt_inverse) calls of njobs jobs, with
 * nets of different sizes, in few launches.  Job i is the call
 *   dwt_forward(jobs[i].plan, jobs[i].in, jobs[i].out, jobs[i].batch,
 *               jobs[i].ld_in, jobs[i].ld_out, in_t, out_t, DWT_ALGO_AUTO, stream)
 * (Algorithm 1 / Algorithm 2 per job, same layout, types and in-place rules),
 * and every output element is bit-identical to that call's.  All plans share
 * p; in_t / out_t apply to every job.  The jobs' passes run as one launch per
 * pass index (the generic passes of every prime), and p = 2 F32 / I32 jobs of
 * 2^12 .. 2^14 points as one launch per size; p = 2 F32 / I32 jobs of
 * 2^16 .. 2^24 points, which fill the GPU alone, run their own launches.
 * Jobs with batch 0 are skipped.  The host array is read before return.
 * Errors: DWT_EINVAL (NULL or empty list, a bad job, mixed p, more than
 * 2^31 - 1 blocks in one pass), DWT_EUNSUPPORTED (types), DWT_ENOMEM.
 */
typedef struct dwt_job {
    dwt_plan_t plan;
    const void *in;
    void *out;
    int batch;
    long long ld_in;
    long long ld_out;
} dwt_job;

int dwt_forward_grouped(const dwt_job *jobs, int njobs, dwt_dtype in_t, dwt_dtype out_t, void *stream);
int dwt_inverse_grouped(const dwt_job *jobs, int njobs, dwt_dtype in_t, dwt_dtype out_t, void *stream);

/*
 * dwt_forward_digits / dwt_inverse_digits: the stages of Algorithm 1
 * (Algorithm 2) for the index digits d0 .. d0+nd-1 only, 0 <= d0,
 * d0 + nd <= m.  The transform is the Kronecker product of one p-point DFT per
 * digit (Sec. 2.2, the nested-sum form of eq. fdwt), and the stages of
 * different digits commute, so the stages of any partition of the digits,
 * applied in any order, compose to dwt_forward (dwt_inverse).  The forward
 * applies the factor p^-nd (none for I32); the inverse none.  Layout, types
 * and in-place use as dwt_forward / dwt_inverse (the generic passes only: no
 * tensor-core form).  This is the building block of a transform split across
 * processes: the digits below a cut on every process, one all-to-all exchange,
 * then the digits above the cut.
 */
int dwt_forward_digits(dwt_plan_t plan, const void *in, void *out, int batch, long long ld_in, long long ld_out,
                       dwt_dtype in_t, dwt_dtype out_t, int d0, int nd, void *stream);
int dwt_inverse_digits(dwt_plan_t plan, const void *in, void *out, int batch, long long ld_in, long long ld_out,
                       dwt_dtype in_t, dwt_dtype out_t, int d0, int nd, void *stream);

/*
 * Spectral weighting and effective dimension in one call (Sec. 3.2-3.3, Sec. 4):
 *   f~ = forward(f);  g(H) = w(H) f~(H);  c = inverse(g);
 *   var[b][0][d] = sum_{H != 0, max supp k(H) <= d} |g(H)|^2,
 *   var[b][1][d] = sum_{H != 0, |supp k(H)| <= d} |g(H)|^2,   d = 0..s,
 *   dim[b][0] = least d with var[b][0][d] >= threshold * var[b][0][s] (0 if that is 0),
 *   dim[b][1] = the same with var[b][1].
 * The weight w is 1 (DWT_WEIGHT_NONE: then c = f, the interpolation property)
 * or the plan's W[H] (DWT_WEIGHT_INV_SQ_WAVENUMBER).  The variances of the
 * finite Walsh series sum_H g(H) wal_{k(H)} split by ANOVA support exactly so.
 *   f: device, ld elements per function, type f_t (p = 2: DWT_F32;
 *      p > 2: DWT_F32 real input or DWT_C64);
 *   c: device output, ld elements per function (p = 2: float, p > 2: complex
 *      float); may equal f when the element sizes agree;
 *   coef: optional device output of g (same layout as c), or NULL;
 *   var: optional device double [batch][2][s+1], or NULL;
 *   dim: optional device int [batch][2], or NULL;
 *   threshold: in (0, 1], 0.99 in the paper.
 *   algo: DWT_ALGO_AUTO / DWT_ALGO_BUTTERFLY (FP32 stages), or
 *      DWT_ALGO_TC_SPLIT_BF16 for p = 2, 18 <= m <= 24 and 16-byte aligned
 *      rows: the low 14 digits of both transforms on the tensor cores (error
 *      relative to the norm of f about 4e-6); this form checks its bounded
 *      device waits before returning, so the call synchronises `stream`
 *      (DWT_ETIMEOUT if a wait expired), DWT_EUNSUPPORTED for other shapes.
 * Variance sums use per-lane FP32 partials inside a tile, then FP64 in a
 * fixed order, so results do not depend on scheduling.  Needs plan tables
 * (DWT_ESPAN / DWT_EUNSUPPORTED otherwise).
 */
int dwt_interpolate(dwt_plan_t plan, const void *f, void *c, void *coef, int batch, long long ld,
                    dwt_dtype f_t, dwt_weight weight, dwt_algo algo, double *var, int *dim,
                    double threshold, void *stream);

/*
 * dwt_interpolate on host-resident data: the same results as copying f to the
 * device, calling dwt_interpolate and copying c, var and dim back, with the
 * copies of one chunk of functions overlapped with the transforms of the next.
 *   f: host, ld elements per function, type as for dwt_interpolate;
 *   c: host output, ld elements per function (p = 2: float; p > 2: complex float);
 *   var: optional host double [batch][2][s+1], or NULL;
 *   dim: optional host int [batch][2], or NULL.
 * Asynchronous like cudaMemcpyAsync: every copy and kernel is ordered on
 * `stream` (two further streams of the plan carry the copies), so f, c, var
 * and dim must stay valid until that stream has been synchronised.  Page-locked
 * host buffers (cudaHostAlloc / cudaHostRegister) let the copies overlap with
 * the computation; pageable buffers give the same results without overlap.
 * The plan keeps three device slots of about 64 MiB of samples each (at least
 * one function) from the first call until it is destroyed; calls on one plan
 * must be issued from one stream or serialised by the caller.
 * No counterpart in the paper: a transport of its interpolation step.
 */
int dwt_interpolate_host(dwt_plan_t plan, const void *f, void *c, int batch, long long ld, dwt_dtype f_t,
                         dwt_weight weight, double *var, int *dim, double threshold, void *stream);

/*
 * The kernel spline of Sec. 3.1 and the variances of its ANOVA effects
 * (Sec. 4), in FP64.  The kernel is K(x, y) = prod_j (1 + gamma_j K'(x_j (-) y_j, 0))
 * with the univariate K' of Sec. 4 (Walsh coefficients proportional to
 * p^{-alpha a} for wavenumbers with top digit a), evaluated by its short form.
 *
 * dwt_spline_prepare(plan, alpha, gamma, stream): alpha > 1; gamma: host
 * double [s], entries >= 0 (the paper takes gamma_j = beta j^q).  Builds in
 * the plan the kernel data at the net points and its DWT K~, the spline weight
 * W_K = 1 / (p^m K~) (eq. splinecoef), and the DWTs of R_d = prod_{j<=d}
 * (1 + gamma_j^2 R') and of the degree-j parts E_j of R_s (the tables of the
 * truncation and superposition variances): (1 + 2s) N doubles, s <= 64.  Works
 * on any plan (the coset tables are not used).  Replaces earlier tables; runs
 * in the order of `stream`.
 *
 * dwt_spline(plan, f, c, batch, ld, var_trc, var_sup, dim, threshold, stream):
 *   f: device double [batch][ld], the function at the net points;
 *   c: device output [batch][ld] of the spline coefficients c_n
 *      (sum_v c_v K(x_n (-) x_v, 0) = f(x_n)): double for p = 2, complex double
 *      (interleaved) for p > 2, whose imaginary parts are rounding; or NULL;
 *   var_trc, var_sup: optional device double [batch][s+1]:
 *      var_trc[d] = sum over nonempty u within 1..d of sigma^2((Sf)_u),
 *      var_sup[d] = sum over 0 < |u| <= d of sigma^2((Sf)_u)   (eq. sig2sfu);
 *   dim: optional device int [batch][2], d_trc and d_sup at `threshold`.
 * c~ = f~ W_K divides by K~, which is small at high H: the coefficients are as
 * well conditioned as that quotient (relative error about
 * 1e-16 max|K(x_n, 0)| / min|K~|).  DWT_EINVAL without dwt_spline_prepare.
 * No counterpart in the paper for the superposition route: the degree-j
 * tables come from the elementary symmetric polynomials of the per-coordinate
 * terms instead of the interpolation in beta^2 of Sec. 4 (same quantities).
 */
int dwt_spline_prepare(dwt_plan_t plan, double alpha, const double *gamma, void *stream);
int dwt_spline(dwt_plan_t plan, const double *f, void *c, int batch, long long ld, double *var_trc,
               double *var_sup, int *dim, double threshold, void *stream);

/*
 * Values of the spline Sf(x) = sum_v c_v K(x (-) x_v, 0) at the digitally
 * shifted points x_n (+) delta, n = 0..N-1 (Sec. 3.1; for p = 2 and
 * delta = x_N of a 2N-point net whose halves are nets these are the hold-out
 * points of the cost function of Sec. 5.1).  As a function of n the values are
 * a convolution over the net, so their DWT is p^m c~ k~ with k~ the DWT of the
 * shifted kernel data K(x_w (+) delta, 0): O(N log N) per function.
 *   c: device spline coefficients [batch][ld] from dwt_spline (double for
 *      p = 2, complex double for p > 2);
 *   delta: host uint32 [s], delta_j = delta[j] / p^M, with m <= M and
 *      p^M <= 2^32 (M = m + 1 for the second half of a 2N-point net);
 *   values: device output [batch][ld], same type as c;
 *   f_shift, sse: optional; with both, sse[b] (device double [batch]) =
 *      sum_n (f_shift[b][n] - Re values[b][n])^2, f_shift device double [batch][ld]
 *      (the function at the shifted points): the cost of eq. splineCostFunc.
 * Uses the kernel of the last dwt_spline_prepare (DWT_EINVAL without one).
 */
int dwt_spline_values_shifted(dwt_plan_t plan, const void *c, const uint32_t *delta, int M, void *values,
                              int batch, long long ld, const double *f_shift, double *sse, void *stream);

/*
 * The spline at arbitrary points (Sec. 3.1): for each function b and point q,
 *   values[b][q] = sum_n Re c[b][n] K(x_q (-) x_n, 0),
 *   K(x, 0) = prod_j (1 + gamma_j K'(x_j, 0)), K' by its short form (Sec. 4)
 * on M digits: it depends only on the first base-p digit where x_{q,j} and
 * x_{j,n} differ (or, when their top m digits agree, the first nonzero digit
 * of x_{q,j} below them).  A direct sum over the net, O(N s) per point and
 * function, FP64.
 *   c: device spline coefficients [batch][ld] from dwt_spline (double for
 *      p = 2, complex double for p > 2, whose real parts are used);
 *   X: device uint32 [Q][s], x_{q,j} = X[q][j] / p^M, m <= M, p^M <= 2^32
 *      (entries are read modulo p^M);
 *   values: device double output [batch][ldv], ldv >= Q.
 * The net is split into chunks summed by separate blocks; the chunk sums are
 * added in chunk order, so results are reproducible for a given device.
 * Uses the kernel of the last dwt_spline_prepare (DWT_EINVAL without one);
 * DWT_EINVAL for M < m or p^M > 2^32.  Allocates its scratch (12 s N bytes
 * plus the chunk sums) in stream order.
 */
int dwt_spline_eval(dwt_plan_t plan, const void *c, int batch, long long ld, const uint32_t *X, int Q, int M,
                    double *values, long long ldv, void *stream);

/*
 * Effective dimension of given coefficients g (Sec. 4), the variance and
 * threshold part of dwt_interpolate alone.  g defines the finite Walsh series
 * sum_H g(H) wal_{k(H)}; its ANOVA effect u collects the H with supp k(H) = u
 * and has variance sum |g(H)|^2 over them (H != 0).
 *   coef: device, DWT_F32 (p = 2) or DWT_C64 (p > 2), ld elements per function.
 *   var_trc, var_sup: device double [batch][s+1] or NULL:
 *     var_trc[b][d] = sum over H != 0 with max{j : k_j != 0} <= d of |g|^2
 *     (the truncation variance), var_sup[b][d] the same over |supp k| <= d
 *     (the superposition variance).
 *   d_trc, d_sup: device int [batch] or NULL: the least d with
 *     var(d) >= threshold * var(s) (threshold in (0, 1], the paper uses 0.99),
 *     0 when the total variance is 0.
 */
int dwt_effdim(dwt_plan_t plan, const void *coef, int batch, long long ld, dwt_dtype t, double *var_trc,
               double *var_sup, int *d_trc, int *d_sup, double threshold, void *stream);

/*
 * dwt_effdim with the packed outputs of dwt_interpolate: var device double
 * [batch][2][s+1] (truncation, then superposition), dim device int [batch][2]
 * (d_trc, d_sup); either may be NULL.
 */
int dwt_effdim_packed(dwt_plan_t plan, const void *coef, int batch, long long ld, dwt_dtype t, double *var,
                      int *dim, double threshold, void *stream);

/*
 * dwt_effdim_static: dwt_effdim that allocates nothing.  (The paper has no
 * counterpart; this is a service of the library.)
 * For callers that must not have the library allocate device memory: a host
 * program that hands out its whole device-memory budget itself and forbids
 * any later cudaMalloc, or a latency-critical loop that cannot absorb the
 * device-wide synchronisation that cudaMalloc / cudaFree may cause.
 * dwt_effdim keeps its per-tile class partials in a workspace that the plan
 * grows with cudaMalloc; this call keeps them in one fixed 8 MiB array
 * compiled into the library (every GPU that loads the library holds it until
 * the process exits), and calls no allocating routine.
 * Arguments, results and tolerance are those of dwt_effdim_packed.
 * Limit: one function may need at most 2^20 partials, i.e.
 * 2 (s+1) (ceil(N / 8192) + 1) <= 1048576 (for s = 32, N <= 2^27); larger
 * requests return DWT_EINVAL with a message.  Batches go through the array in
 * groups, in stream order.
 * The first call on each device looks up the array's device address (with
 * that device current); make that first call before any stream capture.
 * All calls on a device share the one array and it keeps the last call's
 * contents (every entry a call reads it has written first, so nothing needs
 * clearing); calls whose work overlaps on the GPU (different streams, or
 * threads) race on it and must be serialised by the caller.
 */
int dwt_effdim_static(dwt_plan_t plan, const void *coef, int batch, long long ld, dwt_dtype t, double *var,
                      int *dim, double threshold, void *stream);

/*
 * Synthetic test functions at the net points (for workloads and tests):
 *   dwt_eval_product: f_b(x_n) = prod_j (1 + coef[b][j] (x_{j,n} - 1/2)),
 *     coef: device double [batch][s];
 *   dwt_eval_exp: f_b(x_n) = exp(sum_j x_{j,n} / j^2) (j from 1), every b.
 * Output f: device, DWT_F32 or DWT_F64, ld elements per function.
 */
int dwt_eval_product(dwt_plan_t plan, const double *coef, void *f, int batch, long long ld, dwt_dtype t,
                     void *stream);
int dwt_eval_exp(dwt_plan_t plan, void *f, int batch, long long ld, dwt_dtype t, void *stream);

/*
 * Serving: a continuous-batching engine.  One request is a complete job of the
 * method on its own net: build the plan of (p, m, s, C), sample the product
 * test function f(x) = prod_j (1 + coef[j] (x_j - 1/2)) on it, and run
 * dwt_interpolate (forward, weight, class variances / effective dimensions,
 * inverse).  Requests queue FIFO; "slots" worker threads, one CUDA stream
 * each, admit the head of the queue as soon as a slot is idle and its device
 * footprint fits the budget left, so requests that arrive while others run
 * are started as slots and memory free up, and their work overlaps on the GPU.
 * All device memory on that path is stream-ordered (no device-wide sync).
 */
typedef struct dwt_server_s *dwt_server_t;

typedef struct {
    int p, m, s;            /* the net */
    const uint8_t *C;       /* host [s][m][m], copied at submit */
    const double *coef;     /* host [s] product-function coefficients, copied at submit */
    int weight;             /* dwt_weight */
    double threshold;       /* effective-dimension threshold, e.g. 0.99 */
    float *c_out;           /* optional host output for c (N floats for p = 2, 2N for p > 2),
                               written before the request completes; NULL = not returned */
} dwt_request;

typedef struct {
    int status;             /* DWT_OK or the error of the request */
    int s;
    int d_trc, d_sup;
    double var_trc[256];    /* cumulative, entries 0..s */
    double var_sup[256];
    double t_submit, t_admit, t_plan, t_done;   /* seconds since server creation */
    char message[160];      /* error message when status != DWT_OK */
} dwt_result;

/* hbm_budget_bytes: device bytes the admitted requests may hold together
 * (0 = half the free memory); slots: concurrent requests (1..64);
 * max_queue: queued requests before dwt_server_submit returns DWT_EBUSY. */
int dwt_server_create(size_t hbm_budget_bytes, int slots, int max_queue, dwt_server_t *server);
/* Queue a request; *ticket identifies it.  DWT_EBUSY: queue full; DWT_ENOMEM:
 * the request alone exceeds the budget; DWT_EINVAL: bad shape. */
int dwt_server_submit(dwt_server_t server, const dwt_request *req, unsigned long long *ticket);
/* DWT_OK and *res when done (the ticket is then forgotten), DWT_EBUSY while pending. */
int dwt_server_poll(dwt_server_t server, unsigned long long ticket, dwt_result *res);
/* Block until done or timeout_s seconds pass (DWT_ETIMEOUT). */
int dwt_server_wait(dwt_server_t server, unsigned long long ticket, double timeout_s, dwt_result *res);
/* Queue length, device bytes held by admitted requests, server clock. */
int dwt_server_stats(dwt_server_t server, long long *queued, size_t *bytes_in_use, double *now_s);
/* Finish every queued request, then stop the workers and free the server. */
int dwt_server_destroy(dwt_server_t server);

/* Messages. */
const char *dwt_strerror(int status);
const char *dwt_last_error(void);

/*
 * Self-test of the bounded device waits: launches one CTA that waits on an
 * mbarrier phase that never completes, with the same bounded wait as the
 * tensor-core kernels (a few hundred tries of at most 1 us).  Returns
 * DWT_ETIMEOUT (with a message) when the wait gave up as designed, after
 * synchronising `stream`; the context stays usable.  No counterpart in the
 * paper: it checks the failure path of the library's own device waits.
 */
int dwt_selftest_bounded_wait(void *stream);

/* Number of kernels this library has launched in this process. */
long long dwt_launch_count(void);

/* Number of device (and page-locked host) allocations the library has made in
 * this process, over all threads: plans, workspaces, scratch, serving slots.
 * A diagnostic, like dwt_launch_count (no counterpart in the paper). */
long long dwt_alloc_count(void);

/*
 * Optional per-kernel timing with CUDA events recorded on the launching stream
 * around every launch of this library.  dwt_profile_query synchronises on the
 * recorded events and returns, for kernel family "name", the number of
 * launches and their summed duration in milliseconds since the last reset.
 * Families: p = 2 register tiles "p2_lo_fwd", "p2_lo_inv", "p2_hi_fwd",
 * "p2_hi_inv"; p = 2 interpolation "interp_fwd", "interp_top", "interp_inv",
 * "interp_inv_fwd" (two low passes in one launch); tensor-core tiles
 * "tc_lo14"; generic passes "pass_lo", "pass_mid", "pass_hi"; variance classes
 * "effdim_bins", "effdim_classes", "effdim_finalize"; index maps "points",
 * "k_to_h", "h2k_recon", "h2k_copy"; plan build "dp_init", "dp_step",
 * "dp_check", "dp_prefix", "dp_recon", "dp_weights", "dp_small",
 * "tile_tables"; test functions "eval_product", "eval_exp".
 */
int dwt_profile_enable(int on);
int dwt_profile_reset(void);
int dwt_profile_query(const char *name, long long *launches, double *total_ms);

#ifdef __cplusplus
}
#endif
#endif /* DWT_H */
