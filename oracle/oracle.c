/*
 * oracle.c -- plain, slow, obviously correct CPU oracle for the multivariate
 * discrete Walsh transform over digital nets of K.-I. Liu, J. Dick and
 * F. J. Hickernell, "A Multivariate Fast Discrete Walsh Transform with an
 * Application to Function Interpolation".
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library.  The GPU library shares no
 * code, header, table or helper with it, and neither includes the other.
 *
 * Floating point is IEEE double throughout (complex values are carried as
 * separate real and imaginary arrays); integer work is exact.  Each function
 * names the definition, equation or algorithm of the paper that it follows.
 *
 * Conventions
 *   p is prime, m is the number of digits, s the dimension, N = p^m.
 *   Digits are least significant first: n = n_0 + n_1 p + ... + n_{m-1} p^{m-1}.
 *   Generating matrices are stored C[j][i][c] (j = 0..s-1 is the coordinate,
 *   i the row, c the column), entries in 0..p-1.  Row i yields the digit
 *   y_{j,n,i+1} of the point and column c multiplies the digit n_c of the
 *   index (Def. 1.1).
 *   A coset is named by H = h_0 + h_1 p + ... + h_{m-1} p^{m-1}, where
 *   (h_0..h_{m-1}) = C . k (Sec. 2.1).
 *
 * Parity pins for every function live in tests/test_oracle_*.py.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_ESPAN 2
#define ORC_ENOMEM 3
#define ORC_EUNSUPPORTED 7

static uint64_t ipow_u64(int p, int m)
{
    uint64_t v = 1;
    for (int i = 0; i < m; ++i) v *= (uint64_t)p;
    return v;
}

/* base-p digits of v, least significant first (Def. 1.1) */
static void to_digits(uint64_t v, int p, int m, int *d)
{
    for (int r = 0; r < m; ++r) {
        d[r] = (int)(v % (uint64_t)p);
        v /= (uint64_t)p;
    }
}

static uint64_t from_digits(const int *d, int p, int m)
{
    uint64_t v = 0;
    for (int r = m - 1; r >= 0; --r) v = v * (uint64_t)p + (uint64_t)d[r];
    return v;
}

/* omega^e = cos(2 pi e/p) + i sin(2 pi e/p) for e = 0..p-1, with the values
 * that are exactly representable (e = 0, and e = p/2 for p = 2) set exactly. */
static void unit_roots(int p, double *cw, double *sw)
{
    for (int e = 0; e < p; ++e) {
        cw[e] = cos(2.0 * M_PI * e / p);
        sw[e] = sin(2.0 * M_PI * e / p);
        if (e == 0) { cw[e] = 1.0; sw[e] = 0.0; }
        if (2 * e == p) { cw[e] = -1.0; sw[e] = 0.0; }
    }
}

/* perm[h] = h (-) a*r for every coset index h in 0..N-1 (a translation of
 * F_p^m).  Stepping h -> h+1 raises one digit by one, or wraps a run of
 * digits p-1 -> 0 and raises the next; in both cases each touched digit of
 * h (-) a*r also rises by one modulo p, which an odometer tracks.          */
static void translate_perm(uint32_t r, int a, int p, int m, uint64_t N, uint32_t *perm)
{
    int hd[32] = {0}, td[32], rd[32];
    uint64_t pw[32];
    to_digits(r, p, m, rd);
    uint64_t t = 0;
    for (int c = 0; c < m; ++c) {
        pw[c] = ipow_u64(p, c);
        td[c] = ((-a * rd[c]) % p + p) % p;
        t += (uint64_t)td[c] * pw[c];
    }
    for (uint64_t h = 0; h < N; ++h) {
        perm[h] = (uint32_t)t;
        for (int c = 0; c < m; ++c) {
            int nt = (td[c] + 1) % p;
            t = t - (uint64_t)td[c] * pw[c] + (uint64_t)nt * pw[c];
            td[c] = nt;
            if (hd[c] + 1 < p) { hd[c] += 1; break; }
            hd[c] = 0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Def. 1.1, eq. (defy): y_{j,n} = C_j n, x_{j,n} = sum_i y_{j,n,i} p^{-i}.
 * The point is returned as the integer Y_{j,n} = sum_{i=1}^m y_{j,n,i} p^{m-i},
 * so that x_{j,n} = Y_{j,n} / p^m exactly.  Y is [s][N].                      */
int orc_net_points(int p, int m, int s, const uint8_t *C, uint32_t *Y)
{
    uint64_t N = ipow_u64(p, m);
    int nd[32];
    if (p == 2) {
        /* over F_2, C_j n is the sum (XOR) of the columns c with n_c = 1 */
        for (int j = 0; j < s; ++j) {
            const uint8_t *Cj = C + (size_t)j * m * m;
            uint32_t col[32];
            for (int c = 0; c < m; ++c) {
                uint32_t v = 0;
                for (int i = 0; i < m; ++i) v |= (uint32_t)(Cj[i * m + c] & 1) << (m - 1 - i);
                col[c] = v;
            }
            for (uint64_t n = 0; n < N; ++n) {
                uint32_t v = 0;
                for (int c = 0; c < m; ++c)
                    if ((n >> c) & 1) v ^= col[c];
                Y[(size_t)j * N + n] = v;
            }
        }
        return ORC_OK;
    }
    for (int j = 0; j < s; ++j) {
        const uint8_t *Cj = C + (size_t)j * m * m;
        for (uint64_t n = 0; n < N; ++n) {
            to_digits(n, p, m, nd);
            uint64_t Yv = 0;
            for (int i = 0; i < m; ++i) {          /* row i -> digit y_{i+1} */
                int y = 0;
                for (int c = 0; c < m; ++c) y += Cj[i * m + c] * nd[c];
                y %= p;
                Yv = Yv * (uint64_t)p + (uint64_t)y; /* y_{i+1} has weight p^{m-1-i} */
            }
            Y[(size_t)j * N + n] = (uint32_t)Yv;
        }
    }
    return ORC_OK;
}

/* x_{j,n} = Y_{j,n} / p^m, correctly rounded in double (Def. 1.1) */
void orc_net_x(int p, int m, int s, const uint32_t *Y, double *x)
{
    uint64_t N = ipow_u64(p, m);
    double den = (double)N;
    for (uint64_t t = 0; t < (uint64_t)s * N; ++t) x[t] = (double)Y[t] / den;
}

/* ------------------------------------------------------------------------ */
/* Sec. 2.1: C . k = sum_j C_j^T k_j^{(m)} over F_p; digits of k_j at
 * positions >= m are dropped (the m-element truncation).  k is [cnt][s].    */
void orc_k_to_h(int p, int m, int s, const uint8_t *C, const uint32_t *k, int cnt, uint32_t *H)
{
    int kd[32];
    for (int t = 0; t < cnt; ++t) {
        int h[32] = {0};
        for (int j = 0; j < s; ++j) {
            const uint8_t *Cj = C + (size_t)j * m * m;
            to_digits(k[(size_t)t * s + j], p, m, kd);
            for (int c = 0; c < m; ++c)
                for (int i = 0; i < m; ++i) h[c] += Cj[i * m + c] * kd[i];  /* (C_j^T k)_c */
        }
        for (int c = 0; c < m; ++c) h[c] %= p;
        H[t] = (uint32_t)from_digits(h, p, m);
    }
}

/* ------------------------------------------------------------------------ */
/* Direct discrete Walsh transform (eq. dwalshcoeff together with the identity
 * wal_k(x_n) = omega^{n . h}, Sec. 2.2):
 *     f~(H) = p^{-m} sum_n f_n omega^{-(n . h mod p)},   omega = e^{2 pi i/p}.
 * O(N) per output.  Hsel lists the outputs wanted (NULL = all N, in H order). */
void orc_dwt_direct(int p, int m, const double *fre, const double *fim,
                    const uint32_t *Hsel, long nsel, double *ore, double *oim)
{
    uint64_t N = ipow_u64(p, m);
    double cw[32], sw[32];
    unit_roots(p, cw, sw);
    long nout = Hsel ? nsel : (long)N;
    for (long t = 0; t < nout; ++t) {
        uint32_t H = Hsel ? Hsel[t] : (uint32_t)t;
        int hd[32];
        to_digits(H, p, m, hd);
        double ar = 0.0, ai = 0.0;
        if (p == 2) {
            for (uint64_t n = 0; n < N; ++n) {
                double sg = (__builtin_popcountll(n & H) & 1) ? -1.0 : 1.0;
                ar += sg * fre[n];
                if (fim) ai += sg * fim[n];
            }
        } else {
            /* odometer over the digits of n, carrying e = n . h mod p */
            int nd[32] = {0};
            int e = 0;
            for (uint64_t n = 0; n < N; ++n) {
                /* f_n * omega^{-e} = f_n * (cos - i sin)(2 pi e / p) */
                double xr = fre[n], xi = fim ? fim[n] : 0.0;
                ar += xr * cw[e] + xi * sw[e];
                ai += xi * cw[e] - xr * sw[e];
                for (int r = 0; r < m; ++r) {      /* n -> n + 1 */
                    if (nd[r] + 1 < p) {
                        nd[r] += 1;
                        e = (e + hd[r]) % p;
                        break;
                    }
                    e = ((e - (p - 1) * hd[r]) % p + p) % p;
                    nd[r] = 0;
                }
            }
        }
        ore[t] = ar / (double)N;
        oim[t] = ai / (double)N;
    }
}

/* The discrete Walsh coefficient straight from the Walsh function definition
 * (Def. 1.2, Def. 1.3, eq. dwalshcoeff):
 *     f~(k) = p^{-m} sum_n f(x_n) conj(wal_k(x_n)),
 *     wal_k(x) = prod_j omega^{sum_i x_{j,i+1} k_{j,i}}.
 * The digits of x_{j,n} are read from Y (digit x_{i+1} is the base-p digit
 * m-1-i of Y).  Net points have m digits, so digits of k_j at positions >= m
 * meet zeros.  k is [cnt][s].                                               */
void orc_dwt_walsh_def(int p, int m, int s, const uint32_t *Y, const double *fre, const double *fim,
                       const uint32_t *k, long cnt, double *ore, double *oim)
{
    uint64_t N = ipow_u64(p, m);
    double cw[32], sw[32];
    unit_roots(p, cw, sw);
    int yd[32], kd[32];
    for (long t = 0; t < cnt; ++t) {
        double ar = 0.0, ai = 0.0;
        for (uint64_t n = 0; n < N; ++n) {
            int e = 0;
            for (int j = 0; j < s; ++j) {
                to_digits(Y[(size_t)j * N + n], p, m, yd);
                to_digits(k[(size_t)t * s + j], p, m, kd);
                for (int i = 0; i < m; ++i) e += yd[m - 1 - i] * kd[i];   /* x_{i+1} k_i */
            }
            e %= p;
            double xr = fre[n], xi = fim ? fim[n] : 0.0;
            /* times conj(omega^e) = omega^{-e} */
            ar += xr * cw[e] + xi * sw[e];
            ai += xi * cw[e] - xr * sw[e];
        }
        ore[t] = ar / (double)N;
        oim[t] = ai / (double)N;
    }
}

/* ------------------------------------------------------------------------ */
/* One p-point sum over digit r of an array in place: for every setting of the
 * other digits, v(.., t, ..) <- sum_u omega^{sgn * u * t} v(.., u, ..).      */
static void digit_dft(int p, int m, int r, int sgn, double *re, double *im)
{
    uint64_t N = ipow_u64(p, m);
    uint64_t stride = ipow_u64(p, r);
    double cw[32], sw[32];
    unit_roots(p, cw, sw);
    double xr[32], xi[32];
    for (uint64_t base = 0; base < N; base += stride * (uint64_t)p) {
        for (uint64_t off = 0; off < stride; ++off) {
            uint64_t i0 = base + off;
            for (int u = 0; u < p; ++u) {
                xr[u] = re[i0 + (uint64_t)u * stride];
                xi[u] = im ? im[i0 + (uint64_t)u * stride] : 0.0;
            }
            for (int t = 0; t < p; ++t) {
                double ar = 0.0, ai = 0.0;
                for (int u = 0; u < p; ++u) {
                    int e = (u * t) % p;
                    double c = cw[e], sn = sgn * sw[e];   /* omega^{sgn e} */
                    ar += xr[u] * c - xi[u] * sn;
                    ai += xr[u] * sn + xi[u] * c;
                }
                re[i0 + (uint64_t)t * stride] = ar;
                if (im) im[i0 + (uint64_t)t * stride] = ai;
            }
        }
    }
}

/* Algorithm 1 (FWT), eq. (fdwt): for r = 1..m replace digit n_{r-1} by h_{r-1}
 * with sum_{n_{r-1}} omega^{-n_{r-1} h_{r-1}} G^{(r-1)}, then f~ = p^{-m} G^{(m)}.
 * In place; the result is in natural H order.  im may be NULL only for p = 2
 * (real data stays real).                                                    */
void orc_fwt(int p, int m, double *re, double *im)
{
    for (int r = 0; r < m; ++r) digit_dft(p, m, r, -1, re, im);
    uint64_t N = ipow_u64(p, m);
    double den = (double)N;
    for (uint64_t i = 0; i < N; ++i) {
        re[i] /= den;
        if (im) im[i] /= den;
    }
}

/* Algorithm 2 (FIWT): the same stages with omega^{+h n} and no factor, so that
 * c_n = D^{(m)}(n_0..n_{m-1}) (Lemma 3.1).                                   */
void orc_fiwt(int p, int m, double *re, double *im)
{
    for (int r = 0; r < m; ++r) digit_dft(p, m, r, +1, re, im);
}

/* Algorithm 1 for p = 2 in exact 64-bit integers, without the factor 2^{-m}:
 * returns G^{(m)}.                                                           */
void orc_fwt_i64(int m, int64_t *v)
{
    uint64_t N = ipow_u64(2, m);
    for (int r = 0; r < m; ++r) {
        uint64_t stride = (uint64_t)1 << r;
        for (uint64_t base = 0; base < N; base += 2 * stride)
            for (uint64_t off = 0; off < stride; ++off) {
                int64_t a = v[base + off], b = v[base + off + stride];
                v[base + off] = a + b;            /* h = 0: omega^0 */
                v[base + off + stride] = a - b;   /* h = 1: omega^{-n} = (-1)^n */
            }
    }
}

/* Algorithm 2 for p = 2 in exact integers: D^{(m)} (no factor). */
void orc_fiwt_i64(int m, int64_t *v) { orc_fwt_i64(m, v); }

/* ------------------------------------------------------------------------ */
/* nu(k) = 1 + index of the top nonzero base-p digit, nu(0) = 0 (Sec. 2.1). */
static int nu1(uint32_t k, int p)
{
    int n = 0;
    while (k) { k /= (uint32_t)p; ++n; }
    return n;
}

/* W64 = 1/P and W32 = RN_f32(1 / RN_f32(P)) for an exact denominator P. */
static void weight_from_denominator(uint64_t P, float *W32, double *W64)
{
    float Pf;
    if (P < ((uint64_t)1 << 53)) Pf = (float)(double)P;   /* exact, then one rounding */
    else Pf = (float)P;
    volatile float one = 1.0f;
    if (W32) *W32 = one / Pf;
    if (W64) *W64 = 1.0 / (double)P;
}

/* Weight and class of one wavenumber vector k (length s):
 *   P = prod_j (1 + k_j)^2 exactly (returns -1 if it does not fit 64 bits),
 *   W64 = 1/P, W32 = RN_f32(1 / RN_f32(P)) in IEEE single arithmetic,
 *   cls = (max{j : k_j != 0} counted from 1, or 0;  #{j : k_j != 0}).
 * The spectral weight reads |k_j| of w(k) = prod_j (1+|k_j|)^{-2} as the
 * integer value of k_j for the coset representative in K(C).                */
int orc_weight_class_one(int s, const uint32_t *k, float *W32, double *W64, uint8_t *cls)
{
    uint64_t P = 1;
    int maxsupp = 0, nsupp = 0;
    for (int j = 0; j < s; ++j) {
        uint64_t q = (uint64_t)k[j] + 1u;
        if (q > UINT64_MAX / q) return -1;
        uint64_t q2 = q * q;
        if (P > UINT64_MAX / q2) return -1;
        P *= q2;
        if (k[j]) { maxsupp = j + 1; ++nsupp; }
    }
    weight_from_denominator(P, W32, W64);
    if (cls) { cls[0] = (uint8_t)maxsupp; cls[1] = (uint8_t)nsupp; }
    return 0;
}

int orc_weight_class(int s, const uint32_t *k, long cnt, float *W32, double *W64, uint8_t *cls)
{
    for (long t = 0; t < cnt; ++t)
        if (orc_weight_class_one(s, k + (size_t)t * s, W32 ? W32 + t : NULL, W64 ? W64 + t : NULL,
                                 cls ? cls + 2 * t : NULL))
            return ORC_EUNSUPPORTED;
    return ORC_OK;
}

/* Rank over F_p of the s*m rows of C_1..C_s (rows are vectors of F_p^m).  The
 * cosets D(h) of Sec. 2.1 are all nonempty exactly when the rank is m.       */
static int inv_mod(int a, int p)
{
    int r = 1;
    for (int e = 0; e < p - 2; ++e) r = (r * a) % p;   /* a^{p-2} */
    return r;
}

int orc_rank(int p, int m, int s, const uint8_t *C)
{
    int rows = s * m;
    int *A = (int *)malloc(sizeof(int) * rows * m);
    if (!A) return -1;
    for (int t = 0; t < rows * m; ++t) A[t] = C[t] % p;
    int rank = 0;
    for (int c = 0; c < m && rank < rows; ++c) {
        int piv = -1;
        for (int r = rank; r < rows; ++r)
            if (A[r * m + c]) { piv = r; break; }
        if (piv < 0) continue;
        for (int t = 0; t < m; ++t) {
            int tmp = A[rank * m + t]; A[rank * m + t] = A[piv * m + t]; A[piv * m + t] = tmp;
        }
        int iv = inv_mod(A[rank * m + c], p);
        for (int t = 0; t < m; ++t) A[rank * m + t] = (A[rank * m + t] * iv) % p;
        for (int r = 0; r < rows; ++r) {
            if (r == rank || !A[r * m + c]) continue;
            int f = A[r * m + c];
            for (int t = 0; t < m; ++t) A[r * m + t] = ((A[r * m + t] - f * A[rank * m + t]) % p + p) % p;
        }
        ++rank;
    }
    free(A);
    return rank;
}

/* ------------------------------------------------------------------------ */
/* K(C) by brute force (Sec. 2.1): enumerate every k in [0, p^m)^s, and keep for
 * each coset h the k of smallest nu(k), ties going to the lexicographically
 * smallest (k_1, ..., k_s) compared as integers.  Digits of k_j at positions
 * >= m only add to nu, so no larger k_j can be a representative.
 * kmap is [N][s].  Feasible for p^{m s} up to about 10^7.                   */
int orc_coset_leaders_bruteforce(int p, int m, int s, const uint8_t *C, uint32_t *kmap)
{
    uint64_t N = ipow_u64(p, m);
    int *best = (int *)malloc(sizeof(int) * N);
    if (!best) return ORC_ENOMEM;
    for (uint64_t h = 0; h < N; ++h) best[h] = -1;
    uint32_t k[64];
    for (int j = 0; j < s; ++j) k[j] = 0;
    for (;;) {
        uint32_t H;
        orc_k_to_h(p, m, s, C, k, 1, &H);
        int nu = 0;
        for (int j = 0; j < s; ++j) nu += nu1(k[j], p);
        int better = 0;
        if (best[H] < 0 || nu < best[H]) better = 1;
        else if (nu == best[H]) {
            for (int j = 0; j < s; ++j) {
                uint32_t cur = kmap[(size_t)H * s + j];
                if (k[j] != cur) { better = k[j] < cur; break; }
            }
        }
        if (better) {
            best[H] = nu;
            for (int j = 0; j < s; ++j) kmap[(size_t)H * s + j] = k[j];
        }
        /* next k: odometer with k_s least significant */
        int j = s - 1;
        while (j >= 0) {
            if (k[j] + 1 < N) { k[j] += 1; break; }
            k[j] = 0;
            --j;
        }
        if (j < 0) break;
    }
    int status = ORC_OK;
    for (uint64_t h = 0; h < N; ++h)
        if (best[h] < 0) status = ORC_ESPAN;
    free(best);
    return status;
}

/* ------------------------------------------------------------------------ */
/* K(C) for any size by dynamic programming over the coordinates (Sec. 2.1).
 *
 * For coordinate j (0-based) let T_j[h] be the least nu(k_j) + ... + nu(k_{s-1})
 * over wavenumbers of coordinates j..s-1 with image h under C; T_s[h] is 0 for
 * h = 0 and infinite otherwise.  With R_{j,i} the coset index of row i of C_j
 * (so that k_j contributes sum_i k_{j,i} R_{j,i}), a k_j with nu(k_j) = d has a
 * nonzero digit at d-1 and free digits below, hence
 *     M_{j,0} = T_{j+1},   M_{j,i+1}[h] = min_{a in F_p} M_{j,i}[h (-) a R_{j,i}],
 *     E_{j,d}[h] = min_{a != 0} M_{j,d-1}[h (-) a R_{j,d-1}],
 *     T_j[h] = min(T_{j+1}[h], min_d (d + E_{j,d}[h])).
 * T_0[h] is the least nu over the coset.  The representative is then read off
 * coordinate by coordinate: among all completions that reach the least nu,
 * take the smallest integer k_j (k_j = 0 if possible, else the smallest d,
 * then the smallest digits from the top down), exactly the lexicographic
 * tie-break of Sec. 2.1.
 *
 * Values are bytes with 255 standing for "unreachable or >= 255"; a saturated
 * entry exceeds every least nu below 255, so it never lies on an optimal path.
 *
 * Outputs (any may be NULL): numin[N] (least nu), kmap[N][s], W32[N], W64[N],
 * cls[N][2] (see orc_weight_class_one), and for the nsel indices Hsel the
 * vectors ksel[nsel][s].
 * Returns ORC_ESPAN if some coset is empty (rank < m), ORC_EUNSUPPORTED if a
 * least nu reaches 255 or a weight denominator overflows 64 bits.           */
int orc_coset_leaders_dp(int p, int m, int s, const uint8_t *C,
                         uint8_t *numin, uint32_t *kmap, float *W32, double *W64, uint8_t *cls,
                         const uint32_t *Hsel, long nsel, uint32_t *ksel)
{
    const uint8_t INF = 255;
    uint64_t N = ipow_u64(p, m);
    if (orc_rank(p, m, s, C) < m) return ORC_ESPAN;

    uint32_t *R = (uint32_t *)malloc(sizeof(uint32_t) * s * m);
    uint8_t *T = (uint8_t *)malloc((size_t)(s + 1) * N);
    uint8_t *M = (uint8_t *)malloc((size_t)m * N);
    uint8_t *Mn = (uint8_t *)malloc((size_t)N);
    uint32_t *g = (uint32_t *)malloc(sizeof(uint32_t) * N);
    uint32_t *kj = (uint32_t *)malloc(sizeof(uint32_t) * N);
    uint32_t *kall = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(nsel > 0 ? nsel : 1) * s);
    /* translations h -> h (-) a R_{j,i} of the current coordinate, for p > 2 */
    uint32_t *Tr = p > 2 ? (uint32_t *)malloc(sizeof(uint32_t) * (size_t)m * (p - 1) * N) : NULL;
    uint64_t *Pw = (uint64_t *)malloc(sizeof(uint64_t) * N);
    uint8_t *mx = (uint8_t *)calloc(N, 1), *ns = (uint8_t *)calloc(N, 1);
    int status = ORC_OK;
    if (!R || !T || !M || !Mn || !g || !kj || !kall || (p > 2 && !Tr) || !Pw || !mx || !ns) {
        status = ORC_ENOMEM;
        goto done;
    }
    for (int j = 0; j < s; ++j)
        for (int i = 0; i < m; ++i) {
            int d[32];
            for (int c = 0; c < m; ++c) d[c] = C[((size_t)j * m + i) * m + c];
            R[j * m + i] = (uint32_t)from_digits(d, p, m);
        }
#define SUB(h, i, a) (p == 2 ? ((h) ^ R[j * m + (i)]) : Tr[((size_t)(i) * (p - 1) + (a) - 1) * N + (h)])
#define BUILD_TRANSLATIONS(j)                                                                   \
    if (p > 2)                                                                                  \
        for (int i_ = 0; i_ < m; ++i_)                                                          \
            for (int a_ = 1; a_ < p; ++a_)                                                      \
                translate_perm(R[(j) * m + i_], a_, p, m, N, Tr + ((size_t)i_ * (p - 1) + a_ - 1) * N);

    /* backward sweep: T_s, then T_{s-1} .. T_0 */
    uint8_t *Ts = T + (size_t)s * N;
    for (uint64_t h = 0; h < N; ++h) Ts[h] = h == 0 ? 0 : INF;
    for (int j = s - 1; j >= 0; --j) {
        uint8_t *Tj = T + (size_t)j * N, *Tn = T + (size_t)(j + 1) * N;
        BUILD_TRANSLATIONS(j)
        memcpy(Tj, Tn, N);                 /* k_j = 0 */
        memcpy(M, Tn, N);                  /* M_{j,0} */
        for (int i = 0; i < m; ++i) {      /* candidate nu(k_j) = d = i + 1 */
            for (uint64_t h = 0; h < N; ++h) {
                uint8_t e = INF;
                for (int a = 1; a < p; ++a) {
                    uint8_t v = M[SUB((uint32_t)h, i, a)];
                    if (v < e) e = v;
                }
                Mn[h] = e < M[h] ? e : M[h];
                unsigned cand = e == INF ? INF : (unsigned)e + (unsigned)(i + 1);
                if (cand > INF) cand = INF;
                if (cand < Tj[h]) Tj[h] = (uint8_t)cand;
            }
            memcpy(M, Mn, N);
        }
    }
    for (uint64_t h = 0; h < N; ++h) {
        if (T[h] == INF) status = ORC_EUNSUPPORTED;
        if (numin) numin[h] = T[h];
    }
    if (status != ORC_OK) goto done;

    /* forward reconstruction: coordinates 0 .. s-1 in turn */
    for (uint64_t h = 0; h < N; ++h) { g[h] = (uint32_t)h; Pw[h] = 1; }
    for (int j = 0; j < s; ++j) {
        uint8_t *Tj = T + (size_t)j * N, *Tn = T + (size_t)(j + 1) * N;
        BUILD_TRANSLATIONS(j)
        /* M_{j,0..m-1} from T_{j+1} */
        memcpy(M, Tn, N);
        for (int i = 1; i < m; ++i) {
            uint8_t *Mi = M + (size_t)i * N, *Mp = M + (size_t)(i - 1) * N;
            for (uint64_t h = 0; h < N; ++h) {
                uint8_t v = Mp[h];
                for (int a = 1; a < p; ++a) {
                    uint8_t w = Mp[SUB((uint32_t)h, i - 1, a)];
                    if (w < v) v = w;
                }
                Mi[h] = v;
            }
        }
        for (uint64_t H = 0; H < N; ++H) {
            uint32_t gg = g[H];
            unsigned tau = Tj[gg];
            uint32_t k = 0;
            if (Tn[gg] != tau) {
                int d = 0;
                for (int dd = 1; dd <= m && !d; ++dd) {
                    const uint8_t *Md = M + (size_t)(dd - 1) * N;
                    for (int a = 1; a < p; ++a)
                        if ((unsigned)Md[SUB(gg, dd - 1, a)] + (unsigned)dd == tau) {
                            d = dd;
                            break;
                        }
                }
                /* d >= 1 always exists here because tau < T_{j+1}[g] */
                uint64_t pw = ipow_u64(p, d - 1);
                for (int i = d - 1; i >= 0; --i, pw /= (uint64_t)p) {
                    const uint8_t *Mi = M + (size_t)i * N;
                    for (int a = (i == d - 1) ? 1 : 0; a < p; ++a) {
                        uint32_t cand = a ? SUB(gg, i, a) : gg;
                        if ((unsigned)Mi[cand] + (unsigned)d == tau) {
                            gg = cand;
                            k += (uint32_t)(a * pw);
                            break;
                        }
                    }
                }
            }
            g[H] = gg;
            kj[H] = k;
            if (k) {
                uint64_t q = (uint64_t)k + 1u, q2 = q * q;
                if (Pw[H] > UINT64_MAX / q2) status = ORC_EUNSUPPORTED;
                else Pw[H] *= q2;
                mx[H] = (uint8_t)(j + 1);
                ns[H] += 1;
            }
            if (kmap) kmap[(size_t)H * s + j] = k;
        }
        for (long t = 0; t < nsel; ++t) kall[(size_t)t * s + j] = kj[Hsel[t]];
    }
#undef SUB
#undef BUILD_TRANSLATIONS
    if (status == ORC_OK) {
        /* W and cls from the exact denominators accumulated above: the
         * definition of orc_weight_class_one, applied per coset. */
        for (uint64_t H = 0; H < N; ++H) {
            weight_from_denominator(Pw[H], W32 ? W32 + H : NULL, W64 ? W64 + H : NULL);
            if (cls) { cls[2 * H] = mx[H]; cls[2 * H + 1] = ns[H]; }
        }
        if (ksel) memcpy(ksel, kall, sizeof(uint32_t) * (size_t)nsel * s);
    }
done:
    free(R); free(T); free(M); free(Mn); free(g); free(kj); free(kall); free(Tr);
    free(Pw); free(mx); free(ns);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Cumulative class variances -> effective dimensions (Sec. 4): d_trc is the
 * least d with var_trc[d] >= thr * var, d_sup likewise with var_sup, where
 * var = var_trc[s] is the total variance; both are 0 when var = 0.  The
 * superposition condition is read with sigma^2_sup on both sides.           */
void orc_effdim_threshold(int s, const double *var_trc, const double *var_sup, double thr,
                          int *d_trc, int *d_sup)
{
    double tot = var_trc[s];
    *d_trc = 0;
    *d_sup = 0;
    if (!(tot > 0.0)) return;
    for (int d = 0; d <= s; ++d)
        if (var_trc[d] >= thr * tot) { *d_trc = d; break; }
    for (int d = 0; d <= s; ++d)
        if (var_sup[d] >= thr * tot) { *d_sup = d; break; }
}

/* Effective-dimension estimate of the finite Walsh series
 * g = sum_H g(H) wal_{k(H)} (eq. ANOVAdef with orthonormal Walsh functions):
 * its ANOVA effect u collects the terms with supp k(H) = u, so
 *     var_trc[d] = sum_{H != 0, max supp k(H) <= d} |g(H)|^2,
 *     var_sup[d] = sum_{H != 0, |supp k(H)| <= d} |g(H)|^2,
 * d = 0..s (Sec. 4, the truncation and superposition variances), followed by
 * the thresholds above.  gim may be NULL for real coefficients.             */
void orc_effdim(int s, long N, const double *gre, const double *gim, const uint8_t *cls, double thr,
                double *var_trc, double *var_sup, int *d_trc, int *d_sup)
{
    double *bt = (double *)calloc((size_t)s + 1, sizeof(double));
    double *bs = (double *)calloc((size_t)s + 1, sizeof(double));
    for (long H = 1; H < N; ++H) {
        double v = gre[H] * gre[H] + (gim ? gim[H] * gim[H] : 0.0);
        bt[cls[2 * H]] += v;
        bs[cls[2 * H + 1]] += v;
    }
    double ct = 0.0, cs = 0.0;
    for (int d = 0; d <= s; ++d) {
        ct += bt[d];
        cs += bs[d];
        var_trc[d] = ct;
        var_sup[d] = cs;
    }
    free(bt);
    free(bs);
    orc_effdim_threshold(s, var_trc, var_sup, thr, d_trc, d_sup);
}

/* ------------------------------------------------------------------------ */
/* Synthetic test functions evaluated at the net points x_{j,n} = Y_{j,n}/p^m. */

/* f_n = prod_j (1 + c_j (x_{j,n} - 1/2)) */
void orc_eval_product(int p, int m, int s, const uint32_t *Y, const double *c, double *f)
{
    uint64_t N = ipow_u64(p, m);
    double den = (double)N;
    for (uint64_t n = 0; n < N; ++n) {
        double v = 1.0;
        for (int j = 0; j < s; ++j) v *= 1.0 + c[j] * ((double)Y[(size_t)j * N + n] / den - 0.5);
        f[n] = v;
    }
}

/* f_n = exp(sum_j x_{j,n} / j^2), j counted from 1 */
void orc_eval_exp(int p, int m, int s, const uint32_t *Y, double *f)
{
    uint64_t N = ipow_u64(p, m);
    double den = (double)N;
    for (uint64_t n = 0; n < N; ++n) {
        double a = 0.0;
        for (int j = 0; j < s; ++j) a += ((double)Y[(size_t)j * N + n] / den) / ((double)(j + 1) * (j + 1));
        f[n] = exp(a);
    }
}

/* ------------------------------------------------------------------------ */
/* The kernel spline of Sec. 3.1 and its ANOVA variances (Sec. 4).          */

/* position i >= 1 of the first nonzero base-p digit of x = Y / p^m (0 if x = 0) */
static int first_digit_pos(int p, int m, uint32_t Y)
{
    if (Y == 0) return 0;
    int t = 0;                         /* Y in [p^t, p^(t+1)) */
    for (uint64_t q = (uint64_t)Y; q >= (uint64_t)p; q /= (uint64_t)p) ++t;
    return m - t;
}

/* Univariate kernel K'(x, 0) in its short form (Sec. 4): 1 at x = 0, else
 * 1 - p^{i(1-alpha)} (p^alpha - 1)/(p - 1), i the first nonzero digit of x.  */
double orc_kprime(int p, int m, double alpha, uint32_t Y)
{
    int i = first_digit_pos(p, m, Y);
    if (i == 0) return 1.0;
    return 1.0 - pow((double)p, i * (1.0 - alpha)) * (pow((double)p, alpha) - 1.0) / (p - 1.0);
}

/* Univariate kernel R'(x, 0) = int K'(t, x) K'(t, 0) dt in its short form (Sec. 4):
 * (p^a - p)^2 / ((p-1)(p^{2a} - p)) [1 - p^{i(1-2a)} (p^{2a} - 1)/(p - 1)], the
 * bracket being 1 at x = 0.                                                 */
double orc_rprime(int p, int m, double alpha, uint32_t Y)
{
    double pa = pow((double)p, alpha), p2a = pow((double)p, 2.0 * alpha);
    double c = (pa - p) * (pa - p) / ((p - 1.0) * (p2a - p));
    int i = first_digit_pos(p, m, Y);
    if (i == 0) return c;
    return c * (1.0 - pow((double)p, i * (1.0 - 2.0 * alpha)) * (p2a - 1.0) / (p - 1.0));
}

/* Kernel data at the net points (Sec. 3.1 and 4), Y[j][n] the point digits:
 *   K[n]      = prod_j (1 + gamma_j K'(x_{j,n}, 0)),
 *   R[d-1][n] = prod_{j <= d} (1 + gamma_j^2 R'(x_{j,n}, 0)),       d = 1..s,
 *   E[j-1][n] = sum_{|u| = j} prod_{i in u} gamma_i^2 R'(x_{i,n}, 0), j = 1..s,
 * the last by the recurrence of elementary symmetric polynomials, one
 * coordinate at a time.  Any of K, R, E may be NULL.                        */
void orc_kernel_data(int p, int m, int s, const uint32_t *Y, double alpha, const double *gamma,
                     double *K, double *R, double *E)
{
    uint64_t N = ipow_u64(p, m);
    double *e = (double *)malloc(((size_t)s + 1) * sizeof(double));
    for (uint64_t n = 0; n < N; ++n) {
        double kv = 1.0, rv = 1.0;
        e[0] = 1.0;
        for (int j = 1; j <= s; ++j) e[j] = 0.0;
        for (int j = 0; j < s; ++j) {
            uint32_t y = Y[(size_t)j * N + n];
            kv *= 1.0 + gamma[j] * orc_kprime(p, m, alpha, y);
            double a = gamma[j] * gamma[j] * orc_rprime(p, m, alpha, y);
            rv *= 1.0 + a;
            if (R) R[(size_t)j * N + n] = rv;
            for (int q = j + 1; q >= 1; --q) e[q] += a * e[q - 1];
        }
        if (K) K[n] = kv;
        if (E)
            for (int q = 1; q <= s; ++q) E[(size_t)(q - 1) * N + n] = e[q];
    }
    free(e);
}

/* The spline at arbitrary points (Sec. 3.1): for q = 0..Q-1,
 *   out[q] = sum_n c[n] prod_j (1 + gamma_j K'(x_{q,j} (-) x_{j,n}, 0)),
 * x_{q,j} = X[q s + j] / p^M with M >= m digits, x_{j,n} = Y[j][n] / p^m, and (-)
 * the digit-wise difference mod p of the M-digit numerators (the net point's
 * digits below the m-th are zero).  Direct sum, O(N s) per point.           */
void orc_spline_eval(int p, int m, int s, const uint32_t *Y, const double *c, const uint32_t *X, int Q, int M,
                     double alpha, const double *gamma, double *out)
{
    uint64_t N = ipow_u64(p, m);
    uint64_t up = ipow_u64(p, M - m);
    for (int q = 0; q < Q; ++q) {
        double acc = 0.0;
        for (uint64_t n = 0; n < N; ++n) {
            double kv = 1.0;
            for (int j = 0; j < s; ++j) {
                uint64_t a = (uint64_t)X[(size_t)q * s + j], b = (uint64_t)Y[(size_t)j * N + n] * up, z = 0, pw = 1;
                for (int d = 0; d < M; ++d) {          /* digit-wise difference mod p */
                    z += ((a % (uint64_t)p + (uint64_t)p - b % (uint64_t)p) % (uint64_t)p) * pw;
                    a /= (uint64_t)p;
                    b /= (uint64_t)p;
                    pw *= (uint64_t)p;
                }
                kv *= 1.0 + gamma[j] * orc_kprime(p, M, alpha, (uint32_t)z);
            }
            acc += c[n] * kv;
        }
        out[q] = acc;
    }
}

/* Kernel data at digitally shifted points (Sec. 3.1 and 5.1): for w = 0..N-1,
 * Kd[w] = prod_j (1 + gamma_j K'(x_{j,w} (+) delta_j, 0)), where x_{j,w} = Y/p^m has
 * m digits, delta_j = D[j] / p^M has M >= m digits, and (+) adds digits mod p.  */
void orc_kernel_shift_data(int p, int m, int s, const uint32_t *Y, const uint32_t *D, int M, double alpha,
                           const double *gamma, double *Kd)
{
    uint64_t N = ipow_u64(p, m);
    uint64_t up = ipow_u64(p, M - m);
    for (uint64_t w = 0; w < N; ++w) {
        double kv = 1.0;
        for (int j = 0; j < s; ++j) {
            uint64_t a = (uint64_t)Y[(size_t)j * N + w] * up, b = D[j], y = 0, pw = 1;
            for (int c = 0; c < M; ++c) {            /* digit-wise sum mod p of the M-digit numerators */
                y += ((a % (uint64_t)p + b % (uint64_t)p) % (uint64_t)p) * pw;
                a /= (uint64_t)p;
                b /= (uint64_t)p;
                pw *= (uint64_t)p;
            }
            kv *= 1.0 + gamma[j] * orc_kprime(p, M, alpha, (uint32_t)y);
        }
        Kd[w] = kv;
    }
}
