/*
 * tor_oracle.c -- CPU oracle for the Torontonian.  TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, the smoke check and the benchmark's CPU-baseline leg may load
 * this library.  It shares no code, header, table or helper with the CUDA
 * library in paper_2009_01177_gb300/csrc and must stay that way: it is the
 * independent reference the GPU path is compared against.
 *
 * What it computes (paper Sec. 3.1, Eq. 1 and Eq. 2):
 *
 *   Tor(O) = sum over all Z subset of [k] of (-1)^(k-|Z|) / sqrt(det(I - O_Z))
 *
 * for a 2k x 2k real-quadrature matrix O given in xxpp order (rows/cols
 * 0..k-1 are the x quadratures of the k clicked modes, k..2k-1 their p
 * quadratures).  O_Z keeps, for every mode j in Z, row/col j and k+j: the
 * selection rule of Eq. 1 applied a second time.
 *
 * How (Algorithm 1, Sec. 5.1-5.3): the direct subset sum.  Every subset gets
 * a fresh determinant -- there is deliberately no reuse between subsets, no
 * blocking and no reordering.  The arithmetic is the paper's own kind:
 * signed 256-bit fixed point with ONE global scaling factor 2^-F (F = 200
 * fractional bits by default, 55 integer bits).  Every FP64 input converts
 * exactly (for |x| >= 2^(53-F)), additions and subtractions are exact, a
 * product is truncated toward zero after the 512-bit intermediate.
 *
 *   det(I - O_Z): symmetric Gaussian elimination without pivoting, keeping
 *                 only the lower triangle (Sec. 4.2: I - A_Z is Hermitian
 *                 positive definite and stays so during elimination);
 *                 det = product of the pivots.  A pivot <= 0 is an error.
 *   reciprocal:   Newton iteration y <- y (2 - d y) from an FP64 seed (the
 *                 paper uses trial division; any method that reaches full
 *                 precision is equivalent, Sec. 5.3).
 *   1/sqrt(det):  Newton iteration y <- y (3 - x y^2) / 2 from an FP64 seed.
 *   sum:          exact fixed-point accumulation of (-1)^(k-|Z|) t_Z and of
 *                 t_Z (the latter gives the condition number of the sum).
 *
 * Readings of the paper taken here:
 *   - The empty set Z belongs to the sum (Eq. 2 sums over the full power
 *     set) with det(I - O_empty) = 1, i.e. t = 1.
 *   - The absolute value in Eq. 2 is a no-op for positive definite I - O_Z;
 *     a non-positive pivot is reported as an error instead of being folded.
 *   - Eq. 1: p(S) = Tor(O_S) / sqrt(det Sigma), and det Sigma = 1/det(I-O)
 *     for O = I - Sigma^-1, so p(S) = Tor(O_S) * sqrt(det(I - O)).
 *
 * Parallelism: OpenMP over subset masks.  Fixed-point addition is exact, so
 * the result does not depend on the thread count or the schedule.
 *
 * The `mutation` argument exists only so that the test suite can plant a
 * known mistake in the oracle and show that the pins catch it; 0 means the
 * faithful computation.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;
typedef struct { uint64_t w[4]; } fx; /* two's complement, w[0] least significant */

enum { ORC_OK = 0, ORC_EINVAL = 1, ORC_ENOTPD = 2, ORC_EOVERFLOW = 3 };

/* ---------------------------------------------------------------- fx core */

static int fx_is_neg(const fx *a) { return (int)(a->w[3] >> 63); }
static int fx_is_zero(const fx *a) { return (a->w[0] | a->w[1] | a->w[2] | a->w[3]) == 0; }

static fx fx_neg(fx a) {
    fx r; uint64_t c = 1;
    for (int i = 0; i < 4; ++i) { uint64_t v = ~a.w[i] + c; c = (c && v == 0) ? 1 : 0; r.w[i] = v; }
    return r;
}

static fx fx_add(fx a, fx b, int *err) {
    fx r; u128 c = 0;
    for (int i = 0; i < 4; ++i) { u128 s = (u128)a.w[i] + b.w[i] + c; r.w[i] = (uint64_t)s; c = s >> 64; }
    /* signed overflow: operands of equal sign, result of the other sign */
    if (fx_is_neg(&a) == fx_is_neg(&b) && fx_is_neg(&r) != fx_is_neg(&a)) *err = ORC_EOVERFLOW;
    return r;
}

static fx fx_sub(fx a, fx b, int *err) {
    fx nb = fx_neg(b);
    if (!fx_is_zero(&b) && fx_is_neg(&nb) == fx_is_neg(&b)) *err = ORC_EOVERFLOW; /* b = -2^255 */
    return fx_add(a, nb, err);
}

/* arithmetic shift right by s (0 <= s < 64) */
static fx fx_sar(fx a, int s) {
    if (s == 0) return a;
    fx r; uint64_t sign = fx_is_neg(&a) ? ~0ull : 0ull;
    for (int i = 0; i < 4; ++i) {
        uint64_t hi = (i < 3) ? a.w[i + 1] : sign;
        r.w[i] = (a.w[i] >> s) | (hi << (64 - s));
    }
    return r;
}

/* a*b*2^-F, magnitude truncated toward zero; 512-bit intermediate */
static fx fx_mul(fx a, fx b, int F, int *err) {
    int na = fx_is_neg(&a), nb = fx_is_neg(&b);
    fx ua = na ? fx_neg(a) : a, ub = nb ? fx_neg(b) : b;
    uint64_t p[8] = {0};
    for (int i = 0; i < 4; ++i) {
        u128 c = 0;
        for (int j = 0; j < 4; ++j) {
            u128 t = (u128)ua.w[i] * ub.w[j] + p[i + j] + c;
            p[i + j] = (uint64_t)t; c = t >> 64;
        }
        p[i + 4] = (uint64_t)c;
    }
    /* shift the 512-bit product right by F */
    int q = F / 64, s = F % 64;
    uint64_t sh[8] = {0};
    for (int i = 0; i + q < 8; ++i) {
        uint64_t lo = p[i + q];
        uint64_t hi = (i + q + 1 < 8) ? p[i + q + 1] : 0;
        sh[i] = s ? ((lo >> s) | (hi << (64 - s))) : lo;
    }
    if (sh[4] | sh[5] | sh[6] | sh[7] | (sh[3] >> 63)) *err = ORC_EOVERFLOW;
    fx r = {{sh[0], sh[1], sh[2], sh[3]}};
    return (na ^ nb) ? fx_neg(r) : r;
}

/* exact for |x| >= 2^(53-F); smaller magnitudes lose their low bits */
static fx fx_from_double(double x, int F, int *err) {
    fx r = {{0, 0, 0, 0}};
    if (x == 0.0) return r;
    if (!isfinite(x)) { *err = ORC_EINVAL; return r; }
    int e; double f = frexp(fabs(x), &e);          /* |x| = f 2^e, f in [0.5,1) */
    uint64_t m = (uint64_t)ldexp(f, 53);           /* exact 53-bit integer */
    int sh = e - 53 + F;                           /* X = m 2^sh */
    if (sh >= 0) {
        if (sh + 53 > 254) { *err = ORC_EOVERFLOW; return r; }
        int q = sh / 64, s = sh % 64;
        r.w[q] = m << s;
        if (s && q + 1 < 4) r.w[q + 1] = m >> (64 - s);
    } else {
        r.w[0] = (-sh >= 64) ? 0 : (m >> -sh);
    }
    return (x < 0) ? fx_neg(r) : r;
}

/* nearest double of the top 64 bits (used for seeds and for output) */
static double fx_to_double(fx a, int F) {
    int neg = fx_is_neg(&a);
    fx m = neg ? fx_neg(a) : a;
    int top = -1;
    for (int i = 3; i >= 0 && top < 0; --i)
        if (m.w[i]) top = 64 * i + 63 - __builtin_clzll(m.w[i]);
    if (top < 0) return 0.0;
    int lo = top - 63; if (lo < 0) lo = 0;
    int q = lo / 64, s = lo % 64;
    uint64_t bits = m.w[q] >> s;
    if (s && q + 1 < 4) bits |= m.w[q + 1] << (64 - s);
    double d = ldexp((double)bits, lo - F);
    return neg ? -d : d;
}

/* value as an unevaluated sum hi + lo of two doubles */
static void fx_to_dd(fx a, int F, double *hi, double *lo) {
    int err = 0;
    *hi = fx_to_double(a, F);
    fx r = fx_sub(a, fx_from_double(*hi, F, &err), &err);
    *lo = fx_to_double(r, F);
}

static fx fx_int(int64_t v, int F, int *err) { return fx_from_double((double)v, F, err); }

/* 1/d for d > 0 (Sec. 5.3: reciprocal, then multiply) */
static fx fx_recip(fx d, int F, int *err) {
    fx two = fx_int(2, F, err);
    fx y = fx_from_double(1.0 / fx_to_double(d, F), F, err);
    for (int it = 0; it < 6; ++it) y = fx_mul(y, fx_sub(two, fx_mul(d, y, F, err), err), F, err);
    return y;
}

/* 1/sqrt(x) for x > 0 (Sec. 5.3: reciprocal square root) */
static fx fx_rsqrt(fx x, int F, int *err) {
    fx three = fx_int(3, F, err);
    fx y = fx_from_double(1.0 / sqrt(fx_to_double(x, F)), F, err);
    for (int it = 0; it < 6; ++it) {
        fx y2 = fx_mul(y, y, F, err);
        y = fx_sar(fx_mul(y, fx_sub(three, fx_mul(x, y2, F, err), err), F, err), 1);
    }
    return y;
}

/* ------------------------------------------------------- the determinant */

/*
 * det(I - O_Z) for the modes listed in idx[0..m-1] of a 2k x 2k xxpp matrix.
 * a: scratch of (2m)^2 fx.  Returns ORC_ENOTPD on a pivot <= 0.
 */
static int det_I_minus_OZ(const double *O, int k, int ld, const int *idx, int m, fx *a,
                          int F, int mutation, fx *det) {
    int n = 2 * m, err = 0;
    int rows[128];
    for (int j = 0; j < m; ++j) {
        rows[j] = idx[j];                                  /* x quadrature of mode idx[j] */
        rows[m + j] = (mutation == 3) ? idx[j] : k + idx[j]; /* p quadrature (mutation 3: wrong index) */
    }
    fx one = fx_int(1, F, &err);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            fx o = fx_from_double(O[(size_t)rows[i] * ld + rows[j]], F, &err);
            fx b = fx_neg(o);                              /* -O */
            if (mutation == 4) b = o;                      /* mutation 4: I + O */
            if (i == j) b = fx_add(one, b, &err);          /* I - O */
            a[(size_t)i * n + j] = b;
        }
    fx d = one;
    for (int j = 0; j < n; ++j) {
        fx p = a[(size_t)j * n + j];
        if (fx_is_neg(&p) || fx_is_zero(&p)) return ORC_ENOTPD;
        d = fx_mul(d, p, F, &err);
        if (mutation == 5 && j == 0) continue;             /* mutation 5: drop the first update */
        fx r = fx_recip(p, F, &err);
        for (int i = j + 1; i < n; ++i) {
            fx f = fx_mul(a[(size_t)i * n + j], r, F, &err);   /* l_ij = a_ij / p */
            for (int l = j + 1; l <= i; ++l)                   /* a_il -= l_ij a_lj */
                a[(size_t)i * n + l] = fx_sub(a[(size_t)i * n + l],
                                              fx_mul(f, a[(size_t)l * n + j], F, &err), &err);
        }
    }
    *det = d;
    return err;
}

/* ----------------------------------------------------------- public API */

/*
 * Tor(O) by the direct subset sum.
 *   O: 2k x 2k, row-major with leading dimension ld, xxpp order.
 *   out[0..1]: Tor as hi + lo;  out[2..3]: sum_Z t_Z as hi + lo.
 *   mask_lo/mask_hi: only subsets whose mask lies in [mask_lo, mask_hi) are
 *   summed (pass 0 and 2^k for the whole sum).
 * Returns ORC_OK or an ORC_* error.
 */
static int tor_range_fx(const double *O, int k, int ld, int F, int nthreads, int mutation,
                        uint64_t mask_lo, uint64_t mask_hi, fx *tor_out, fx *sabs_out) {
    /* ranges of masks work up to k = 64 (the whole sum is limited to k <= 40 below) */
    if (k < 0 || k > 64 || ld < 2 * k || F < 64 || F > 240) return ORC_EINVAL;
    if (k < 64 && mask_hi > (1ull << k)) mask_hi = 1ull << k;
    if (mask_lo > mask_hi) mask_lo = mask_hi;
    const long long count = (long long)(mask_hi - mask_lo);
    if (count < 0) return ORC_EINVAL; /* more than 2^63 masks */
    int status = ORC_OK;
    fx tor = {{0, 0, 0, 0}}, sabs = {{0, 0, 0, 0}};
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int err = 0;
        fx ltor = {{0, 0, 0, 0}}, lsabs = {{0, 0, 0, 0}};
        fx *a = (fx *)malloc(sizeof(fx) * (size_t)(2 * k + 1) * (size_t)(2 * k + 1));
        int idx[64];
        if (!a) err = ORC_EINVAL;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (long long mm = 0; mm < count; ++mm) {
            if (err) continue;
            uint64_t mask = mask_lo + (uint64_t)mm;
            int m = 0;
            for (int j = 0; j < k; ++j) if (mask >> j & 1) idx[m++] = j;
            if (mutation == 1 && m == 0) continue;                 /* mutation 1: drop Z = {} */
            fx det, t;
            int e = det_I_minus_OZ(O, k, ld, idx, m, a, F, mutation, &det);
            if (e) { err = e; continue; }
            t = fx_rsqrt(det, F, &err);                             /* t_Z = 1/sqrt(det) */
            if (mutation == 6) t = fx_mul(det, t, F, &err);         /* mutation 6: sqrt(det) */
            int negative = ((k - m) & 1);                           /* (-1)^(k-|Z|) */
            if (mutation == 2) negative = (m & 1);                  /* mutation 2: (-1)^|Z| */
            ltor = negative ? fx_sub(ltor, t, &err) : fx_add(ltor, t, &err);
            lsabs = fx_add(lsabs, t, &err);
        }
        free(a);
#ifdef _OPENMP
#pragma omp critical
#endif
        {
            int e2 = 0;
            tor = fx_add(tor, ltor, &e2);
            sabs = fx_add(sabs, lsabs, &e2);
            if (err && !status) status = err;
            if (e2 && !status) status = e2;
        }
    }
    *tor_out = tor;
    *sabs_out = sabs;
    return status;
}

int oracle_tor_range(const double *O, int k, int ld, int F, int nthreads, int mutation,
                     uint64_t mask_lo, uint64_t mask_hi, double *out) {
    fx tor, sabs;
    int status = tor_range_fx(O, k, ld, F, nthreads, mutation, mask_lo, mask_hi, &tor, &sabs);
    fx_to_dd(tor, F, &out[0], &out[1]);
    fx_to_dd(sabs, F, &out[2], &out[3]);
    return status;
}

/*
 * The same sum as oracle_tor_range, returned exactly: raw[0..3] = the signed
 * sum, raw[4..7] = sum_Z t_Z, each a two's-complement 256-bit integer with F
 * fractional bits (value = integer / 2^F), little-endian 64-bit limbs.  The
 * double-double output of oracle_tor_range resolves only about 106 bits of
 * the result; this one gives every bit the fixed-point arithmetic computed.
 */
int oracle_tor_range_raw(const double *O, int k, int ld, int F, int nthreads, uint64_t mask_lo,
                         uint64_t mask_hi, uint64_t *raw) {
    fx tor, sabs;
    int status = tor_range_fx(O, k, ld, F, nthreads, 0, mask_lo, mask_hi, &tor, &sabs);
    for (int i = 0; i < 4; ++i) { raw[i] = tor.w[i]; raw[4 + i] = sabs.w[i]; }
    return status;
}



int oracle_tor(const double *O, int k, int ld, int F, int nthreads, int mutation, double *out) {
    if (k < 0 || k > 40) return ORC_EINVAL;
    return oracle_tor_range(O, k, ld, F, nthreads, mutation, 0, 1ull << k, out);
}

/*
 * det(I - O_Z) for one subset mask of a 2k x 2k xxpp matrix, as hi + lo.
 * Exposed so that tests can compare the fixed-point elimination with exact
 * rational arithmetic.
 */
int oracle_det(const double *O, int k, int ld, uint64_t mask, int F, double *out) {
    if (k < 0 || k > 64 || ld < 2 * k || F < 64 || F > 240) return ORC_EINVAL;
    int idx[64], m = 0;
    for (int j = 0; j < k; ++j) if (mask >> j & 1) idx[m++] = j;
    fx *a = (fx *)malloc(sizeof(fx) * (size_t)(2 * m + 1) * (size_t)(2 * m + 1));
    if (!a) return ORC_EINVAL;
    fx det;
    int e = det_I_minus_OZ(O, k, ld, idx, m, a, F, 0, &det);
    free(a);
    if (e) return e;
    fx_to_dd(det, F, &out[0], &out[1]);
    return ORC_OK;
}

/*
 * Click probability of Eq. 1:  p(S) = Tor(O_S) / sqrt(det Sigma).
 *   Ofull: 2M x 2M, leading dimension ld, xxpp order, O = I - Sigma^-1.
 *   pattern: M bytes, 0 or 1.
 * O_S takes row/col j and M+j of Ofull for every j with pattern[j] = 1
 * (selection rule of Eq. 1).  det Sigma = 1 / det(I - Ofull).
 *   out[0..1] = p(S) as hi + lo; out[2..3] = Tor(O_S); out[4..5] = sum t_Z.
 */
int oracle_prob(const double *Ofull, int M, int ld, const unsigned char *pattern, int F,
                int nthreads, double *out) {
    if (M < 0 || M > 64 || ld < 2 * M || F < 64 || F > 240) return ORC_EINVAL;
    int sel[64], k = 0;
    for (int j = 0; j < M; ++j) if (pattern[j]) sel[k++] = j;
    if (k > 40) return ORC_EINVAL;
    double *OS = (double *)malloc(sizeof(double) * (size_t)(2 * k + 1) * (size_t)(2 * k + 1));
    if (!OS) return ORC_EINVAL;
    for (int a = 0; a < 2 * k; ++a)
        for (int b = 0; b < 2 * k; ++b) {
            int ra = (a < k) ? sel[a] : M + sel[a - k];
            int rb = (b < k) ? sel[b] : M + sel[b - k];
            OS[(size_t)a * 2 * k + b] = Ofull[(size_t)ra * ld + rb];
        }
    double tor[4] = {0, 0, 0, 0};
    int e = oracle_tor(OS, k, 2 * k > 0 ? 2 * k : 1, F, nthreads, 0, tor);
    free(OS);
    if (e) return e;
    /* sqrt(det(I - Ofull)) = det * rsqrt(det), all in fixed point */
    int err = 0, idx[64];
    for (int j = 0; j < M; ++j) idx[j] = j;
    fx *a = (fx *)malloc(sizeof(fx) * (size_t)(2 * M + 1) * (size_t)(2 * M + 1));
    if (!a) return ORC_EINVAL;
    fx det;
    e = det_I_minus_OZ(Ofull, M, ld, idx, M, a, F, 0, &det);
    free(a);
    if (e) return e;
    fx sq = fx_mul(det, fx_rsqrt(det, F, &err), F, &err);
    fx torfx = fx_add(fx_from_double(tor[0], F, &err), fx_from_double(tor[1], F, &err), &err);
    fx p = fx_mul(torfx, sq, F, &err);
    fx_to_dd(p, F, &out[0], &out[1]);
    out[2] = tor[0]; out[3] = tor[1]; out[4] = tor[2]; out[5] = tor[3];
    return err;
}

/* 256-bit fixed-point self tests exposed for the test suite:
 * returns a*b and 1/a, 1/sqrt(a) of doubles through the fixed-point path. */
int oracle_fx_ops(double a, double b, int F, double *out) {
    int err = 0;
    fx x = fx_from_double(a, F, &err), y = fx_from_double(b, F, &err);
    fx_to_dd(fx_mul(x, y, F, &err), F, &out[0], &out[1]);
    fx_to_dd(fx_add(x, y, &err), F, &out[2], &out[3]);
    fx_to_dd(fx_sub(x, y, &err), F, &out[4], &out[5]);
    if (a > 0) {
        fx_to_dd(fx_recip(x, F, &err), F, &out[6], &out[7]);
        fx_to_dd(fx_rsqrt(x, F, &err), F, &out[8], &out[9]);
    } else {
        out[6] = out[7] = out[8] = out[9] = 0.0;
    }
    return err;
}
