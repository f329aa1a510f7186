/*
 * oracle.c -- plain CPU oracle for batched big-integer arithmetic.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, by the smoke check and by
 * the benchmark's CPU-baseline leg, never by the product path.  It shares no
 * code, header or table with the CUDA library.
 *
 * Representation: little-endian arrays of 64-bit limbs, B = 2^64 (Sec. II,
 * Sec. VI).  All arithmetic below runs on 32-bit half-digits ("digits",
 * base 2^32) held in uint32_t arrays, with uint64_t intermediates: a digit
 * product plus two digits always fits, (2^32-1)^2 + 2(2^32-1) = 2^64 - 1.
 * Limbs are split into digits with shifts, never with pointer casts, so the
 * code is independent of the host's byte order.
 *
 * Each routine is the textbook definition of its operation:
 *   add/sub    ripple carry / borrow (Sec. V-A, Fig. 3, read sequentially)
 *   mul        operand-scanning schoolbook (Sec. V-B column formula)
 *   divmod     Knuth, TAOCP vol. 2, Sec. 4.3.1, Algorithm D (Sec. V-C)
 *   shinv      floor(B^h / v) by long division (Sec. V-C)
 *   step       the Newton step formula of Sec. V-C, Fig. 6, evaluated with
 *              the exact operations above
 * Parity pins: every public routine is pinned in tests/test_oracle_pins.py
 * (brute force, closed forms, invariants, CPython int); none is unpinned.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------
 * A natural number as a digit array (base 2^32) with a logical length.
 * len is always trimmed (no leading zero digits); zero has len 0.
 * ---------------------------------------------------------------------- */
typedef struct {
    uint32_t *d;
    int64_t len;
    int64_t cap;
} nat;

static void nat_init(nat *x, int64_t cap)
{
    if (cap < 1) cap = 1;
    x->d = (uint32_t *)calloc((size_t)cap, sizeof(uint32_t));
    x->len = 0;
    x->cap = cap;
    if (!x->d) abort();
}

static void nat_free(nat *x)
{
    free(x->d);
    x->d = NULL;
    x->len = x->cap = 0;
}

static void nat_trim(nat *x)
{
    while (x->len > 0 && x->d[x->len - 1] == 0) x->len--;
}

static void nat_from_limbs(nat *x, const uint64_t *limbs, int64_t n)
{
    nat_init(x, 2 * n + 1);
    for (int64_t i = 0; i < n; i++) {
        x->d[2 * i] = (uint32_t)(limbs[i] & 0xffffffffu);
        x->d[2 * i + 1] = (uint32_t)(limbs[i] >> 32);
    }
    x->len = 2 * n;
    nat_trim(x);
}

/* Writes x into out[0..n) (zero-filled); returns 1 if x needs more than n
 * limbs (the low n limbs are written anyway), else 0. */
static int nat_to_limbs(const nat *x, uint64_t *out, int64_t n)
{
    for (int64_t i = 0; i < n; i++) {
        uint64_t lo = (2 * i < x->len) ? x->d[2 * i] : 0;
        uint64_t hi = (2 * i + 1 < x->len) ? x->d[2 * i + 1] : 0;
        out[i] = lo | (hi << 32);
    }
    return x->len > 2 * n;
}

static int nat_cmp(const nat *a, const nat *b)
{
    if (a->len != b->len) return a->len < b->len ? -1 : 1;
    for (int64_t i = a->len - 1; i >= 0; i--)
        if (a->d[i] != b->d[i]) return a->d[i] < b->d[i] ? -1 : 1;
    return 0;
}

/* out = a + b (out must not alias). */
static void nat_add(const nat *a, const nat *b, nat *out)
{
    int64_t n = a->len > b->len ? a->len : b->len;
    nat_init(out, n + 1);
    uint64_t carry = 0;
    for (int64_t i = 0; i < n; i++) {
        uint64_t t = carry;
        if (i < a->len) t += a->d[i];
        if (i < b->len) t += b->d[i];
        out->d[i] = (uint32_t)t;
        carry = t >> 32;
    }
    out->d[n] = (uint32_t)carry;
    out->len = n + 1;
    nat_trim(out);
}

/* out = a - b, requires a >= b (out must not alias). */
static void nat_sub(const nat *a, const nat *b, nat *out)
{
    nat_init(out, a->len);
    uint64_t borrow = 0;
    for (int64_t i = 0; i < a->len; i++) {
        uint64_t t = (uint64_t)a->d[i] - (i < b->len ? b->d[i] : 0) - borrow;
        out->d[i] = (uint32_t)t;
        borrow = t >> 63; /* a wrapped difference has its top bit set */
    }
    out->len = a->len;
    nat_trim(out);
}

/* out = a * b by operand scanning: for each digit a_i, add the row
 * a_i * b shifted by i digits into the running sum (Knuth Algorithm M). */
static void nat_mul(const nat *a, const nat *b, nat *out)
{
    nat_init(out, a->len + b->len + 1);
    for (int64_t i = 0; i < a->len; i++) {
        uint64_t carry = 0;
        for (int64_t j = 0; j < b->len; j++) {
            uint64_t t = (uint64_t)a->d[i] * b->d[j] + out->d[i + j] + carry;
            out->d[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        out->d[i + b->len] = (uint32_t)carry;
    }
    out->len = a->len + b->len;
    nat_trim(out);
}

/* out = x * 2^(32 s), s >= 0. */
static void nat_shl_digits(const nat *x, int64_t s, nat *out)
{
    nat_init(out, x->len + s);
    if (x->len == 0) return;
    memcpy(out->d + s, x->d, (size_t)x->len * sizeof(uint32_t));
    out->len = x->len + s;
}

/* out = floor(x / 2^(32 s)), s >= 0; *dropped = 1 if any dropped digit is
 * nonzero. */
static void nat_shr_digits(const nat *x, int64_t s, nat *out, int *dropped)
{
    int64_t n = x->len - s;
    *dropped = 0;
    for (int64_t i = 0; i < s && i < x->len; i++)
        if (x->d[i]) *dropped = 1;
    nat_init(out, n > 0 ? n : 1);
    if (n <= 0) return;
    memcpy(out->d, x->d + s, (size_t)n * sizeof(uint32_t));
    out->len = n;
}

static int clz32(uint32_t x)
{
    int n = 0;
    if (x == 0) return 32;
    while (!(x & 0x80000000u)) {
        x <<= 1;
        n++;
    }
    return n;
}

/* q = floor(u / v), r = u - q v, for v > 0.  Knuth's Algorithm D:
 * normalise so the divisor's top digit has its top bit set, estimate each
 * quotient digit from the top two dividend digits and the top divisor digit,
 * refine the estimate with the second divisor digit, multiply and subtract,
 * and add back in the rare case the estimate was still one too large. */
static void nat_divmod(const nat *u, const nat *v, nat *q, nat *r)
{
    const int64_t n = v->len;
    if (nat_cmp(u, v) < 0) {
        nat_init(q, 1);
        nat_init(r, u->len);
        if (u->len) memcpy(r->d, u->d, (size_t)u->len * sizeof(uint32_t));
        r->len = u->len;
        return;
    }
    const int64_t m = u->len - n;
    nat_init(q, m + 1);
    if (n == 1) {
        /* short division by a single digit */
        uint64_t rem = 0;
        for (int64_t i = u->len - 1; i >= 0; i--) {
            uint64_t cur = (rem << 32) | u->d[i];
            q->d[i] = (uint32_t)(cur / v->d[0]);
            rem = cur % v->d[0];
        }
        q->len = m + 1;
        nat_trim(q);
        nat_init(r, 1);
        r->d[0] = (uint32_t)rem;
        r->len = 1;
        nat_trim(r);
        return;
    }
    const int s = clz32(v->d[n - 1]);
    uint32_t *vn = (uint32_t *)calloc((size_t)n, sizeof(uint32_t));
    uint32_t *un = (uint32_t *)calloc((size_t)(u->len + 1), sizeof(uint32_t));
    if (!vn || !un) abort();
    for (int64_t i = n - 1; i > 0; i--)
        vn[i] = (v->d[i] << s) | (s ? v->d[i - 1] >> (32 - s) : 0);
    vn[0] = v->d[0] << s;
    un[u->len] = s ? u->d[u->len - 1] >> (32 - s) : 0;
    for (int64_t i = u->len - 1; i > 0; i--)
        un[i] = (u->d[i] << s) | (s ? u->d[i - 1] >> (32 - s) : 0);
    un[0] = u->d[0] << s;

    const uint64_t base = (uint64_t)1 << 32;
    for (int64_t j = m; j >= 0; j--) {
        uint64_t num = ((uint64_t)un[j + n] << 32) | un[j + n - 1];
        uint64_t qhat = num / vn[n - 1];
        uint64_t rhat = num % vn[n - 1];
        while (qhat >= base ||
               qhat * vn[n - 2] > ((rhat << 32) | un[j + n - 2])) {
            qhat--;
            rhat += vn[n - 1];
            if (rhat >= base) break;
        }
        /* un[j .. j+n] -= qhat * vn[0 .. n) */
        uint64_t carry = 0;
        int64_t borrow = 0;
        for (int64_t i = 0; i < n; i++) {
            uint64_t p = qhat * vn[i] + carry;
            carry = p >> 32;
            int64_t t = (int64_t)un[i + j] - (int64_t)(p & 0xffffffffu) - borrow;
            un[i + j] = (uint32_t)t;
            borrow = t < 0;
        }
        int64_t t = (int64_t)un[j + n] - (int64_t)carry - borrow;
        un[j + n] = (uint32_t)t;
        if (t < 0) {
            /* the estimate was one too large: add the divisor back */
            qhat--;
            uint64_t c = 0;
            for (int64_t i = 0; i < n; i++) {
                uint64_t s2 = (uint64_t)un[i + j] + vn[i] + c;
                un[i + j] = (uint32_t)s2;
                c = s2 >> 32;
            }
            un[j + n] += (uint32_t)c;
        }
        q->d[j] = (uint32_t)qhat;
    }
    q->len = m + 1;
    nat_trim(q);

    /* the remainder is un[0 .. n] shifted back right by s bits */
    nat_init(r, n);
    for (int64_t i = 0; i < n; i++)
        r->d[i] = (un[i] >> s) | (s ? un[i + 1] << (32 - s) : 0);
    r->len = n;
    nat_trim(r);
    free(vn);
    free(un);
}

/* ------------------------------------------------------------------------
 * Public routines.
 * ---------------------------------------------------------------------- */

int orc_add(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t n)
{
    uint64_t carry = 0;
    for (int64_t i = 0; i < n; i++) {
        uint64_t lo = (a[i] & 0xffffffffu) + (b[i] & 0xffffffffu) + carry;
        uint64_t hi = (a[i] >> 32) + (b[i] >> 32) + (lo >> 32);
        out[i] = (lo & 0xffffffffu) | (hi << 32);
        carry = hi >> 32;
    }
    return (int)carry;
}

int orc_sub(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t n)
{
    uint64_t borrow = 0;
    for (int64_t i = 0; i < n; i++) {
        uint64_t lo = (a[i] & 0xffffffffu) - (b[i] & 0xffffffffu) - borrow;
        uint64_t blo = lo >> 63;
        uint64_t hi = (a[i] >> 32) - (b[i] >> 32) - blo;
        out[i] = (lo & 0xffffffffu) | (hi << 32);
        borrow = hi >> 63;
    }
    return (int)borrow;
}

void orc_mul(const uint64_t *a, int64_t na, const uint64_t *b, int64_t nb,
             uint64_t *out)
{
    nat x, y, z;
    nat_from_limbs(&x, a, na);
    nat_from_limbs(&y, b, nb);
    nat_mul(&x, &y, &z);
    nat_to_limbs(&z, out, na + nb);
    nat_free(&x);
    nat_free(&y);
    nat_free(&z);
}

void orc_mul_lo(const uint64_t *a, int64_t na, const uint64_t *b, int64_t nb,
                int64_t m, uint64_t *out)
{
    nat x, y, z;
    nat_from_limbs(&x, a, na);
    nat_from_limbs(&y, b, nb);
    nat_mul(&x, &y, &z);
    nat_to_limbs(&z, out, m); /* keeps the low m limbs: the product mod B^m */
    nat_free(&x);
    nat_free(&y);
    nat_free(&z);
}

int orc_divmod(const uint64_t *u, int64_t nu, const uint64_t *v, int64_t nv,
               uint64_t *q, uint64_t *r)
{
    const int64_t nq = nu - nv + 1 > 1 ? nu - nv + 1 : 1;
    nat x, y, qq, rr;
    nat_from_limbs(&y, v, nv);
    if (y.len == 0) {
        memset(q, 0, (size_t)nq * sizeof(uint64_t));
        memset(r, 0, (size_t)nv * sizeof(uint64_t));
        nat_free(&y);
        return ORC_EDIVZERO;
    }
    nat_from_limbs(&x, u, nu);
    nat_divmod(&x, &y, &qq, &rr);
    int over = nat_to_limbs(&qq, q, nq);
    nat_to_limbs(&rr, r, nv);
    nat_free(&x);
    nat_free(&y);
    nat_free(&qq);
    nat_free(&rr);
    return over ? ORC_EINVAL : ORC_OK;
}

int orc_shinv(const uint64_t *v, int64_t nv, int64_t h, uint64_t *w, int64_t nw)
{
    nat x, y, qq, rr;
    nat_from_limbs(&y, v, nv);
    if (y.len == 0) {
        memset(w, 0, (size_t)nw * sizeof(uint64_t));
        nat_free(&y);
        return ORC_EDIVZERO;
    }
    nat_init(&x, 2 * h + 1); /* B^h = 2^(64 h): digit 2h is 1 */
    x.d[2 * h] = 1;
    x.len = 2 * h + 1;
    nat_divmod(&x, &y, &qq, &rr);
    int over = nat_to_limbs(&qq, w, nw);
    nat_free(&x);
    nat_free(&y);
    nat_free(&qq);
    nat_free(&rr);
    return over ? ORC_EINVAL : ORC_OK;
}

int orc_step(int64_t h, int64_t m, const uint64_t *v, int64_t nv,
             const uint64_t *w, int64_t nw, uint64_t *out, int64_t nout)
{
    if (h < m || m < 0) return ORC_EINVAL;
    nat V, W, VW, P, D, T, Y, WS, R;
    int neg, dropped = 0;
    nat_from_limbs(&V, v, nv);
    nat_from_limbs(&W, w, nw);
    nat_mul(&V, &W, &VW);
    /* P = B^(h-m) */
    nat_init(&P, 2 * (h - m) + 1);
    P.d[2 * (h - m)] = 1;
    P.len = 2 * (h - m) + 1;
    /* d = P - v w, kept as sign and magnitude */
    if (nat_cmp(&P, &VW) >= 0) {
        neg = 0;
        nat_sub(&P, &VW, &D);
    } else {
        neg = 1;
        nat_sub(&VW, &P, &D);
    }
    nat_mul(&W, &D, &T); /* w |d| */
    if (h - 2 * m >= 0) {
        nat_shr_digits(&T, 2 * (h - 2 * m), &Y, &dropped); /* floor(w|d| / B^(h-2m)) */
        if (neg && dropped) {
            /* ceiling: one more unless the dropped digits are all zero */
            nat one, Y1;
            nat_init(&one, 1);
            one.d[0] = 1;
            one.len = 1;
            nat_add(&Y, &one, &Y1);
            nat_free(&Y);
            nat_free(&one);
            Y = Y1;
        }
    } else {
        nat_shl_digits(&T, 2 * (2 * m - h), &Y);
    }
    nat_shl_digits(&W, 2 * m, &WS); /* w B^m */
    int rc = ORC_OK;
    if (!neg) {
        nat_add(&WS, &Y, &R);
    } else if (nat_cmp(&WS, &Y) >= 0) {
        nat_sub(&WS, &Y, &R);
    } else {
        nat_init(&R, 1);
        rc = ORC_EINVAL; /* negative result */
    }
    if (rc == ORC_OK && nat_to_limbs(&R, out, nout)) rc = ORC_EINVAL;
    if (rc != ORC_OK) memset(out, 0, (size_t)nout * sizeof(uint64_t));
    nat_free(&V);
    nat_free(&W);
    nat_free(&VW);
    nat_free(&P);
    nat_free(&D);
    nat_free(&T);
    nat_free(&Y);
    nat_free(&WS);
    nat_free(&R);
    return rc;
}

int64_t orc_prec(const uint64_t *x, int64_t n)
{
    int64_t p = 0;
    for (int64_t i = 0; i < n; i++)
        if (x[i] != 0) p = i + 1;
    return p;
}

int orc_add_chain(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t n, int k)
{
    int carries = 0;
    for (int64_t i = 0; i < n; i++) out[i] = a[i];
    for (int it = 0; it < k; it++) carries += orc_add(out, b, out, n);
    return carries;
}

void orc_poly(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t n)
{
    uint64_t *t1 = malloc(sizeof(uint64_t) * (size_t)n);
    uint64_t *t2 = malloc(sizeof(uint64_t) * (size_t)n);
    uint64_t *t3 = malloc(sizeof(uint64_t) * (size_t)n);
    orc_mul_lo(a, n, a, n, n, t1);   /* a a */
    orc_add(t1, b, t1, n);           /* a a + b */
    orc_mul_lo(b, n, b, n, n, t2);   /* b b */
    orc_add(t2, b, t2, n);           /* b b + b */
    orc_mul_lo(t1, n, t2, n, n, t3); /* (a a + b)(b b + b) */
    orc_mul_lo(a, n, b, n, n, out);  /* a b */
    orc_add(out, t3, out, n);        /* ... + a b */
    free(t1);
    free(t2);
    free(t3);
}

/* ------------------------------------------------------------------------
 * Batched drivers.
 * ---------------------------------------------------------------------- */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

int orc_batch_add(const uint64_t *a, const uint64_t *b, uint64_t *out,
                  uint8_t *carry, int64_t count, int64_t n)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < count; i++) {
        int c = orc_add(a + i * n, b + i * n, out + i * n, n);
        if (carry) carry[i] = (uint8_t)c;
    }
    return orc_num_threads();
}

int orc_batch_sub(const uint64_t *a, const uint64_t *b, uint64_t *out,
                  uint8_t *borrow, int64_t count, int64_t n)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int64_t i = 0; i < count; i++) {
        int c = orc_sub(a + i * n, b + i * n, out + i * n, n);
        if (borrow) borrow[i] = (uint8_t)c;
    }
    return orc_num_threads();
}

int orc_batch_mul(const uint64_t *a, const uint64_t *b, uint64_t *out,
                  int64_t count, int64_t na, int64_t nb)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < count; i++)
        orc_mul(a + i * na, na, b + i * nb, nb, out + i * (na + nb));
    return orc_num_threads();
}

int orc_batch_divmod(const uint64_t *u, const uint64_t *v, uint64_t *q,
                     uint64_t *r, int32_t *status, int64_t count, int64_t nu,
                     int64_t nv)
{
    const int64_t nq = nu - nv + 1 > 1 ? nu - nv + 1 : 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t i = 0; i < count; i++) {
        int s = orc_divmod(u + i * nu, nu, v + i * nv, nv, q + i * nq, r + i * nv);
        if (status) status[i] = s;
    }
    return orc_num_threads();
}
