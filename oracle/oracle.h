/*
 * oracle.h -- plain CPU oracle for batched big-integer arithmetic.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it, and the two share
 * no code.
 *
 * Numbers are little-endian arrays of 64-bit limbs (base B = 2^64), as in the
 * paper's machine model (Sec. II: an integer is an array of M digits in base
 * B = 2^b, least significant first; Sec. VI: the digit type is 64-bit).
 * Internally every routine works on 32-bit half-digits with 64-bit
 * intermediates, so no 128-bit type and no carry-flag trick is involved.
 *
 * Every function below is the plain definition of the operation it names;
 * none of them uses the GPU path's methods (no carry scan, no Newton
 * iteration).  Parity status per function is stated in its comment.
 */
#ifndef BIGINT_ORACLE_H
#define BIGINT_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_OK 0
#define ORC_EDIVZERO 2
#define ORC_EINVAL 1

/* (a + b) mod B^n into out[0..n); returns the carry out (0 or 1).
 * Sec. V-A, Fig. 3 (golden addition): sequential ripple-carry reading. */
int orc_add(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t n);

/* (a - b) mod B^n into out[0..n); returns the borrow out (1 iff a < b).
 * Sec. V-A (subtraction is named, not shown): sequential ripple borrow. */
int orc_sub(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t n);

/* Full product a*b into out[0..na+nb).  Sec. V-B column formula
 * C_k = sum_{i+j=k} A_i B_j, without truncation, by operand-scanning
 * schoolbook multiplication on 32-bit half-digits. */
void orc_mul(const uint64_t *a, int64_t na, const uint64_t *b, int64_t nb,
             uint64_t *out);

/* Low m limbs of a*b (the product modulo B^m), Sec. V-C, Fig. 6 varPrecMul:
 * "computes the first m digits of A*B".  out[0..m). */
void orc_mul_lo(const uint64_t *a, int64_t na, const uint64_t *b, int64_t nb,
                int64_t m, uint64_t *out);

/* Quotient and remainder: q = floor(u/v) into q[0..nq), nq = max(nu-nv+1, 1),
 * r = u - q*v into r[0..nv).  Sec. V-C ("compute the quotient and
 * remainder") by Knuth's long division (TAOCP vol. 2, 4.3.1, Algorithm D) on
 * 32-bit half-digits.  Returns ORC_EDIVZERO (q = r = 0) when v = 0. */
int orc_divmod(const uint64_t *u, int64_t nu, const uint64_t *v, int64_t nv,
               uint64_t *q, uint64_t *r);

/* Shifted inverse shinv_h(v) = floor(B^h / v) into w[0..nw).  Sec. V-C
 * (Watt's shifted inverse), computed here by definition with orc_divmod.
 * Returns ORC_EINVAL if the result needs more than nw limbs,
 * ORC_EDIVZERO if v = 0. */
int orc_shinv(const uint64_t *v, int64_t nv, int64_t h, uint64_t *w,
              int64_t nw);

/* One Newton step of the shifted inverse, Sec. V-C, Fig. 6 (step):
 *   d  = B^(h-m) - v*w
 *   w' = w*B^m + floor(w*d / B^(h-2m))        if d >= 0
 *   w' = w*B^m - ceil(w*|d| / B^(h-2m))       if d <  0
 * (when h-2m < 0 the division is an exact multiplication by B^(2m-h)).
 * Writes w' into out[0..nout).  Returns ORC_EINVAL if w' < 0 or does not
 * fit in nout limbs, or if h < m. */
int orc_step(int64_t h, int64_t m, const uint64_t *v, int64_t nv,
             const uint64_t *w, int64_t nw, uint64_t *out, int64_t nout);

/* Precision: index of the highest nonzero limb plus one (0 for zero).
 * Sec. V-C, Fig. 6 (prec). */
int64_t orc_prec(const uint64_t *x, int64_t n);

/* The add chain r = a + b + ... + b (k additions), each addition mod B^n as
 * orc_add; returns the number of carries out (floor((a + k b) / B^n)).
 * Sec. VI, Table I (6-Add is k = 6). */
int orc_add_chain(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t n, int k);

/* Poly = (a a + b) (b b + b) + a b, every product and sum kept to n limbs
 * (mod B^n, as the paper's same-width multiply and add), into out[0..n).
 * Sec. VI, Table II: four multiplications (orc_mul_lo) and three additions
 * (orc_add), in that order. */
void orc_poly(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t n);

/* ---- batched drivers (uniform batches, instance-major), OpenMP over
 * instances when built with OpenMP.  Each returns the number of host
 * threads it used.  They exist to time the oracle as the CPU baseline. */
int orc_batch_add(const uint64_t *a, const uint64_t *b, uint64_t *out,
                  uint8_t *carry, int64_t count, int64_t n);
int orc_batch_sub(const uint64_t *a, const uint64_t *b, uint64_t *out,
                  uint8_t *borrow, int64_t count, int64_t n);
int orc_batch_mul(const uint64_t *a, const uint64_t *b, uint64_t *out,
                  int64_t count, int64_t na, int64_t nb);
int orc_batch_divmod(const uint64_t *u, const uint64_t *v, uint64_t *q,
                     uint64_t *r, int32_t *status, int64_t count, int64_t nu,
                     int64_t nv);
int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
