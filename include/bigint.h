/*
 * bigint.h -- C ABI of libbigint: batched exact arithmetic on midsize
 * unsigned integers on one GB300 (sm_103a).
 *
 * Method: "High-Level Big Integer Arithmetic in Futhark for GPUs"
 * (Oancea and Watt).  Section numbers below refer to that paper.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - An integer is an array of 64-bit limbs, least significant first
 *   (Sec. II: M digits of base B = 2^b, little-endian; Sec. VI: b = 64).
 * - A uniform batch of `count` instances of `n` limbs is one contiguous
 *   array of count*n limbs, instance i at offset i*n (instance-major).
 * - All data pointers are DEVICE pointers owned by the caller.  The library
 *   never frees them and keeps no reference after the call returns.
 * - Every compute call is asynchronous on `stream` (a cudaStream_t passed as
 *   void*; NULL is the legacy default stream).  Output buffers must not
 *   overlap input buffers.
 * - Return value: BIGINT_OK or a negative error code.  Argument errors are
 *   detected on the host before anything is launched.  Per-instance
 *   conditions (division by zero, quotient overflow) are reported through
 *   per-instance status arrays and never abort the batch.
 */
#ifndef BIGINT_H
#define BIGINT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------*/
#define BIGINT_OK 0
#define BIGINT_EINVAL (-1)     /* bad argument (sizes, NULL, alignment)       */
#define BIGINT_EDIVZERO (-2)   /* per instance: divisor is zero               */
#define BIGINT_ENOMEM (-3)     /* workspace too small                         */
#define BIGINT_ETIMEOUT (-4)   /* a device-side wait hit its iteration limit  */
#define BIGINT_EINTERNAL (-5)  /* an internal correction limit was exceeded   */
#define BIGINT_ECUDA (-6)      /* a CUDA runtime call failed                  */
#define BIGINT_ERANGE (-7)     /* per instance: quotient does not fit in nq   */

/* Largest operand accepted by add, sub and divmod, in limbs (2^20 bits). */
#define BIGINT_MAX_LIMBS 16384
/* Largest operand accepted by mul and mul_lo, in limbs (both operands of
 * one product are held in one SM's shared memory). */
#define BIGINT_MUL_MAX_LIMBS 10000

/* Human-readable name of a status code (static storage, never NULL). */
const char *bigint_strerror(int status);

/* Library version as major*10000 + minor*100 + patch. */
int bigint_version(void);

/* ---- addition and subtraction (Sec. V-A, Figs. 3 and 4) -----------------
 * out = (a + b) mod B^n, carry_out[i] = floor((a_i + b_i) / B^n) in {0,1}.
 * The carry is propagated as an exclusive scan over per-digit
 * (generate, propagate) pairs with the operator
 *   (g1,p1) o (g2,p2) = (g2 | (g1 & p2), p1 & p2)                (Fig. 3)
 * blocked as in Fig. 4: each thread folds its own limbs sequentially, then
 * a block-level scan joins the threads.
 * a, b, out: count*n limbs.  carry_out: count bytes, or NULL.
 * 1 <= n <= BIGINT_MAX_LIMBS, count >= 0 (count == 0 is a no-op).      */
int bigint_add(const uint64_t *a, const uint64_t *b, uint64_t *out,
               uint8_t *carry_out, int64_t count, int32_t n, void *stream);

/* out = (a - b) mod B^n, borrow_out[i] = 1 iff a_i < b_i.  Subtraction is
 * named but not shown in the paper (Sec. V-C uses bsubReg); it is the same
 * scan with generate = (a_j < b_j) and propagate = (a_j == b_j).
 * Same layout and limits as bigint_add.                                  */
int bigint_sub(const uint64_t *a, const uint64_t *b, uint64_t *out,
               uint8_t *borrow_out, int64_t count, int32_t n, void *stream);

/* ---- multiplication (Sec. V-B, Fig. 5) ----------------------------------
 * out = a * b, the FULL product of na + nb limbs per instance: the
 * schoolbook convolution C_k = sum_{i+j=k} a_i b_j of Sec. V-B, exact.
 * When the shorter operand has 256 limbs or more (and fits one SM's shared
 * memory) the convolution runs on the tensor cores: the operands as signed
 * base-256 digits, the convolution as fp16 matrix products (tcgen05.mma,
 * Toeplitz blocks of one operand times shifted blocks of the other) with
 * exact fp32 accumulation in tensor memory, the column sums turned into
 * limbs by one carry scan per output tile (Fig. 3).  Smaller products use
 * the integer pipes: column blocks ("chunks") with rising and falling chunks
 * paired per thread (Fig. 5 threadConv), one 32x32->64-bit multiply-add per
 * digit product with deferred carries, and one carry-scan addition of the
 * chunks' digits and overflow words (Fig. 5 combineQ, bmulReg).
 * a: count*na limbs, b: count*nb limbs, out: count*(na+nb) limbs.
 * 1 <= na, nb <= BIGINT_MUL_MAX_LIMBS.                                     */
int bigint_mul(const uint64_t *a, const uint64_t *b, uint64_t *out,
               int64_t count, int32_t na, int32_t nb, void *stream);

/* Low m limbs of a*b (the product modulo B^m): the variable-precision
 * multiply of Sec. V-C, Fig. 6 (varPrecMul, "computes the first m digits
 * of A*B").  a: count*na, b: count*nb, out: count*m limbs,
 * 1 <= na, nb <= BIGINT_MUL_MAX_LIMBS, 1 <= m <= na + nb.                 */
int bigint_mul_lo(const uint64_t *a, const uint64_t *b, uint64_t *out,
                  int64_t count, int32_t na, int32_t nb, int32_t m,
                  void *stream);

/* The products of bigint_mul with each product spread over several CTAs,
 * for few, large products (serving), where one CTA per product would leave
 * most SMs idle.  Up to 16 products with a shorter operand of 256 limbs or
 * more: each product's output tiles (4096 limbs each) are cut further into
 * units of consecutive groups of Toeplitz blocks, about one unit per SM;
 * every unit adds its tile's partial column sums into a buffer in the
 * workspace with integer atomic adds (exact, in any order), and one CTA per
 * product turns the sums into limbs.  Larger batches: each product's output
 * tiles on different CTAs, linked by a second small kernel (the carries
 * between tiles and the column-sum bias are settled there).  Any other
 * product runs as bigint_mul.  Results are bit-identical to bigint_mul.
 * workspace: bigint_mul_split_workspace(count, na, nb) bytes of device
 * memory (up to 512 KB per product for the column sums of the first form,
 * 16 bytes per tile for the second, 0 when nothing splits), 8-byte
 * aligned; BIGINT_ENOMEM if smaller.  Multi-CTA per instance: a latency
 * form, not part of Sec. VI's one-instance-per-CTA design.                 */
size_t bigint_mul_split_workspace(int64_t count, int32_t na, int32_t nb);
int bigint_mul_split(const uint64_t *a, const uint64_t *b, uint64_t *out,
                     int64_t count, int32_t na, int32_t nb, void *workspace,
                     size_t workspace_bytes, void *stream);

/* ---- sub-quadratic full products (Karatsuba over the products above) -----
 * out = a * b for square operands (a, b: count x n limbs, out: count x 2n,
 * disjoint from a and b), by `levels` levels of Karatsuba's method in its
 * subtractive form -- x y = z2 B^2k + (z0 + z2 + (x0 - x1)(y1 - y0)) B^k +
 * z0 with n = 2k -- every step batched across the instances, the leaf
 * products those of bigint_mul (tensor cores from 256 limbs).  The paper
 * names sub-quadratic multiplication as its next step; this is its exact
 * integer form.  levels: 0..3, or -1 for the measured choice on GB300 (two
 * from 8192 limbs, one from 4096, none below); a level that would not halve
 * n exactly is dropped.  Bit-identical to bigint_mul.
 * workspace: device memory, 256-byte aligned, owned by the caller, contents
 * clobbered; bigint_mul_kara_workspace(count, n, levels) bytes run the
 * batch in one pass, fewer run it in chunks of as many instances as fit
 * (BIGINT_ENOMEM if not even one fits; NULL is fine when no level runs).
 * 1 <= n <= BIGINT_MUL_MAX_LIMBS; BIGINT_EINVAL otherwise.                  */
size_t bigint_mul_kara_workspace(int64_t count, int32_t n, int32_t levels);
int bigint_mul_kara(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count,
                    int32_t n, int32_t levels, void *workspace, size_t workspace_bytes,
                    void *stream);

/* ---- division (Sec. V-C, Fig. 6) ----------------------------------------
 * q = floor(u / v), r = u - q v, by the shifted inverse
 *   w = shinv_h(v) = floor(B^h / v)
 * computed with Newton steps (Fig. 6 `step`) over variable-precision
 * multiplications, followed by q = floor(u w / B^h) with an exact final
 * correction.
 * u: count*nu limbs, v: count*nv limbs, q: count*nq limbs with
 * nq = max(nu - nv + 1, 1), r: count*nv limbs, status: count int32 (may be
 * NULL): 0, BIGINT_EDIVZERO (v = 0; q and r are set to 0) or BIGINT_ERANGE
 * (v has leading zero limbs and the quotient needs more than nq limbs; q
 * holds the quotient mod B^nq and r is exact).
 * workspace: device scratch of at least bigint_divmod_workspace(count, nu,
 * nv) bytes, 256-byte aligned, owned by the caller, contents clobbered.
 * 1 <= nu, nv <= BIGINT_MAX_LIMBS.
 * Schedule: with divisors of 128 limbs or more (and nu >= nv) every Newton
 * step runs for all instances at once -- each product one batched launch
 * of the multiply kernels, each linear step one small launch -- and only
 * instances whose divisor has a zero top limb are divided one CTA each at
 * the end; smaller divisions run one CTA per division (the paper's
 * intragroup form).  Results are the same either way.                     */
int bigint_divmod(const uint64_t *u, const uint64_t *v, uint64_t *q,
                  uint64_t *r, int32_t *status, int64_t count, int32_t nu,
                  int32_t nv, void *workspace, size_t workspace_bytes,
                  void *stream);

/* Bytes of device workspace bigint_divmod needs for this batch shape. */
size_t bigint_divmod_workspace(int64_t count, int32_t nu, int32_t nv);

/* Division for callers that cannot allocate device memory (no counterpart
 * in the paper: it exists for callers that may not call cudaMalloc, such as
 * a host application that gives this library a fixed memory budget, or a
 * latency-critical loop that cannot afford cudaMalloc's implicit device
 * synchronisation).  Same arguments, results and per-instance status as
 * bigint_divmod, without the workspace: the scratch is one file-scope
 * __device__ array of bigint_divmod_noalloc_scratch_bytes() bytes (32 MiB)
 * that every GPU loading the library holds until the process exits.  It
 * allocates nothing itself.
 * - The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress); make that first call before any stream capture.
 *   The lookup is repeated only when the device's context has been
 *   destroyed and created again (cudaDeviceReset), which can move the
 *   array.
 * - Batches larger than the array holds run as consecutive launches on
 *   `stream`; a shape whose single instance needs more scratch than the
 *   array is rejected with BIGINT_ENOMEM.
 * - All calls share the array and nothing in it needs to start at zero;
 *   calls that overlap on the GPU (different streams, or several host
 *   threads) race on it and must be serialised by the caller.            */
int bigint_divmod_noalloc(const uint64_t *u, const uint64_t *v, uint64_t *q,
                          uint64_t *r, int32_t *status, int64_t count,
                          int32_t nu, int32_t nv, void *stream);
size_t bigint_divmod_noalloc_scratch_bytes(void);

/* Shifted inverse w = floor(B^h / v) (Sec. V-C; the Newton loop of Fig. 6).
 * v: count*nv limbs, w: count*nw limbs.  status as for bigint_divmod
 * (BIGINT_ERANGE if the inverse needs more than nw limbs).
 * nv <= h <= 2*BIGINT_MAX_LIMBS.  workspace: bigint_shinv_workspace bytes. */
int bigint_shinv(const uint64_t *v, uint64_t *w, int32_t *status,
                 int64_t count, int32_t nv, int32_t h, int32_t nw,
                 void *workspace, size_t workspace_bytes, void *stream);
size_t bigint_shinv_workspace(int64_t count, int32_t nv, int32_t h);

/* Division by a shifted inverse computed once and reused (Sec. V-C: the
 * quotient is floor(u w / B^h) up to the exact final correction; here w is
 * an input, e.g. from bigint_shinv, so many dividends share one divisor's
 * Newton loop).  w = floor(B^h / v) exactly, nw limbs, h >= nu, h >= nv,
 * nw <= h + 1; the kernel takes the top limbs of w, floor(w / B^(h - k)) =
 * floor(B^k / v) with k = prec(u), and finishes as bigint_divmod does.
 * v_stride: nv (one divisor per instance) or 0 (one divisor for the whole
 * batch, v holds nv limbs); w_stride likewise nw or 0.  q, r, status and
 * the workspace (bigint_divmod_workspace(count, nu, nv) bytes) as for
 * bigint_divmod.  w is not checked: a value other than that inverse gives
 * BIGINT_EINTERNAL where the correction does not settle (a w far off), and
 * otherwise no guarantee on q and r.                                       */
int bigint_divmod_inv(const uint64_t *u, const uint64_t *v, const uint64_t *w,
                      uint64_t *q, uint64_t *r, int32_t *status, int64_t count,
                      int32_t nu, int32_t nv, int32_t nw, int32_t h,
                      int64_t v_stride, int64_t w_stride, void *workspace,
                      size_t workspace_bytes, void *stream);

/* ---- ragged batches of mixed operations (the batched form) --------------
 * A batch is an array of operation descriptors over one input pool and one
 * output pool of limbs (device memory, caller-owned).  Offsets are in limbs
 * from the start of the pool.  Each operation is exactly the uniform entry
 * point's computation (same kernels' block routines), so results do not
 * depend on the batch an operation runs in.
 *   ADD/SUB: out[o1 .. o1+n) = a +- b, n = na = nb, or n = max(na, nb)
 *            with the flag BIGINT_ZEXT in `flags` (the shorter operand
 *            zero-extended); status = carry / borrow
 *   MUL:     out[o1 .. o1+na+nb) = a * b (na, nb <= BIGINT_MUL_MAX_LIMBS)
 *   DIVMOD:  u = a (na limbs), v = b (nb limbs); q at o1 (max(na-nb+1,1)
 *            limbs), r at o2 (nb limbs); status as for bigint_divmod.
 * Output ranges must not overlap each other or the inputs.               */
#define BIGINT_OP_ADD 1
#define BIGINT_OP_SUB 2
#define BIGINT_OP_MUL 3
#define BIGINT_OP_DIVMOD 4
/* ADD/SUB with operands of different lengths: zero-extend the shorter one
 * (without it such an operation is rejected with BIGINT_EINVAL). */
#define BIGINT_ZEXT 1
typedef struct {
  int32_t op;        /* BIGINT_OP_*                                       */
  int32_t na, nb;    /* limbs of a and b                                  */
  int32_t flags;     /* 0 or BIGINT_ZEXT (ADD/SUB only)                   */
  int64_t a, b;      /* input offsets (limbs)                             */
  int64_t o1, o2;    /* output offsets (limbs)                            */
} bigint_op;

/* Launch forms: one persistent launch with a device-side work queue
 * (cost-sorted, largest first); one launch per (op, size class); or the
 * steps form: the divisions with divisors of 128 limbs or more grouped into
 * classes of nearby shapes (divisors within 1/8, quotients within 1/4 plus
 * 64 limbs, at least 8 members), each class padded to one shape (u and v
 * shifted up by the same number of zero limbs: the quotient is the same,
 * the remainder comes back shifted down) and divided in the step-batched
 * form of bigint_divmod, everything else in one persistent launch.  All
 * forms are device work only (a CUDA graph can capture them) and give the
 * same results. */
#define BIGINT_BATCH_PERSISTENT 0
#define BIGINT_BATCH_PER_CLASS 1
#define BIGINT_BATCH_STEPS 2

typedef struct bigint_batch bigint_batch; /* opaque host-side plan */

/* Validates the host array of descriptors, sorts and groups it, and picks
 * the launch shapes.  Host memory only; the descriptors are copied.
 * Returns BIGINT_EINVAL for a malformed descriptor. */
int bigint_batch_create(const bigint_op *ops_host, int64_t nops,
                        bigint_batch **batch);
/* Device workspace bytes the batch needs (descriptors, queue, division
 * scratch for each resident CTA). */
size_t bigint_batch_workspace(const bigint_batch *batch);
/* Copies the plan into the workspace (asynchronous on `stream`; the host
 * copy stays owned by the batch until bigint_batch_destroy). */
int bigint_batch_upload(bigint_batch *batch, void *workspace, size_t bytes,
                        void *stream);
/* Runs the batch (device work only: a counter reset and one kernel, or one
 * kernel per class), so it can be captured in a CUDA graph.  status: one
 * int32 per operation, or NULL. */
int bigint_batch_launch(const bigint_batch *batch, const uint64_t *in_pool,
                        uint64_t *out_pool, int32_t *status, void *workspace,
                        int mode, void *stream);
/* ---- ragged views and the per-operation ragged forms ---------------------
 * A view is a batch of `count` integers of possibly different lengths whose
 * limbs lie in DEVICE memory at `data` (8-byte aligned): instance i has
 * nlimbs[i] limbs starting offset[i] limbs from data -- or, with offset /
 * nlimbs NULL, the uniform layout of n limbs at i*n.  offset and nlimbs are
 * HOST arrays (the shapes are needed on the host to plan the launch), read
 * during the call only.  bigint_batch_cview is the read-only view of the
 * inputs, bigint_batch_view the view of the outputs.                       */
typedef struct {
  const uint64_t *data;   /* device limbs                                   */
  const int64_t *offset;  /* host, count entries, or NULL (instance i at i*n) */
  const int32_t *nlimbs;  /* host, count entries, or NULL (every length n)  */
  int64_t count;
  int32_t n;              /* uniform length where nlimbs is NULL            */
} bigint_batch_cview;
typedef struct {
  uint64_t *data;
  const int64_t *offset;
  const int32_t *nlimbs;
  int64_t count;
  int32_t n;
} bigint_batch_view;

/* The operations of Sec. V over ragged batches, instance by instance, as
 * one persistent launch of the batched form (the kernels above: each
 * instance's result is that of the uniform entry point).  All views have
 * the same count; the output lengths must be the results' lengths:
 *   add / sub: max(na, nb) limbs (na == nb unless flags has BIGINT_ZEXT,
 *     which zero-extends the shorter operand); carry_out / borrow_out:
 *     count int32 (0 or 1), or NULL
 *   mul: na + nb limbs (na, nb <= BIGINT_MUL_MAX_LIMBS)
 *   divmod: q of max(nu - nv + 1, 1) limbs, r of nv limbs; status as for
 *     bigint_divmod, count int32, or NULL
 * Output instances must not overlap each other or the inputs.  workspace:
 * bigint_batch_views_workspace(op, a, b) bytes of device memory, 256-byte
 * aligned.  The call plans on the host and copies the plan to the device
 * from pageable memory, which waits for the stream's earlier work; the
 * launch itself is asynchronous.  BIGINT_EINVAL for malformed views or
 * mismatched lengths, BIGINT_ENOMEM for a short workspace.                */
size_t bigint_batch_views_workspace(int op, const bigint_batch_cview *a,
                                    const bigint_batch_cview *b);
int bigint_batch_add(const bigint_batch_cview *a, const bigint_batch_cview *b,
                     const bigint_batch_view *out, int32_t *carry_out, int flags,
                     void *workspace, size_t bytes, void *stream);
int bigint_batch_sub(const bigint_batch_cview *a, const bigint_batch_cview *b,
                     const bigint_batch_view *out, int32_t *borrow_out, int flags,
                     void *workspace, size_t bytes, void *stream);
int bigint_batch_mul(const bigint_batch_cview *a, const bigint_batch_cview *b,
                     const bigint_batch_view *out, void *workspace, size_t bytes,
                     void *stream);
int bigint_batch_divmod(const bigint_batch_cview *u, const bigint_batch_cview *v,
                        const bigint_batch_view *q, const bigint_batch_view *r,
                        int32_t *status, void *workspace, size_t bytes, void *stream);

/* A mixed batch of bigint_op descriptors in one call: plan, upload and
 * launch (mode: BIGINT_BATCH_PERSISTENT or BIGINT_BATCH_PER_CLASS) -- the
 * create / upload / launch / destroy sequence above without keeping the
 * plan (for a batch run once; keep the plan with bigint_batch_create to
 * launch it repeatedly or capture it in a CUDA graph).  workspace:
 * bigint_batch_run_workspace(ops, nops) bytes, 256-byte aligned.           */
size_t bigint_batch_run_workspace(const bigint_op *ops, int64_t nops);
int bigint_batch_run(const bigint_op *ops, int64_t nops, const uint64_t *in_pool,
                     uint64_t *out_pool, int32_t *status, void *workspace, size_t bytes,
                     int mode, void *stream);

/* Autotuner of the batched form: times the persistent launch on this batch
 * (synchronous) in each candidate form -- large products on the tensor
 * cores (CTAs of 544 threads holding their SM's tensor memory; only if the
 * batch has such products) or integer products only with CTAs of 256, 384
 * or 512 threads -- and keeps the fastest for this batch (an integer CTA
 * size also as the process default for new batches); *best_threads
 * receives the chosen CTA size (544 for the tensor-core form). */
int bigint_batch_tune(bigint_batch *batch, const uint64_t *in_pool,
                      uint64_t *out_pool, int32_t *status, void *workspace,
                      size_t bytes, void *stream, int *best_threads);
void bigint_batch_destroy(bigint_batch *batch);

/* Autotuner for the multiply (the paper tunes its kernels' thresholds by
 * measurement, Sec. III): times, on this batch (synchronous), the
 * tensor-core product with its tile chosen by size and forced to 64, 128
 * and 256 output columns per tile -- the tile also fixes how many CTAs share
 * an SM (three, two, one) -- and the integer products (29-bit digits with
 * 16-column chunks, 28-bit digits with 8-column chunks, and for square
 * products one level of Karatsuba); records the fastest for the operands'
 * size class (class c: longer operand of [2^c, 2^(c+1)) limbs; variant 0
 * uses it from then on) and returns it in *best_variant (a
 * bigint_set_variant(0, .) number).  Results do not depend on the choice. */
int bigint_tune(const uint64_t *a, const uint64_t *b, uint64_t *out,
                int64_t count, int32_t na, int32_t nb, void *stream,
                int *best_variant);
/* Saves / loads the tuning table (multiply variant per size class, batch
 * CTA size) as a small JSON file keyed by the GPU name.  Loading a table
 * written for another GPU, or one with an unknown variant, returns
 * BIGINT_EINVAL and changes nothing. */
int bigint_save_tuning(const char *path);
int bigint_load_tuning(const char *path);

/* ---- fused programs (Sec. VI, Tables I and II) ----------------------------
 * bigint_add_chain: out = a + b + ... + b with k additions (1 <= k <= 255),
 * each a full carry-propagating addition mod B^n (Table I's 6-Add is k = 6);
 * carry_out[i] = floor((a + k b) / B^n) (may be NULL).  One launch, the
 * running sum held in registers: global traffic is that of one addition.
 * a, b, out: count x n limbs, device pointers, out may alias a.
 *
 * bigint_poly: out = (a a + b)(b b + b) + a b mod B^n (Table II's Poly: four
 * multiplications, three additions, every value kept to n limbs as the
 * paper's same-width multiply and add).  One persistent launch; products of
 * n >= 256 limbs run on the tensor cores, with the smallest tile that holds
 * a low n x n product's n / 16 columns (up to four CTAs per SM for n <=
 * 1024, two up to 2048, one above); intermediates live in `workspace`
 * (device memory of bigint_poly_workspace(count, n) bytes: 3 n limbs per
 * resident CTA, small enough to stay in L2).  a, b, out: count x n limbs,
 * out disjoint from a and b.  n <= BIGINT_MUL_MAX_LIMBS.
 * Both return BIGINT_EINVAL for bad shapes or pointers, BIGINT_ENOMEM for a
 * short workspace, BIGINT_ECUDA for a launch error.                         */
int bigint_add_chain(const uint64_t *a, const uint64_t *b, uint64_t *out, uint8_t *carry_out,
                     int64_t count, int32_t n, int32_t k, void *stream);
size_t bigint_poly_workspace(int64_t count, int32_t n);
int bigint_poly(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int32_t n,
                void *workspace, size_t bytes, void *stream);

/* ---- host-buffer entry points --------------------------------------------
 * The operations above on operands and results in HOST memory.  The library
 * splits the batch into chunks and overlaps, on three streams of its own,
 * the host->device copy of chunk i+1, the kernel of chunk i and the
 * device->host copy of chunk i-1 (two staging slots in `workspace`, device
 * memory of `bytes` bytes, 256-byte aligned); the call returns when all
 * results are in host memory (synchronous; not thread-safe).  Host buffers
 * should be pinned (cudaHostAlloc / cudaHostRegister) for the copies to
 * overlap; pageable buffers give the same results more slowly.  Layouts and
 * result semantics are those of the device entry points: a, b instance-major
 * limb arrays, carry/borrow one byte and status one int32 per instance (these
 * may be NULL: not returned).  Returns BIGINT_EINVAL for bad shapes, null or
 * misaligned buffers, BIGINT_ENOMEM if two slots of one instance do not fit
 * `bytes`, BIGINT_ECUDA for a CUDA error.  The paper has no counterpart
 * (its measurements keep data on the device); this is the library's own
 * end-to-end path.
 *
 * bigint_host_workspace: bytes of workspace for two staging slots of
 * `chunk` instances of op (BIGINT_OP_ADD .. BIGINT_OP_DIVMOD; for divmod
 * na = nu, nb = nv); 0 for invalid arguments.  A call cuts its batch into
 * chunks of at most a quarter of the batch (and what two slots of the
 * given workspace hold) and uses as many slots as the workspace holds, up
 * to one per chunk and 8: a larger workspace lets more copy-ins run ahead. */
size_t bigint_host_workspace(int op, int64_t chunk, int32_t na, int32_t nb);
int bigint_add_host(const uint64_t *a, const uint64_t *b, uint64_t *out, uint8_t *carry_out,
                    int64_t count, int32_t n, void *workspace, size_t bytes);
int bigint_sub_host(const uint64_t *a, const uint64_t *b, uint64_t *out, uint8_t *borrow_out,
                    int64_t count, int32_t n, void *workspace, size_t bytes);
int bigint_mul_host(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count,
                    int32_t na, int32_t nb, void *workspace, size_t bytes);
int bigint_divmod_host(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                       int32_t *status, int64_t count, int32_t nu, int32_t nv,
                       void *workspace, size_t bytes);
/* The same, enqueued only (returns before the copies and kernels finish, so
 * the copies of one call overlap the kernels of the next): op is
 * BIGINT_OP_ADD .. BIGINT_OP_DIVMOD; out0 = result / quotient, out1 = the
 * remainder (divmod; else unused), aux = carry / borrow bytes (add, sub) or
 * int32 statuses (divmod), may be NULL; na = nb = n for add and sub.  Host
 * buffers and the workspace must stay untouched until bigint_host_sync()
 * returns, which waits for every enqueued call of the current device (and
 * returns BIGINT_ECUDA if one failed).  Calls that share a workspace are
 * ordered by the library.                                                   */
int bigint_host_async(int op, const uint64_t *a, const uint64_t *b, uint64_t *out0,
                      uint64_t *out1, void *aux, int64_t count, int32_t na, int32_t nb,
                      void *workspace, size_t bytes);
int bigint_host_sync(void);

/* ---- tuning and measurement ---------------------------------------------
 * Selects the kernel variant an operation uses from now on (process-wide,
 * not thread-safe; call it before launching work).  op 0 = multiply:
 *   variant 0 (default): chosen by operand size from GB300 measurements (the
 *   tensor-core product from a shorter operand of 256 limbs, integer
 *   products below), or the variant bigint_tune recorded for the size class
 *   variant 8: integer product, 29-bit digits, 16-column chunks
 *   variant 9: integer product, 28-bit digits, 8-column chunks
 *   variant 10: one level of Karatsuba (square full products of at least 64
 *   limbs; otherwise variant 8) over variant 8's half products
 *   variant 11: one warp per instance, 128-bit column sums (operands of at
 *   most 64 limbs; otherwise variant 9) -- what the products inside
 *   step-batched divisions use for operands of at most 64 limbs
 *   variant 12: the tensor-core product -- the digit convolution of the
 *   schoolbook product (Sec. V-B) as fp16 matrix products (tcgen05.mma)
 *   over signed base-256 digits with exact fp32 accumulation -- with its
 *   tile chosen by a cost model of its MMAs; bit-identical results.  Needs the shorter operand to fit shared memory
 *   (about 10700 limbs; otherwise variant 8).
 *   variants 13, 14, 15: variant 12 with 128-digit x blocks and tiles of
 *   64, 128, 256 output columns (three, two, one CTAs per SM)
 *   variants 16, 17: variant 12 with x blocks of 64 or 32 digits (128-column
 *   tiles, two CTAs per SM: each MMA 2 or 4 times as wide)
 *   Variants 13-17 also force the shape of the tensor-core products inside
 *   divisions (where a forced shape cannot take a product, the model's
 *   choice runs); variants 8-10 keep those on the integer pipes.
 * op 1 = division (divmod, shinv, divmod_inv):
 *   variant 0 (default): bigint_divmod on divisors of 128 limbs or more in
 *   the step-batched form (see bigint_divmod), everything else as variant 1
 *   variant 1: one CTA per division; operands of 1536 limbs and more run in
 *   a kernel that holds its SM's tensor memory and computes products whose
 *   shorter operand has at least 256 limbs on the tensor cores (as variant
 *   12 of the multiply); smaller divisions use the integer products
 *   variant 2: one CTA per division, integer products (blk_mul) only
 *   variant 3: as 0, with the step-batched form for divisors of 8 limbs
 *   and more
 * op 2 = ragged batches (bigint_batch_*, for batches created afterwards):
 *   variant 0 (default) or 1: a batch with multiplications or divisions
 *   whose products have a shorter operand of 256 limbs or more runs them in
 *   512-thread launches that hold their SM's tensor memory and compute those
 *   products on the tensor cores (the CTA size tuner then has no choice)
 *   variant 2: integer products only
 * Returns BIGINT_EINVAL for an unknown op or variant.                      */
int bigint_set_variant(int op, int variant);

/* BIGINT_ETIMEOUT if a tensor-core product (multiply variant 12 or a
 * division's tensor-core product) stopped at one of its device wait limits
 * (about one second per wait; its outputs are then undefined, and a
 * division reports BIGINT_ETIMEOUT in its status) since the previous call,
 * else BIGINT_OK.  Synchronises the device and
 * clears the record.  The paper has no counterpart: the waits exist only in
 * the tensor-core schedule, which hands work between threads and the
 * tensor cores through shared-memory barriers.                              */
int bigint_check_timeout(void);

/* Sets the cycle limit of the device-side waits of the tensor-core products
 * for every launch from now on: cycles > 0 the limit, 0 the default (about
 * one second).  cycles < 0 injects a timeout for testing: every such wait
 * first waits for the tensor-core work it guards, then spins for -cycles
 * cycles on a flag that nothing sets and gives up, so that a product stops
 * as at a real timeout (BIGINT_ETIMEOUT from bigint_check_timeout and in a
 * division's status, tensor memory released, the device usable
 * afterwards).  An ordinary product cannot be made to time out with a low
 * positive limit: its waits find the work done at their first probe.  The
 * waits that guard the release of tensor memory always keep the full
 * limit.  Synchronous; process-wide; not thread-safe.  The paper has no
 * counterpart (its kernels have no such waits).                            */
int bigint_set_wait_limit(long long cycles);

/* Number of kernels the library has launched in this process so far (every
 * launch of every entry point, counted when it is enqueued), so that a
 * caller can report how many kernels a piece of work took. */
unsigned long long bigint_kernel_launches(void);

/* The multiply variant (1..12) a full na x nb product runs with the current
 * settings (default choice, tuning table, fallbacks), so that measurements
 * can count the digit products of the algorithm actually used. */
int bigint_mul_variant_for(int32_t na, int32_t nb);

/* Integer-pipe throughput probe used for the multiply roofline: every SM
 * runs a register-only loop of one instruction form at full occupancy and
 * times itself with the SM cycle counter.  Returns thread-level operations
 * per SM per SM clock cycle (*ops_per_clk_sm) and the SM clock seen
 * (*sm_mhz).
 *   variant 0: 32x32->64-bit multiply-add (mad.wide.u32, IMAD.WIDE)
 *   variant 1: 32-bit multiply-add, low half (mad.lo.u32)
 *   variant 2: 32-bit multiply-add, high half (mad.hi.u32)
 *   variant 3: the multiply kernel's inner step (one mad.wide.u32 per digit
 *              product into 8 column accumulators), ops = digit products
 * Synchronous; allocates two small device buffers for the duration.       */
int bigint_probe_int_throughput(int variant, double *ops_per_clk_sm,
                                double *sm_mhz);

#ifdef __cplusplus
}
#endif
#endif /* BIGINT_H */
