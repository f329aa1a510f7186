// tccore.cuh -- exact products on the 5th-generation tensor cores, one CTA
// per product (used by the batched multiply and by the division kernel).
//
// The schoolbook product of Sec. V-B is a convolution of digit sequences:
// coefficient s of x*y is sum_i x_i y_(s-i).  This kernel evaluates that
// convolution as fp16 matrix products with fp32 accumulators (tcgen05.mma,
// accumulators in tensor memory), exactly:
//
//  * Digits.  Each operand is read as base-256 digits (its bytes) recoded to
//    signed digits e_i = sext(d_i) + top_bit(d_(i-1)) in [-128, 128] plus
//    the carry digit e_(8n) = top_bit(d_(8n-1)) in {0, 1}; sum e_i 256^i is
//    the operand again.  y's carry digit falls in the last Toeplitz block y
//    already has; x's costs an extra block of 128 digits, so with XC =
//    false x goes without it: its digits spell x_s = x - t_x B^nx (t_x its
//    top bit), an nx-limb x fills exactly nx/16 blocks (a 1024-limb product
//    has 128 output columns, not 129, and fits the two-CTA tile), and
//    x y = x_s y + t_x y B^nx is restored by one carry-scan addition at the
//    end when t_x = 1.  Every digit is an exact fp16 value and every digit
//    product is at most 2^14 in magnitude.
//  * Blocks.  Output coefficients are grouped in columns of 128 (column c
//    holds s = 128 c + t).  With x cut into blocks of 128 digits,
//      coef(128 c + t) = sum_e sum_i A_e[t][i] * x[128 (c - e) + i],
//      A_e[t][i] = y[128 e + t - i]            (a Toeplitz block of y),
//    i.e. for each e one MMA with M = 128 (t), K = 128 (i), N = columns c,
//    whose B operand is x shifted by e blocks.  Summing over e is the K loop.
//  * Layouts (no swizzle, K-major core matrices of 8 rows x 16 bytes).
//    B: x is stored once per instance as 16-byte chunks "8 digits of block
//    p", chunk (p, h) at (p + 16 + h P) * 16 bytes; 8 consecutive blocks are
//    then 128 bytes apart (stride offset 128) and the 16 digit groups of a
//    block P*16 bytes apart (leading offset), so shifting by e blocks is a
//    shift of the descriptor's start address by 16 e bytes.  A: storing the
//    rows in reverse (TMEM lane t' holds t = 127 - t'), A_e[t'][i] depends
//    on t' + i only, so its 8x8 core matrix (g, h) depends on g + h only:
//    core matrix j = "8 rows of 8 digits, row r starting at digit 8j + r" of
//    the reversed digit stream, and a descriptor with leading and stride
//    offsets both 128 bytes reads the whole 128 x 128 Toeplitz block from
//    31 such 128-byte core matrices (a group of G blocks needs 16 G + 15).
//  * Exactness.  Each accumulator sums at most G x 128 products between
//    drains: every partial sum is an integer of magnitude at most
//    G * 2^21 <= 2^24 (G = 8), and all integers up to 2^24 are exact in fp32
//    and in the tensor core's fp32 accumulation (the byte pattern 0x7F80...
//    makes every digit +-128 and every product of a column the same sign,
//    reaching 2^24 exactly; it is a parity case).  The accumulator is then
//    converted exactly (cvt.rni) and added to int32 column sums in
//    registers; a column sum is at most (8 n + 1) * 2^14 < 2^31 for
//    n <= 16383 limbs.
//  * Output.  Each limb j is V_j = sum_k (coef(8j+k) + 2^31) 2^(8k) (biased
//    so that all terms are unsigned): the limb's low 64 bits plus a high word
//    that goes to limb j + 1, and the bias sum 2^31 sum_s 2^(8s) -- the word
//    0x8080808080808080 in every limb, 0x8080808080000000 in limb 0 -- to
//    subtract; both in one pass per tile (blk_add_then_sub: the carry scan
//    of Fig. 3 for the sum, then as a borrow chain for the difference).
//
// Schedule: a persistent CTA of 2 NT drain threads and one issuer warp loops
// over instances; per instance over tiles of NT output columns; per tile
// over groups of G Toeplitz blocks (8; 7 for NT = 64; 4 when the longer
// Hankel buffers do not fit).  Fewer, larger groups matter: every drain
// reads the whole accumulator out of tensor memory.  The issuer warp's lane
// 0 issues a group's MMAs into one of two NT-column fp32 accumulators in
// tensor memory and commits them to an mbarrier (it blocks on the tensor
// core's shallow instruction queue for most of a group, hence a warp of its
// own); meanwhile the drain threads drain the other accumulator and build
// the next group's Hankel core matrices (double buffered; each y digit of
// the group recoded once into a staging run, the rows copied out of it),
// then report that buffer and accumulator ready on an mbarrier, on which
// the issuer waits before the next group.
// NT = 256 (one CTA per SM, all of its tensor memory) serves large
// products; NT = 128 (two CTAs per SM) and NT = 64 (three) keep several
// issuers per SM for small ones, where an MMA's time is its A operand's
// shared-memory read rather than N.  Split mode computes one tile of a
// product per call, so that a product's tiles can run on different CTAs.
// Every wait has a cycle limit; a CTA that reaches it stops, records the
// event for bigint_check_timeout() and releases its tensor memory.
#pragma once
#include <cuda_fp16.h>

#include "blockops.cuh"

namespace bigint {
namespace tcm {

// G: Toeplitz blocks per accumulation group; KB: digits per x block (the
// K of one Toeplitz block).  A group's Hankel buffer holds 16 G + KB / 8 - 1
// core matrices.
__host__ __device__ constexpr int hankel_blocks(int G, int KB = 128) { return 16 * G + KB / 8 - 1; }
// 32-bit words of one copy of a group's Hankel staging run (hank_build).
template <int G, int KB = 128>
__host__ __device__ constexpr int hank_stage_words() { return 4 * hankel_blocks(G, KB) + 20; }
constexpr int ZB = 18;           // zero core matrices (operand of the clearing MMA)
// NT: output columns per tile (= MMA N at most); 2 NT threads, 2 NT TMEM
// columns (two accumulators).
constexpr long long WAIT_LIMIT = 1ll << 31;  // cycles, about one second
// kind::f16 instruction descriptor: fp32 accumulator (bits 4-5 = 1), fp16 A
// and B (bits 7-12 = 0), both K-major (bits 15, 16 = 0), M = 128 (bits
// 24-28 = M >> 4); N >> 3 goes to bits 17-22.
constexpr uint32_t IDESC_M128 = (1u << 4) | ((uint32_t)(128 >> 4) << 24);

// Set when a CTA gives up at a wait limit (one copy per translation unit;
// each unit that launches tensor-core products reads and clears its own
// copy through take_timeout_here, and bigint_check_timeout asks them all).
static __device__ int g_timeout = 0;
// Cycle limit of the waits of a product (one copy per translation unit, set
// through set_wait_limit_here; the default is WAIT_LIMIT).  Lowering it
// makes ordinary products give up, which is how the timeout path is tested;
// the waits of tc_release always use the full WAIT_LIMIT, so tensor memory
// is never freed while an MMA that was committed may still write to it.
static __device__ long long g_wait_limit = WAIT_LIMIT;
// A flag nothing sets: with a negative g_wait_limit every wait of a product
// first waits (full limit) for its phase, so no MMA it guards is left in
// flight, and then runs out on this flag after -g_wait_limit cycles -- a
// timeout made on purpose, so that tests can drive the timeout path (a
// positive limit cannot: the phases a product waits for have completed by
// the time its first probe returns).
static __device__ int g_never_set = 0;

struct Layout {
  int mx;    // x blocks of KB digits (8 nx digits, + the carry digit if XC)
  int ey;    // last Toeplitz block index of y (e in [0, ey])
  int ctot;  // output columns with nonzero coefficients: mx + S ey + S - 1 (S = 128 / KB)
  int ptot;  // stored x blocks (16 zero blocks on each side; odd)
  // byte offsets in dynamic shared memory: x (B layout), zero core matrices,
  // the two Hankel buffers, the Hankel staging run, the column-sum transpose
  // area, high words of the tile's limbs
  uint32_t xs, z, h0, h1, st, cs, his, total;
};

// KB = 128: one output column per 128 digits, each coefficient in one TMEM
// row.  KB = 64 or 32 (narrow x blocks): columns of KB digits whose 128-row
// windows overlap, S = 128 / KB rows per coefficient (below).  Shared memory:
// x, the zero core matrices, two Hankel buffers, the Hankel staging run,
// the column-sum transpose area (32 columns, then S - 1 columns carried from
// the previous 32) and the high words of the tile's limbs.  The last two
// are live only between a tile's last drain and the next tile's first
// Hankel build, when no MMA reads the Hankel buffers: with KB = 128 they
// share those buffers' memory where it is large enough (a 512-limb product
// then fits four CTAs per SM instead of three); otherwise the staging run
// lies in the transpose area, which is free while a tile's groups run.
template <int NT, int G, bool XC = true, int KB = 128>
__host__ __device__ inline Layout layout(int nx, int ny) {
  static_assert(KB == 128 || KB == 64 || KB == 32, "x blocks of 128, 64 or 32 digits");
  constexpr int HB = hankel_blocks(G, KB), S = 128 / KB, R = KB / 8;
  Layout L;
  L.mx = (8 * nx + (XC ? 1 : 0) + KB - 1) / KB;
  // block e meets y digits 128 e - KB + 1 .. 128 e + 127
  L.ey = (8 * ny + KB - 1) / 128;
  // the MMAs write columns up to mx - 1 + S ey; the rows of the last ones
  // reach S - 1 columns further
  L.ctot = L.mx + S * L.ey + S - 1;
  L.ptot = (L.mx + 32) | 1;  // odd: the h-rows of a warp's x stores hit distinct banks
  L.xs = 0;
  L.z = (uint32_t)L.ptot * 16u * R;
  L.h0 = L.z + ZB * 128;
  L.h1 = L.h0 + HB * 128;
  const uint32_t cs_bytes = (32 + S - 1) * 128 * 4, his_bytes = NT * R * 4;
  if (S == 1 && cs_bytes + his_bytes <= 2u * HB * 128) {
    L.cs = L.h0;
    L.his = L.h0 + cs_bytes;
    L.st = L.h1 + HB * 128;
    L.total = L.st + 2 * hank_stage_words<G, KB>() * 4;
  } else {
    L.cs = L.h1 + HB * 128;
    L.st = L.cs;
    L.his = L.cs + cs_bytes;
    L.total = L.his + his_bytes;
  }
  return L;
}

// ---- PTX wrappers ----------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared memory matrix descriptor, no swizzle: start address, leading
// (K-direction) and stride (M/N-direction) byte offsets, all >> 4, and the
// fixed version bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
      : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// One arrival (release semantics at CTA scope).
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

// Named barrier 2 over the first NTH threads of the CTA with an OR of v over
// them: every participant gets the same answer.
template <int NTH>
__device__ __forceinline__ bool bar_or_drain(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 2, %2, q;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(NTH)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking probe of the phase with this parity.
__device__ __forceinline__ bool mbar_test_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// Waits for the phase with this parity to complete; false after `limit`
// cycles (default: the launch's g_wait_limit).  try_wait suspends the
// thread in hardware for a while before it reports failure, longer than a
// small product takes, so a lowered limit (the test of the timeout path)
// polls with the non-blocking test_wait instead, which sees the limit pass.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  if (limit < WAIT_LIMIT) {
    while (!mbar_test_wait(mbar, parity))
      if (clock64() - t0 > limit) return false;
    return true;
  }
  while (!mbar_try_wait(mbar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}
// The launch's wait limit (g_wait_limit), read once per CTA: a load of it
// per wait put an L2 round trip in front of every group's MMAs.
__device__ __forceinline__ long long wait_limit_here() {
  return *(volatile long long *)&g_wait_limit;
}
// Waits with the launch's limit `lim` (wait_limit_here()): lim >= 0 the
// cycle limit, lim < 0 the injected timeout of g_never_set.  A phase that
// has already completed is seen by a non-blocking probe first, which costs
// about half of a try_wait on a completed phase (~180 vs ~340 cycles).
__device__ __forceinline__ bool mbar_wait_lim(uint32_t mbar, uint32_t parity, long long lim) {
  if (lim >= 0) return mbar_test_wait(mbar, parity) || mbar_wait(mbar, parity, lim);
  if (!mbar_wait(mbar, parity, WAIT_LIMIT)) return false;
  const long long t0 = clock64();
  while (*(volatile int *)&g_never_set == 0)
    if (clock64() - t0 > -lim) return false;
  return true;
}

__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_smem),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Orders this thread's shared memory stores before later tensor-core reads.
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// 32 TMEM lanes (one per thread of the warp) x 16 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Asks L2 for the 16-byte-aligned part of [p, p + bytes) (no completion to
// wait for): the next instance's operands come in from HBM while this one
// is computed, so its first loads meet L2 rather than HBM.
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes) {
  const uintptr_t a = (reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15;
  const uintptr_t e = (reinterpret_cast<uintptr_t>(p) + bytes) & ~(uintptr_t)15;
  if (e > a)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(e - a))
                 : "memory");
}

// ---- digits ----------------------------------------------------------------
// Recoded digit k of a limb (k = 0..7): its byte k sign-extended plus the top
// bit of byte k - 1 (byte -1 = the top byte of the limb below), so a number
// of n limbs spells sum_k e_k 256^k with digits in [-128, 128] and a carry
// digit (the top bit of its last byte) at position 8n.
// Plain (coherent) loads of the limbs: inside the division and program
// kernels an operand can be a value the same CTA wrote earlier in the launch
// (a Newton iterate in a reused buffer), which the non-coherent read-only
// path may not see.
//
// The digits of limb v (below = the limb underneath) as 16-bit lanes biased
// by 0x6600: lane j of ev is digit 2j, lane j of od digit 2j + 1; dm1 is
// digit 7 of below (position -1).  Each lane stays in [0x6580, 0x6680], so
// the lanes of a 64-bit sum never carry into each other.
struct Digits16 {
  uint64_t ev, od;
  uint32_t dm1;
};

__device__ __forceinline__ Digits16 recode16(uint64_t v, uint64_t below) {
  constexpr uint64_t LANE = 0x00FF00FF00FF00FFull, TOP = 0x0080008000800080ull;
  constexpr uint64_t ONE = 0x0001000100010001ull, BIAS = 0x6600660066006600ull;
  const uint64_t E = v & LANE, O = (v >> 8) & LANE;
  Digits16 d;
  d.ev = BIAS + E - ((E & TOP) << 1) + (((O >> 7) & ONE) << 16) + (below >> 63);
  d.od = BIAS + O - ((O & TOP) << 1) + ((E >> 7) & ONE);
  const uint32_t b7 = (uint32_t)(below >> 56);
  d.dm1 = 0x6600u + b7 - ((b7 & 0x80u) << 1) + ((uint32_t)(below >> 55) & 1u);
  return d;
}

// Two biased lanes (0x6600 + v, |v| <= 128) to an fp16 pair: 0x6600 + v is
// the fp16 pattern of 1536 + v (ulp 1 there), and subtracting 1536 is exact.
__device__ __forceinline__ uint32_t unbias_h2(uint32_t m) {
  const __half2 a = *reinterpret_cast<const __half2 *>(&m);
  const __half2 r = __hsub2(a, __half2half2(__ushort_as_half((unsigned short)0x6600u)));
  return *reinterpret_cast<const uint32_t *>(&r);
}

// x blocks p in [-16, mx + 16) into the B layout: with R = KB / 8 limbs per
// block, chunk (p, h) = digits KB p + 8 h .. + 8 = the digits of limb R p +
// h, stored at ((p + 16) + h ptot) * 16.  Without XC the digits past limb
// nx - 1 are 0 (they spell x - top_bit(x) B^nx).  Thread i takes limb
// i - 16 R, so a warp's loads are coalesced; a thread issues the loads of
// four limbs before it recodes any, so their latencies overlap.
template <bool XC, int KB = 128>
__device__ __forceinline__ void fill_x(uint8_t *xs, const uint64_t *x, int nx, int ptot) {
  constexpr int U = 4, R = KB / 8, LR = KB == 128 ? 4 : (KB == 64 ? 3 : 2);
  const int total = R * ptot, step = (int)blockDim.x;
  for (int i0 = threadIdx.x; i0 < total; i0 += U * step) {
    uint64_t v[U], below[U];
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int i = i0 + u * step, L = i - 16 * R;
      v[u] = (L >= 0 && L < nx && i < total) ? x[L] : 0ull;
      below[u] = (L >= 1 && L - 1 < nx && (XC || L < nx) && i < total) ? x[L - 1] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < U; u++) {
      const int i = i0 + u * step;
      if (i < total) {
        const int pp = i >> LR, h = i & (R - 1);
        const Digits16 d = recode16(v[u], below[u]);
        const uint32_t el = (uint32_t)d.ev, eh = (uint32_t)(d.ev >> 32);
        const uint32_t ol = (uint32_t)d.od, oh = (uint32_t)(d.od >> 32);
        *reinterpret_cast<uint4 *>(xs + (size_t)(pp + h * ptot) * 16) = make_uint4(
            unbias_h2(__byte_perm(el, ol, 0x5410)), unbias_h2(__byte_perm(el, ol, 0x7632)),
            unbias_h2(__byte_perm(eh, oh, 0x5410)), unbias_h2(__byte_perm(eh, oh, 0x7632)));
      }
    }
  }
}

// Hankel core matrices of the group whose last block is eb: matrix j, row r,
// element w = recoded y digit at 128 eb + 127 - 8 j - r - w.  Row s = 8 j + r
// is the run D[s .. s + 8) of the reversed digit sequence D[i] = digit at
// 128 eb + 127 - i, so each digit is recoded once into D and the rows are
// copied out of it: D is held twice in the staging area (the second copy one
// element ahead, so that every run starts on a 4-byte boundary in one of
// them; the copies 16 banks apart).  Thread t <= HB recodes limb
// 16 eb + 15 - t, i.e. D[8 t .. 8 t + 8), from that limb and the one below;
// hank_load fetches them (so the loads can be issued ahead of a wait) and
// hank_build, called by threads 0 .. NTH - 1 (NTH a multiple of 32, named
// barrier 1), writes D and the rows.
struct HankLimbs {
  uint64_t hi, lo;
};

template <int G, int KB = 128>
__device__ __forceinline__ HankLimbs hank_load(const uint64_t *y, int ny, int eb, int t) {
  constexpr int HB = hankel_blocks(G, KB);
  HankLimbs v{0ull, 0ull};
  if (t <= HB) {
    const int64_t U = 16ll * eb + 15 - t;
    if (U >= 0 && U < ny) v.hi = y[U];
    if (U >= 1 && U - 1 < ny) v.lo = y[U - 1];
  }
  return v;
}


template <int G, int NTH, int KB = 128>
__device__ __forceinline__ void hank_build(uint8_t *hb, uint8_t *st, HankLimbs v, int t) {
  constexpr int HB = hankel_blocks(G, KB);
  static_assert(HB + 1 <= NTH && NTH % 32 == 0, "one limb per staging thread");
  static_assert(2 * hank_stage_words<G, KB>() * 4 <= 32 * 128 * 4,
                "staging fits the 32 columns of the column-sum area");
  uint32_t *D0 = reinterpret_cast<uint32_t *>(st), *D1 = D0 + hank_stage_words<G, KB>();
  if (t <= HB) {
    // D[8 t + w] = digit 7 - w of limb U; the second copy starts at D[1]
    const Digits16 d = recode16(v.hi, v.lo);
    const uint32_t el = (uint32_t)d.ev, eh = (uint32_t)(d.ev >> 32);
    const uint32_t ol = (uint32_t)d.od, oh = (uint32_t)(d.od >> 32);
    *reinterpret_cast<uint4 *>(D0 + 4 * t) =
        make_uint4(unbias_h2(__byte_perm(oh, eh, 0x7632)), unbias_h2(__byte_perm(oh, eh, 0x5410)),
                   unbias_h2(__byte_perm(ol, el, 0x7632)), unbias_h2(__byte_perm(ol, el, 0x5410)));
    *reinterpret_cast<uint4 *>(D1 + 4 * t) =
        make_uint4(unbias_h2(__byte_perm(eh, oh, 0x5432)), unbias_h2(__byte_perm(eh, ol, 0x7610)),
                   unbias_h2(__byte_perm(el, ol, 0x5432)), unbias_h2(__byte_perm(el, d.dm1, 0x5410)));
  }
  asm volatile("bar.sync 1, %0;" ::"n"(NTH) : "memory");
  for (int s = t; s < 8 * HB; s += NTH) {
    const uint32_t *p = ((s & 1) ? D1 : D0) + (s >> 1);
    *reinterpret_cast<uint4 *>(hb + 16 * s) = make_uint4(p[0], p[1], p[2], p[3]);
  }
}

// Thread 0: the MMAs of one group (blocks ea..eb) into the accumulator at
// TMEM column dtm, then a commit to mbar.  Block e (y digits around 128 e)
// meets x block p in output column p + S e (S = 128 / KB); only the columns
// of the tile that meet x are computed, widened to multiples of 16; the
// group's first MMA overwrites the accumulator if it spans the group's
// columns (group_span), otherwise a clearing MMA with a zero A operand over
// those columns comes first.
// Tile columns [lo, hi) (multiples of 16) that the MMAs of blocks ea..eb
// write: block e meets columns [max(c0, S e), min(c0 + W, S e + mx)), both
// ends growing with e.
template <int KB = 128>
__device__ __forceinline__ void group_span(int c0, int W, int ea, int eb, int mx, int &lo,
                                           int &hi) {
  constexpr int S = 128 / KB;
  lo = ((c0 > S * ea ? c0 : S * ea) - c0) & ~15;
  hi = ((c0 + W < S * eb + mx ? c0 + W : S * eb + mx) - c0 + 15) & ~15;
}

template <int KB = 128>
__device__ __forceinline__ void issue_group(uint32_t dtm, uint32_t ha, uint32_t xs_a,
                                            uint32_t z_a, uint32_t lbo_b, int c0, int W, int ea,
                                            int eb, int mx, uint32_t mbar) {
  constexpr int S = 128 / KB;
  tc_fence_after();
  int slo, shi;
  group_span<KB>(c0, W, ea, eb, mx, slo, shi);
  bool first = true;
  for (int e = ea; e <= eb; e++) {
    const int ca = (c0 > S * e ? c0 : S * e) - c0;
    const int cb = (c0 + W < S * e + mx ? c0 + W : S * e + mx) - c0;
    const int lo = ca & ~15, hi = (cb + 15) & ~15;
    const uint32_t id = IDESC_M128 | ((uint32_t)((hi - lo) >> 3) << 17);
    const uint32_t aa = ha + (uint32_t)(16 * (eb - e)) * 128u;
    const uint32_t ba = xs_a + (uint32_t)(c0 + lo - S * e + 16) * 16u;
    uint32_t accf = 1;
    if (first) {  // columns outside the span are neither written nor drained
      first = false;
      if (lo == slo && hi == shi) {
        accf = 0;
      } else {
        mma_f16(dtm + (uint32_t)slo, sdesc(z_a, 128, 128), sdesc(xs_a, lbo_b, 128),
                IDESC_M128 | ((uint32_t)((shi - slo) >> 3) << 17), 0);
      }
    }
    // K steps of 16 digits: A moves by 2 core matrices (256 bytes), B by two
    // leading offsets; the start-address field is bits 0-13 (address >> 4)
    uint64_t da = sdesc(aa, 128, 128), db = sdesc(ba, lbo_b, 128);
    const uint64_t step_b = (2u * lbo_b) >> 4;
#pragma unroll
    for (int s = 0; s < KB / 16; s++) {
      mma_f16(dtm + (uint32_t)lo, da, db, id, s == 0 ? accf : 1u);
      da += 16;
      db += step_b;
    }
  }
  mma_commit(mbar);
}

// Adds the accumulator (this warp's 32 lanes, its 64-column slice, the
// group's columns [lo, hi)) to the thread's int32 column sums; the values
// are integers of magnitude at most 2^24.
__device__ __forceinline__ void drain(uint32_t taddr, int cq, int lo, int hi, int (&acc)[64]) {
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const int col = 64 * cq + 16 * k;
    if (col >= lo && col < hi) {
      uint32_t r[16];
      tmem_ld16(taddr + (uint32_t)col, r);
      tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 16; i++) acc[16 * k + i] += __float2int_rn(__uint_as_float(r[i]));
    }
  }
}


// ---- per-CTA product ---------------------------------------------------------
// Shared state of the tensor-core product (static shared memory of the
// calling kernel).
struct TcShared {
  uint64_t bars[2];   // mbarriers: MMAs of the group in accumulator b completed
  uint64_t ready[2];  // mbarriers: Hankel buffer b built and accumulator b drained
                      // for the next group there (one arrival per drain warp)
  uint64_t carry_hi;  // high word carried into the next tile's first limb
  uint32_t carry;     // carry bit carried into the next tile
  uint32_t borrow;    // borrow of the bias subtraction carried into the next tile
  uint32_t tmem_slot;
};

struct TcCtx {
  uint8_t *sm;        // dynamic shared memory the products use
  uint32_t sbase;     // its shared-window address
  uint32_t tmem;      // TMEM base: 2 NT columns, two NT-column accumulators
  TcShared *sh;
  uint32_t *scr;      // BLK_SCRATCH_WORDS words for the carry scans
  uint32_t phase;     // bit b: parity of the next completion of bars[b]
  uint32_t pending;   // bit b: a commit on bars[b] not yet waited for (tc_product:
                      // kept by the issuing thread only)
  uint32_t rphase;    // issuing thread: parity of the next completion of ready[b]
  long long wlim;     // the launch's wait limit (wait_limit_here)
  bool aborted;       // a wait hit its limit: no further products
};

// Threads of a CTA running tc_product<256, G, true>: 16 drain warps and one
// issuer warp.
constexpr int TC_CTA_THREADS = 2 * 256 + 32;

// All threads of the CTA: barriers and TMEM (warp 0).
template <int NT>
__device__ void tc_init(TcCtx &c, uint8_t *sm, TcShared *sh, uint32_t *scr) {
  c.sm = sm;
  c.sbase = smem_u32(sm);
  c.sh = sh;
  c.scr = scr;
  c.phase = 0;
  c.pending = 0;
  c.rphase = 0;
  c.wlim = wait_limit_here();
  c.aborted = false;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&sh->bars[0]), 1);
    mbar_init(smem_u32(&sh->bars[1]), 1);
    mbar_init(smem_u32(&sh->ready[0]), 2 * NT / 32);
    mbar_init(smem_u32(&sh->ready[1]), 2 * NT / 32);
    fence_mbar_init();
  }
  if (threadIdx.x < 32) {
    tmem_alloc(smem_u32(&sh->tmem_slot), 2 * NT);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  c.tmem = sh->tmem_slot;
}

// All threads: after an abort, waits (bounded) for MMAs still in flight and
// records the timeout; then frees the TMEM.
template <int NT>
__device__ void tc_release(TcCtx &c) {
  if (c.aborted) {
    // groups whose commit this thread has not seen arrive (including one
    // whose wait gave up) may still be running: wait for them with the full
    // limit before the tensor memory is freed
    if (c.pending & 1u) mbar_wait(smem_u32(&c.sh->bars[0]), c.phase & 1u, WAIT_LIMIT);
    if (c.pending & 2u) mbar_wait(smem_u32(&c.sh->bars[1]), (c.phase >> 1) & 1u, WAIT_LIMIT);
    if (threadIdx.x == 0) atomicExch(&g_timeout, 1);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (threadIdx.x < 32) tmem_dealloc(c.tmem, 2 * NT);
}

// out[0..nout) = low nout limbs of x * y, by the whole CTA (blockDim = 2 NT,
// plus one issuer warp when IW), with nout <= nx + ny, x, y, out in global
// memory (out disjoint from x and y) and c.sm holding layout<NT, G>(nx,
// ny).total bytes.  Either operand may be the longer one (x is stored whole
// in shared memory, y is read group by group); the column sums stay below
// 2^31 while the shorter operand has at most 16383 limbs.
//
// Band mode (lo > 0): the tiles start at the column that holds limb lo
// (limb L0 = 16 floor(lo / 16) <= lo), so no column below it is computed;
// limbs below L0 are left untouched, and out[L0..nout) holds
// (x y - D) / B^L0 + 2^32 with D the skipped part of the convolution,
// |D| < 2^31 B^L0 / 255 (every column sum is below 2^31 in magnitude).  So for h >= lo + 2 the value
// floor(out / B^(h - L0)) is floor(x y / B^h) or one more, and never wraps
// while x y + B^h < B^nout.
//
// IW (required): one extra warp (the last) only issues MMAs; the issuing
// thread blocks while the tensor core's queue is full, so on its own warp
// that wait does not hold up any drain or Hankel build.  It waits for the
// drain warps only through the ready[] mbarriers (one per Hankel buffer and
// accumulator), never at a block barrier inside a tile (with a block
// barrier per group it spent ~0.65K cycles per group outside the MMA issue,
// by clock64 probes).
//
// Split mode (SPLIT, lo = 0): only tile `tile` (columns [NT tile, NT tile +
// W)) is computed, with no carry in, and neither the bias nor x's top bit is
// accounted for; its limbs [16 NT tile, + nl) get their internal carries and
// tile_carry[0..1] = (high word of its last column sum, carry out).  The
// tiles of one product can so run on different CTAs; tc_split_finish then
// links them (Sec. VI's per-instance work spread over several SMs).
//
// Narrow x blocks (KB = 64 or 32 digits, S = 128 / KB): an MMA then covers
// S times as many output columns for the same 4 KB A operand, which is what
// bounds narrow MMAs.  Column c holds, in its 128 rows, partial sums of the
// coefficients KB c .. KB c + 127, so coefficient KB c + u (u < KB) is the
// sum over a < S of row u + KB a of column c - a (each pair of digits is
// counted in exactly one of them: x digit KB p + k and y digit d meet in
// block e = floor((d + k) / 128) only).  The column-sum pass adds the S
// rows; the S - 1 columns before each run of 32 are kept in shared memory,
// and band mode starts the tiles S - 1 columns early, so that the first
// limb kept has all of its parts.  G KB <= 1024 keeps each accumulator's
// partial sums within 2^24 as for KB = 128.  Not with SPLIT.
//
// Returns false (and sets c.aborted) if a wait hit its limit.
template <int NT, int G, bool IW = false, bool XC = true, bool SPLIT = false, int KB = 128>
__device__ __forceinline__ bool tc_product(TcCtx &c, const uint64_t *x, int nx, const uint64_t *y,
                                           int ny, uint64_t *out, int nout, int lo, int tile = 0,
                                           uint64_t *tile_carry = nullptr) {
  constexpr int DRAIN = 2 * NT;                // threads that drain and build
  constexpr int THREADS = DRAIN + (IW ? 32 : 0);
  constexpr int S = 128 / KB, R = KB / 8;      // rows per coefficient, limbs per column
  static_assert(G * KB <= 1024, "partial sums of a group stay within 2^24");
  static_assert(KB == 128 || !SPLIT, "split tiles with 128-digit columns only");
  static_assert(IW, "the MMAs are issued by a warp of their own");
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool issuer = tid == DRAIN;
  const bool worker = tid < DRAIN;
  const Layout Ly = layout<NT, G, XC, KB>(nx, ny);
  uint8_t *sm = c.sm;
  const uint32_t sbase = c.sbase;
  const uint32_t xs_a = sbase + Ly.xs, z_a = sbase + Ly.z;
  const uint32_t lbo_b = (uint32_t)Ly.ptot * 16u;
  uint32_t *Cs = reinterpret_cast<uint32_t *>(sm + Ly.cs);
  uint32_t *His = reinterpret_cast<uint32_t *>(sm + Ly.his);
  const uint32_t mb[2] = {smem_u32(&c.sh->bars[0]), smem_u32(&c.sh->bars[1])};
  const uint32_t rb[2] = {smem_u32(&c.sh->ready[0]), smem_u32(&c.sh->ready[1])};
  const int q = warp & 3, cq = warp >> 2;  // TMEM lane quadrant, 64-column slice
  const uint32_t t_lane = c.tmem + ((uint32_t)(32 * q) << 16);
  int acc[64];

  for (int i = tid; i < ZB * 128 / 16; i += THREADS)
    reinterpret_cast<uint4 *>(sm + Ly.z)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (S > 1)  // no columns before the first one
    for (int i = tid; i < (S - 1) * 128; i += THREADS) Cs[32 * 128 + i] = 0u;
  fill_x<XC, KB>(sm + Ly.xs, x, nx, Ly.ptot);
  if (tid == 0) { c.sh->carry_hi = 0; c.sh->carry = 0; c.sh->borrow = 0; }
  fence_async_smem();
  __syncthreads();

  int L0 = -1;  // first limb kept (that of the first computed tile, or limb lo's column)
  // band mode: tiles anchored at the column of limb lo rather than at 0, so
  // that the columns below it (a whole tile of them, or most of one) are
  // not computed (with narrow blocks from S - 1 columns before it, whose
  // rows hold parts of its coefficients)
  const int cfirst = lo > 0 ? (lo / R - (S - 1) > 0 ? lo / R - (S - 1) : 0) : 0;
  for (int c0 = cfirst; R * c0 < nout; c0 += NT) {
    int W = Ly.ctot - c0;
    if (W > NT) W = NT;
    const int need = (nout - R * c0 + R - 1) / R;  // columns holding limbs < nout
    if (W > need) W = need;
    W = (W + 15) & ~15;
    if (R * (c0 + W) <= lo) continue;  // band: the whole tile lies below limb lo
    if (SPLIT && c0 != NT * tile) continue;
    if (L0 < 0) {
      L0 = lo > 0 ? R * (lo / R) : R * c0;
      if (lo > 0 && tid == 0) c.sh->carry_hi = 1ull << 32;  // + 2^32 B^L0
    }
    // blocks e whose columns [S e, S e + mx) meet the tile's [c0, c0 + W)
    const int e_lo = c0 - Ly.mx + 1 > 0 ? (c0 - Ly.mx + S) / S : 0;
    const int e_hi = (c0 + W - 1) / S < Ly.ey ? (c0 + W - 1) / S : Ly.ey;
    const int NG = e_hi >= e_lo ? (e_hi - e_lo + G) / G : 0;
#pragma unroll
    for (int i = 0; i < 64; i++) acc[i] = 0;
    if (NG > 0) {
      if (worker)
        hank_build<G, DRAIN, KB>(
            sm + Ly.h0, sm + Ly.st,
            hank_load<G, KB>(y, ny, e_lo + G - 1 < e_hi ? e_lo + G - 1 : e_hi, tid), tid);
      fence_async_smem();
      __syncthreads();
      bool bad = false;
      auto last_block = [&](int gi) {
        return e_lo + gi * G + G - 1 < e_hi ? e_lo + gi * G + G - 1 : e_hi;
      };
      if (issuer) {
        // group gi into accumulator and Hankel buffer gi & 1, as soon as the
        // drain warps report that buffer built and that accumulator drained
        // (from the second group on): no block barrier between groups, so
        // the tensor core's queue is refilled while it still holds work
        for (int gi = 0; gi < NG; gi++) {
          const int b = gi & 1;
          if (gi >= 1) {
            if (!mbar_wait_lim(rb[b], (c.rphase >> b) & 1u, c.wlim)) { bad = true; break; }
            c.rphase ^= 1u << b;
          }
          if (gi >= 2) {  // drained: group gi - 2 has completed
            c.phase ^= 1u << b;
            c.pending &= ~(1u << b);
          }
          issue_group<KB>(c.tmem + (uint32_t)(b * NT), b ? sbase + Ly.h1 : sbase + Ly.h0, xs_a,
                          z_a, lbo_b, c0, W, e_lo + gi * G, last_block(gi), Ly.mx, mb[b]);
          c.pending |= 1u << b;
        }
      } else if (worker) {
        for (int gi = 0; gi < NG; gi++) {
          const int ob = (gi & 1) ^ 1;
          const bool more = gi + 1 < NG;
          // the next group's y limbs are fetched before the wait
          HankLimbs hv{0ull, 0ull};
          if (more) hv = hank_load<G, KB>(y, ny, last_block(gi + 1), tid);
          if (gi >= 1 && !mbar_wait_lim(mb[ob], (c.phase >> ob) & 1u, c.wlim)) bad = true;
          // all drain threads agree; past this barrier every one of them has
          // finished the previous iteration (the Hankel staging run is free)
          if (bar_or_drain<DRAIN>(bad)) { bad = true; break; }
          if (gi >= 1) {  // group gi - 1 (accumulator ob): drain
            c.phase ^= 1u << ob;
            tc_fence_after();
            int slo, shi;
            group_span<KB>(c0, W, e_lo + (gi - 1) * G, last_block(gi - 1), Ly.mx, slo, shi);
            drain(t_lane + (uint32_t)(ob * NT), cq, slo, shi, acc);
          }
          if (more) {  // group gi + 1 into Hankel buffer ob, then report it
            hank_build<G, DRAIN, KB>(ob ? sm + Ly.h1 : sm + Ly.h0, sm + Ly.st, hv, tid);
            tc_fence_before();
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(rb[ob]);
          }
        }
        if (!bad) {
          const int lb = (NG - 1) & 1;
          if (!mbar_wait_lim(mb[lb], (c.phase >> lb) & 1u, c.wlim)) {
            bad = true;
          } else {
            c.phase ^= 1u << lb;
            tc_fence_after();
            int slo, shi;
            group_span<KB>(c0, W, e_lo + (NG - 1) * G, e_hi, Ly.mx, slo, shi);
            drain(t_lane + (uint32_t)(lb * NT), cq, slo, shi, acc);
          }
        }
      }
      tc_fence_before();
      // an abort leaves the issuing thread's pending bits for tc_release
      if (__syncthreads_or(bad)) { c.aborted = true; return false; }
      tc_fence_after();
      if (issuer) {  // the last one or two groups have completed (drained above)
        for (int gi = NG >= 2 ? NG - 2 : 0; gi < NG; gi++) {
          c.phase ^= 1u << (gi & 1);
          c.pending &= ~(1u << (gi & 1));
        }
      }
    }

    // ---- column sums -> limbs of this tile (low words to out, high words to His)
    // Cs: columns 0..31 of the current run of 32, then at 32 .. 32 + S - 2
    // the S - 1 columns before it (virtual columns -(S - 1) .. -1)
    const int j0 = R * c0;
    const int nl = R * W < nout - j0 ? R * W : nout - j0;
    const int skip = L0 > j0 ? L0 - j0 : 0;  // band: limbs below L0 are not kept
#pragma unroll
    for (int rr = 0; rr < NT / 32; rr++) {
      if (32 * rr < W) {
        if (cq == (rr >> 1)) {
          const int t = 127 - (32 * q + lane);
#pragma unroll
          for (int i = 0; i < 32; i++) Cs[i * 128 + t] = (uint32_t)acc[(rr & 1) * 32 + i];
        }
        __syncthreads();
        for (int idx = tid; idx < 32 * R; idx += THREADS) {  // 32 columns x R limbs
          const int col = idx / R, jj = idx % R;
          const int lt = (32 * rr + col) * R + jj;
          if (lt < nl && lt >= skip) {
            uint32_t cw[8];
#pragma unroll
            for (int a = 0; a < S; a++) {  // row 8 jj + KB a of column col - a
              const int v = col - a, slot = v >= 0 ? v : 32 + S - 1 + v;
              const uint4 u0 = *reinterpret_cast<const uint4 *>(&Cs[slot * 128 + 8 * jj + KB * a]);
              const uint4 u1 =
                  *reinterpret_cast<const uint4 *>(&Cs[slot * 128 + 8 * jj + KB * a + 4]);
              const uint32_t w[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
              for (int k = 0; k < 8; k++) cw[k] = a == 0 ? w[k] : cw[k] + w[k];
            }
            unsigned __int128 V = 0;
#pragma unroll
            for (int k = 0; k < 8; k++) V += (unsigned __int128)(cw[k] ^ 0x80000000u) << (8 * k);
            out[j0 + lt] = (uint64_t)V;
            His[lt] = (uint32_t)(V >> 64);
          }
        }
        __syncthreads();
        if (S > 1) {  // the last S - 1 columns of this run precede the next one
          for (int i = tid; i < (S - 1) * 128; i += THREADS)
            Cs[32 * 128 + i] = Cs[(33 - S) * 128 + i];
          __syncthreads();
        }
      }
    }
    {
      // band mode's first tile: the kept limbs start at L0 (skip > 0), with
      // the margin (carry_hi = 2^32) in place of what limb L0 - 1 would carry
      const uint64_t hprev = c.sh->carry_hi;
      const uint32_t cprev = c.sh->carry;
      uint64_t *o = out + j0 + skip;
      auto load = [&](int j) {
        return make_ulonglong2(o[j], j == 0 ? hprev : (uint64_t)His[skip + j - 1]);
      };
      auto store = [&](int j, uint64_t v) { o[j] = v; };
      if (SPLIT) {
        const uint32_t cout = blk_addsub<false>(nl, cprev, load, store, c.scr);
        if (tid == 0) {
          tile_carry[0] = His[nl - 1];
          tile_carry[1] = cout;
        }
      } else {
        // with the bias sum 2^31 sum_s 2^(8 s) of the column sums subtracted
        // in the same pass (0x8080808080808080 per limb from L0 on,
        // 0x8080808080000000 in limb L0); the carry and the borrow run on
        // into the next tile
        uint32_t cc = cprev, bb = c.sh->borrow;
        auto bias = [&](int j) {
          return j0 + skip + j == L0 ? 0x8080808080000000ull : 0x8080808080808080ull;
        };
        blk_add_then_sub(nl - skip, &cc, &bb, load, bias, store, c.scr);
        if (tid == 0) {
          c.sh->carry_hi = His[nl - 1];
          c.sh->carry = cc;
          c.sh->borrow = bb;
        }
      }
      __syncthreads();
    }
  }
  if (!SPLIT && L0 >= 0) {
    // without x's carry digit the digits spelled x_s = x - t_x B^nx:
    // x y = x_s y + t_x y B^nx.  In band mode the part of the correction
    // below L0 is dropped (its carry into L0 is within the band's margin).
    const uint32_t tx = XC ? 0u : (uint32_t)(x[nx - 1] >> 63);
    auto add_shifted = [&](int off, const uint64_t *src, int nsrc) {
      const int st = off > L0 ? off : L0;
      if (st >= nout) return;
      uint64_t *oo = out + st;
      auto ld = [&](int j) {
        const int k = st + j - off;
        return make_ulonglong2(oo[j], k < nsrc ? src[k] : 0ull);
      };
      auto sto = [&](int j, uint64_t v) { oo[j] = v; };
      blk_addsub<false>(nout - st, 0u, ld, sto, c.scr);
    };
    if (tx) add_shifted(nx, y, ny);
  }
  __syncthreads();
  return true;
}

// ---- partial tiles (split-K) ---------------------------------------------
// Groups [g0, g1) of tile `tile` of x * y (x with its carry digit, tiles of
// NT columns from column cfirst), added into colsum: for each of the tile's
// columns c (relative to the tile) and positions t, the int32 partial sum of
// the coefficient 128 (c0 + c) + t is added to colsum[c * 128 + t] with an
// atomic add (exact and order-independent: a coefficient's full sum is below
// 2^31 in magnitude, so every partial sum is too).  The CTAs of one product
// thus share its tiles' Toeplitz blocks, and tc_colsum_limbs turns the sums
// into limbs.  Returns false (and sets c.aborted) if a wait hit its limit.
template <int NT, int G>
__device__ bool tc_partial(TcCtx &c, const uint64_t *x, int nx, const uint64_t *y, int ny,
                           int c0, int W, int g0, int g1, int *colsum) {
  constexpr int DRAIN = 2 * NT, THREADS = DRAIN + 32;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool issuer = tid == DRAIN, worker = tid < DRAIN;
  const Layout Ly = layout<NT, G, true>(nx, ny);
  uint8_t *sm = c.sm;
  const uint32_t sbase = c.sbase;
  const uint32_t xs_a = sbase + Ly.xs, z_a = sbase + Ly.z;
  const uint32_t lbo_b = (uint32_t)Ly.ptot * 16u;
  const uint32_t mb[2] = {smem_u32(&c.sh->bars[0]), smem_u32(&c.sh->bars[1])};
  const int q = warp & 3, cq = warp >> 2;
  const uint32_t t_lane = c.tmem + ((uint32_t)(32 * q) << 16);
  const int e_lo = c0 - Ly.mx + 1 > 0 ? c0 - Ly.mx + 1 : 0;
  const int e_hi = c0 + W - 1 < Ly.ey ? c0 + W - 1 : Ly.ey;
  const int NG = e_hi >= e_lo ? (e_hi - e_lo + G) / G : 0;
  if (g1 > NG) g1 = NG;
  if (g0 >= g1) return true;
  const int ng = g1 - g0;
  int acc[64];
#pragma unroll
  for (int i = 0; i < 64; i++) acc[i] = 0;

  for (int i = tid; i < ZB * 128 / 16; i += THREADS)
    reinterpret_cast<uint4 *>(sm + Ly.z)[i] = make_uint4(0u, 0u, 0u, 0u);
  fill_x<true>(sm + Ly.xs, x, nx, Ly.ptot);
  auto last_block = [&](int gi) { return e_lo + gi * G + G - 1 < e_hi ? e_lo + gi * G + G - 1 : e_hi; };
  if (worker) hank_build<G, DRAIN>(sm + Ly.h0, sm + Ly.st, hank_load<G>(y, ny, last_block(g0), tid), tid);
  fence_async_smem();
  __syncthreads();
  bool bad = false;
  for (int k = 0; k < ng; k++) {
    const int gi = g0 + k, b = k & 1;
    const int ea = e_lo + gi * G, eb = last_block(gi);
    if (issuer)
      issue_group(c.tmem + (uint32_t)(b * NT), b ? sbase + Ly.h1 : sbase + Ly.h0, xs_a, z_a,
                  lbo_b, c0, W, ea, eb, Ly.mx, mb[b]);
    c.pending |= 1u << b;
    const bool more = k + 1 < ng && worker;
    HankLimbs hv{0ull, 0ull};
    if (more) hv = hank_load<G>(y, ny, last_block(gi + 1), tid);
    if (k >= 1) {
      const int ob = b ^ 1;
      if (worker && !mbar_wait_lim(mb[ob], (c.phase >> ob) & 1u, c.wlim)) {
        bad = true;
      } else {
        c.phase ^= 1u << ob;
        c.pending &= ~(1u << ob);
      }
      tc_fence_after();
      int slo, shi;
      group_span(c0, W, ea - G, ea - 1, Ly.mx, slo, shi);
      if (worker) drain(t_lane + (uint32_t)(ob * NT), cq, slo, shi, acc);
    }
    if (more) hank_build<G, DRAIN>(b ? sm + Ly.h0 : sm + Ly.h1, sm + Ly.st, hv, tid);
    tc_fence_before();
    fence_async_smem();
    if (__syncthreads_or(bad)) { c.aborted = true; return false; }
  }
  const int lb = (ng - 1) & 1;
  if (!mbar_wait_lim(mb[lb], (c.phase >> lb) & 1u, c.wlim)) {
    bad = true;
  } else {
    c.phase ^= 1u << lb;
    c.pending &= ~(1u << lb);
  }
  tc_fence_after();
  {
    int slo, shi;
    group_span(c0, W, e_lo + (g1 - 1) * G, last_block(g1 - 1), Ly.mx, slo, shi);
    if (worker) drain(t_lane + (uint32_t)(lb * NT), cq, slo, shi, acc);
  }
  tc_fence_before();
  if (__syncthreads_or(bad)) { c.aborted = true; return false; }
  if (worker) {
    const int t = 127 - (32 * q + lane);
#pragma unroll
    for (int i = 0; i < 64; i++) {
      const int col = 64 * cq + i;
      if (col < W && acc[i] != 0) atomicAdd(&colsum[col * 128 + t], acc[i]);
    }
  }
  __syncthreads();  // the shared memory (x, Hankel buffers) is reused by the next unit
  return true;
}

// out[L0 .. nout) of the product whose column sums (coefficients 128 c + t
// for the columns c from cfirst = L0 / 16 on) are in colsum[(c - cfirst) *
// 128 + t], by the whole CTA: limb j is V_j = sum_k (coef(8 j + k) + 2^31)
// 2^(8 k), i.e. its low word plus the high word of V_(j-1) (plus `margin` at
// L0), less the bias sum of the column sums (0x8080808080000000 at L0,
// 0x8080808080808080 above); one carry scan then one borrow scan
// (blk_add_then_sub), as at the end of each of tc_product's tiles.
__device__ inline void tc_colsum_limbs(const int *colsum, int L0, int nout, uint64_t margin,
                                uint64_t *out, uint32_t *scr) {
  auto V = [&](int j) {
    const int *cs = colsum + (size_t)(j - L0) * 8;  // 16 limbs per 128-position column
    unsigned __int128 v = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) v += (unsigned __int128)((uint32_t)cs[k] ^ 0x80000000u) << (8 * k);
    return v;
  };
  auto load = [&](int jj) {
    const int j = L0 + jj;
    const uint64_t hi = jj == 0 ? margin : (uint64_t)(V(j - 1) >> 64);
    return make_ulonglong2((uint64_t)V(j), hi);
  };
  auto bias = [&](int jj) { return jj == 0 ? 0x8080808080000000ull : 0x8080808080808080ull; };
  auto store = [&](int jj, uint64_t v) { out[L0 + jj] = v; };
  uint32_t cc = 0, bb = 0;
  blk_add_then_sub(nout - L0, &cc, &bb, load, bias, store, scr);
}

// ---- host side, per translation unit ---------------------------------------
// BIGINT_ETIMEOUT if a product launched from this translation unit gave up
// at a wait limit since the last call (synchronises the device; clears the
// record), else BIGINT_OK.
static inline int take_timeout_here() {
  if (cudaDeviceSynchronize() != cudaSuccess) return BIGINT_ECUDA;
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_timeout, sizeof(int)) != cudaSuccess) return BIGINT_ECUDA;
  if (v) {
    const int zero = 0;
    if (cudaMemcpyToSymbol(g_timeout, &zero, sizeof(int)) != cudaSuccess) return BIGINT_ECUDA;
    return BIGINT_ETIMEOUT;
  }
  return BIGINT_OK;
}

// Sets the wait limit of the products launched from this translation unit
// from now on (synchronous): cycles > 0 the limit, 0 the default WAIT_LIMIT,
// cycles < 0 the injected timeout of g_never_set after -cycles cycles.
static inline int set_wait_limit_here(long long cycles) {
  const long long v = cycles != 0 ? cycles : WAIT_LIMIT;
  if (cudaDeviceSynchronize() != cudaSuccess) return BIGINT_ECUDA;
  return cudaMemcpyToSymbol(g_wait_limit, &v, sizeof(v)) == cudaSuccess ? BIGINT_OK
                                                                        : BIGINT_ECUDA;
}

}  // namespace tcm
}  // namespace bigint
