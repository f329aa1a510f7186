// mul.cu -- batched multiplication kernels (Sec. V-B, Fig. 5).
//
// One CTA per instance; the whole product is computed by blk_mul
// (mulcore.cuh) with both operands resident in shared memory.  The digit
// size RB, the chunk width Q and the flush interval F are compile-time; a
// few variants are instantiated and one is chosen per call (the default, or
// the one the tuning hook selected).
#include "mulcore.cuh"

namespace bigint {

// Instance i: a at A + i sa, b at Bm + i sb, result at Out + i so (limbs).
template <int RB, int Q, int F>
__global__ void __launch_bounds__(Q >= 16 ? 640 : 1024)
    k_mul(const uint64_t *__restrict__ A, const uint64_t *__restrict__ Bm,
          uint64_t *__restrict__ Out, int na, int nb, int nout, int64_t sa, int64_t sb,
          int64_t so) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int64_t inst = blockIdx.x;
  blk_mul<RB, Q, F>(A + inst * sa, na, Bm + inst * sb, nb, Out + inst * so, nout, smem);
}

// ---- small products, one warp each -------------------------------------------
// Products whose operands have at most SMALL_LIMBS limbs, thousands at a
// time: a CTA per instance (blk_mul) spends most of such a launch on its
// fixed costs, so here one warp takes an instance and runs warp_mul
// (blockops.cuh: whole schoolbook columns per lane, then the carry scan).
// Exact low nout limbs (nout <= na + nb).
constexpr int SMALL_LIMBS = 64, SMALL_WARPS = 8;

__global__ void __launch_bounds__(32 * SMALL_WARPS)
    k_mul_small(const uint64_t *__restrict__ A, const uint64_t *__restrict__ Bm,
                uint64_t *__restrict__ Out, int na, int nb, int nout, int64_t count, int64_t sa,
                int64_t sb, int64_t so) {
  __shared__ uint64_t xs[SMALL_WARPS][SMALL_LIMBS], ys[SMALL_WARPS][SMALL_LIMBS];
  __shared__ uint64_t os[SMALL_WARPS][2 * SMALL_LIMBS], cs[SMALL_WARPS][6 * SMALL_LIMBS];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t inst = (int64_t)blockIdx.x * SMALL_WARPS + w;
  if (inst >= count) return;  // the whole warp: no block barrier below
  const uint64_t *a = A + inst * sa, *b = Bm + inst * sb;
  for (int i = lane; i < na; i += 32) xs[w][i] = a[i];
  for (int i = lane; i < nb; i += 32) ys[w][i] = b[i];
  __syncwarp();
  warp_mul(xs[w], na, ys[w], nb, os[w], nout, cs[w]);
  uint64_t *o = Out + inst * so;
  for (int j = lane; j < nout; j += 32) o[j] = os[w][j];
}

static int launch_mul_small(const uint64_t *a, int64_t sa, const uint64_t *b, int64_t sb,
                            uint64_t *out, int64_t so, int64_t count, int na, int nb, int nout,
                            cudaStream_t st) {
  if (na > SMALL_LIMBS || nb > SMALL_LIMBS || nout > na + nb) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  const int64_t blocks = (count + SMALL_WARPS - 1) / SMALL_WARPS;
  k_mul_small<<<(unsigned)blocks, 32 * SMALL_WARPS, 0, st>>>(a, b, out, na, nb, nout, count, sa,
                                                             sb, so);
  return bigint_launch_status();
}

template <int RB, int Q, int F>
__global__ void __launch_bounds__(Q >= 16 ? 640 : 1024)
    k_mul_kara(const uint64_t *__restrict__ A, const uint64_t *__restrict__ Bm,
               uint64_t *__restrict__ Out, int n) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int64_t inst = blockIdx.x;
  blk_mul_kara<RB, Q, F>(A + inst * (int64_t)n, Bm + inst * (int64_t)n, n,
                         Out + inst * (int64_t)(2 * n), smem);
}

// Threads per CTA for a product with `units` units of work: as few rounds as
// the 1024-thread limit allows, then the smallest multiple of 32 that covers
// the units in that many rounds.
static int pick_threads(int units, int max_threads) {
  int rounds = (units + max_threads - 1) / max_threads;
  if (rounds < 1) rounds = 1;
  int T = (units + rounds - 1) / rounds;
  T = (T + 31) / 32 * 32;
  return T < 32 ? 32 : T;
}

static int g_smem_optin = 0;

static int smem_optin() {
  if (g_smem_optin == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&g_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
      return 0;
  }
  return g_smem_optin;
}

template <int RB, int Q, int F>
static int launch_variant(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count,
                          int na, int nb, int nout, cudaStream_t st, int64_t sa = -1,
                          int64_t sb = -1, int64_t so = -1) {
  const size_t smem = sizeof(uint32_t) * (size_t)blk_mul_smem_words<RB, Q>(na, nb);
  const int optin = smem_optin();
  if (optin == 0) return BIGINT_ECUDA;
  if (smem > (size_t)optin) return BIGINT_EINVAL;
  static int dyn_max = -1;  // opt-in limit minus the kernel's static shared memory
  if (dyn_max < 0) {
    cudaFuncAttributes fa;
    BIGINT_CUDA_TRY(cudaFuncGetAttributes(&fa, k_mul<RB, Q, F>));
    BIGINT_CUDA_TRY(cudaFuncSetAttribute(k_mul<RB, Q, F>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         optin - (int)fa.sharedSizeBytes));
    dyn_max = optin - (int)fa.sharedSizeBytes;
  }
  if (smem > (size_t)dyn_max) return BIGINT_EINVAL;
  const int T = pick_threads(blk_mul_units<RB, Q>(na, nb), Q >= 16 ? 640 : 1024);
  k_mul<RB, Q, F><<<(unsigned)count, T, smem, st>>>(
      a, b, out, na, nb, nout, sa < 0 ? na : sa, sb < 0 ? nb : sb, so < 0 ? nout : so);
  return bigint_launch_status();
}

template <int RB, int Q, int F>
static int launch_kara(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int n,
                       cudaStream_t st) {
  const size_t smem = sizeof(uint32_t) * (size_t)blk_kara_smem_words<RB, Q>(n);
  const int optin = smem_optin();
  if (optin == 0) return BIGINT_ECUDA;
  if (smem > (size_t)optin) return BIGINT_EINVAL;
  static int dyn_max = -1;  // opt-in limit minus the kernel's static shared memory
  if (dyn_max < 0) {
    cudaFuncAttributes fa;
    BIGINT_CUDA_TRY(cudaFuncGetAttributes(&fa, k_mul_kara<RB, Q, F>));
    BIGINT_CUDA_TRY(cudaFuncSetAttribute(k_mul_kara<RB, Q, F>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         optin - (int)fa.sharedSizeBytes));
    dyn_max = optin - (int)fa.sharedSizeBytes;
  }
  if (smem > (size_t)dyn_max) return BIGINT_EINVAL;
  const int T = pick_threads(blk_kara_units<RB, Q>(n), Q >= 16 ? 640 : 1024);
  k_mul_kara<RB, Q, F><<<(unsigned)count, T, smem, st>>>(a, b, out, n);
  return bigint_launch_status();
}

// Variant table (see bigint_set_variant).  Variant 0 picks by size from
// measurements on GB300 (full-product sweep, 2^32-bit operand arrays): the
// tensor-core product (tcmul.cu) once the shorter operand has TC_MIN_LIMBS
// limbs and fits shared memory; below, the integer product with 28-bit
// digits and 8-column chunks (variant 9), or 29-bit digits and 16-column
// chunks (variant 8) past 1535 limbs.  A size class the tuner has measured
// (bigint_tune) takes its recorded variant instead.
size_t mul_tc_smem(int na, int nb);
int launch_mul_tc(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na,
                  int nb, int nout, cudaStream_t st, int force_nt);

// Shorter operand (limbs) from which the default is the tensor-core product.
constexpr int TC_MIN_LIMBS = 256;

static int g_mul_variant = 0;
// Tuned variant per size class (class c: operands of [2^c, 2^(c+1)) limbs),
// 0 = not tuned (built-in choice).  Written by bigint_tune / bigint_tune_mul
// and bigint_tuning_load.
int g_mul_tuned[32] = {};

int mul_size_class(int na, int nb) {
  const int n = na > nb ? na : nb;
  int c = 0;
  while ((2 << c) <= n) c++;
  return c;
}

bool mul_variant_valid(int v) {
  return v == 0 || (v >= 8 && v <= 17);
}

int mul_set_variant(int v) {
  if (!mul_variant_valid(v)) return BIGINT_EINVAL;
  g_mul_variant = v;
  return BIGINT_OK;
}

// Largest square operand (limbs) whose product fits one CTA's shared memory.
int mul_max_limbs() { return BIGINT_MUL_MAX_LIMBS; }

// The variant a call with these shapes runs (after defaults and fallbacks).
int mul_variant_for(int na, int nb, int nout) {
  int v = g_mul_variant;
  if (v == 0) v = g_mul_tuned[mul_size_class(na, nb)];
  if (v == 0) {
    const int nmax = na > nb ? na : nb, nmin = na < nb ? na : nb;
    if (nmin >= TC_MIN_LIMBS && mul_tc_smem(na, nb) > 0)
      v = 12;
    else
      v = nmax < 1536 ? 9 : 8;
  }
  const bool square_full = na == nb && nout == na + nb && na >= 64;
  if (v == 10 && !square_full) v = 8;                // Karatsuba: square full products only
  if (v == 11 && (na > SMALL_LIMBS || nb > SMALL_LIMBS)) v = 9;  // warp per instance: small only
  if (v >= 12 && mul_tc_smem(na, nb) == 0) v = 8;    // tensor-core product: shared memory bound
  return v;
}

int launch_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na,
               int nb, int nout, cudaStream_t st) {
  const int v = mul_variant_for(na, nb, nout);
  switch (v) {
    case 12: return launch_mul_tc(a, b, out, count, na, nb, nout, st, 0);
    case 13: return launch_mul_tc(a, b, out, count, na, nb, nout, st, TC_FORCE_64);
    case 14: return launch_mul_tc(a, b, out, count, na, nb, nout, st, TC_FORCE_128);
    case 15: return launch_mul_tc(a, b, out, count, na, nb, nout, st, TC_FORCE_256);
    case 16: return launch_mul_tc(a, b, out, count, na, nb, nout, st, TC_FORCE_N64);
    case 17: return launch_mul_tc(a, b, out, count, na, nb, nout, st, TC_FORCE_N32);
    case 10: return launch_kara<29, 16, 32>(a, b, out, count, na, st);
    case 11: return launch_mul_small(a, na, b, nb, out, nout, count, na, nb, nout, st);
    case 9: return launch_variant<28, 8, 128>(a, b, out, count, na, nb, nout, st);
    default: return launch_variant<29, 16, 32>(a, b, out, count, na, nb, nout, st);
  }
}

int launch_mul_tc_ex(const uint64_t *a, int64_t sa, const uint64_t *b, int64_t sb, uint64_t *out,
                     int64_t so, int64_t count, int na, int nb, int nout, int lo, int *abort_flag,
                     cudaStream_t st, int force_nt);

size_t mul_sk_bytes_per_product(int na, int nb, int nout, int lo);
bool mul_sk_worth(int64_t count, int na, int nb, int nout, int lo);
int launch_mul_tc_sk(const uint64_t *a, int64_t sa, const uint64_t *b, int64_t sb, uint64_t *out,
                     int64_t so, int64_t count, int na, int nb, int nout, int lo, void *colsum,
                     size_t colsum_bytes, int *abort_flag, cudaStream_t st);

// The products inside divisions and programs: variant 0 or 12 runs the
// tensor-core product with its shape by the cost model (split-K for a few
// products), variants 13-17 force its shape as for launch_mul, and variants
// 8-10 keep them on the integer pipes.
int launch_mul_ex(const uint64_t *a, int64_t sa, const uint64_t *b, int64_t sb, uint64_t *out,
                  int64_t so, int64_t count, int na, int nb, int nout, int lo, int *abort_flag,
                  cudaStream_t st, int tc_min, void *sk_ws, size_t sk_bytes) {
  if (count == 0) return BIGINT_OK;
  const int nmin = na < nb ? na : nb;
  const int v = g_mul_variant;
  if (v == 0 || (v >= 12 && v <= 17)) {
    if (nmin >= tc_min && mul_tc_smem(na, nb) > 0) {
      // few products: cut each into units over the SMs (split-K)
      if (v <= 12 && sk_ws != nullptr && mul_sk_worth(count, na, nb, nout, lo) &&
          sk_bytes >= (size_t)count * mul_sk_bytes_per_product(na, nb, nout, lo))
        return launch_mul_tc_sk(a, sa, b, sb, out, so, count, na, nb, nout, lo, sk_ws, sk_bytes,
                                abort_flag, st);
      static const int force[6] = {0, TC_FORCE_64, TC_FORCE_128, TC_FORCE_256, TC_FORCE_N64,
                                   TC_FORCE_N32};
      return launch_mul_tc_ex(a, sa, b, sb, out, so, count, na, nb, nout, lo, abort_flag, st,
                              v <= 12 ? 0 : force[v - 12]);
    }
  }
  const int nmax = na > nb ? na : nb;
  if (nmax <= SMALL_LIMBS) return launch_mul_small(a, sa, b, sb, out, so, count, na, nb, nout, st);
  if (nmax < 1536) return launch_variant<28, 8, 128>(a, b, out, count, na, nb, nout, st, sa, sb, so);
  return launch_variant<29, 16, 32>(a, b, out, count, na, nb, nout, st, sa, sb, so);
}

}  // namespace bigint
