// kara.cu -- full products of square operands by Karatsuba's method over the
// batched products of mul.cu / tcmul.cu (sub-quadratic multiplication, the
// next step the paper names; exact integer arithmetic throughout).
//
// With n = 2k, x = x1 B^k + x0 and y = y1 B^k + y0:
//   x y = z2 B^(2k) + (z0 + z2 + (x0 - x1)(y1 - y0)) B^k + z0,
//   z0 = x0 y0,  z2 = x1 y1,
// the subtractive form, whose middle product |x0 - x1| |y1 - y0| has k-limb
// operands (no carry limb).  Every step runs for the whole batch at once:
// one launch forms |x0 - x1|, |y1 - y0| and the sign of their product, the
// three k-limb products are batched launches (strided views of the
// operands; z0 and z2 written straight into the two halves of the result)
// or, with levels left, the same method one level down, and one launch adds
// the middle term into the result.  Three products of n/2 limbs do 3/4 of
// the digit products of one of n limbs; measured on GB300 the tensor-core
// product of 2048 limbs is about as efficient per digit product as that of
// 4096 and 8192 limbs, so one level pays at 4096 limbs and two at 8192.
#include "blockops.cuh"

namespace bigint {

int launch_mul_ex(const uint64_t *a, int64_t sa, const uint64_t *b, int64_t sb, uint64_t *out,
                  int64_t so, int64_t count, int na, int nb, int nout, int lo, int *abort_flag,
                  cudaStream_t st, int tc_min, void *sk_ws, size_t sk_bytes);
int launch_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na,
               int nb, int nout, cudaStream_t st);

namespace kara {

constexpr int PRE_THREADS = 512, POST_THREADS = 1024;
// Shorter operand (limbs) from which the leaf products run on the tensor
// cores, as for bigint_mul.
constexpr int TC_LEAF_MIN = 256;

// One CTA per instance: da = |x0 - x1|, db = |y1 - y0| (k limbs each) and
// neg = 1 if (x0 - x1)(y1 - y0) < 0.
__global__ void __launch_bounds__(PRE_THREADS)
    k_kara_pre(const uint64_t *__restrict__ X, int64_t sx, const uint64_t *__restrict__ Y,
               int64_t sy, int k, uint64_t *__restrict__ DA, uint64_t *__restrict__ DB,
               int64_t sd, int8_t *__restrict__ neg) {
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  const int64_t i = blockIdx.x;
  const uint64_t *x = X + i * sx, *y = Y + i * sy;
  uint64_t *da = DA + i * sd, *db = DB + i * sd;
  const int cx = blk_cmp(x, x + k, k, scr);  // sign of x0 - x1
  const uint64_t *xa = cx >= 0 ? x : x + k, *xb = cx >= 0 ? x + k : x;
  blk_addsub<true>(k, 0u, [&](int j) { return make_ulonglong2(xa[j], xb[j]); },
                   [&](int j, uint64_t v) { da[j] = v; }, scr);
  const int cy = blk_cmp(y + k, y, k, scr);  // sign of y1 - y0
  const uint64_t *ya = cy >= 0 ? y + k : y, *yb = cy >= 0 ? y : y + k;
  blk_addsub<true>(k, 0u, [&](int j) { return make_ulonglong2(ya[j], yb[j]); },
                   [&](int j, uint64_t v) { db[j] = v; }, scr);
  if (threadIdx.x == 0) neg[i] = (int8_t)(cx * cy < 0);
}

// One CTA per instance: out holds z0 in limbs [0, 2k) and z2 in [2k, 4k);
// z1 = |x0 - x1| |y1 - y0| (2k limbs).  mid = z0 + z2 -+ z1 (2k + 1 limbs,
// in shared memory; nonnegative, it is x0 y1 + x1 y0), then
// out[k, 4k) += mid.
__global__ void __launch_bounds__(POST_THREADS)
    k_kara_post(uint64_t *__restrict__ Out, int64_t so, const uint64_t *__restrict__ Z1,
                int64_t sz, const int8_t *__restrict__ neg, int k) {
  extern __shared__ uint64_t mid[];
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  const int64_t i = blockIdx.x;
  uint64_t *o = Out + i * so;
  const uint64_t *z1 = Z1 + i * sz;
  const uint32_t c = blk_addsub<false>(
      2 * k, 0u, [&](int j) { return make_ulonglong2(o[j], o[2 * k + j]); },
      [&](int j, uint64_t v) { mid[j] = v; }, scr);
  uint64_t top = c;
  if (neg[i]) {
    const uint32_t b = blk_addsub<true>(
        2 * k, 0u, [&](int j) { return make_ulonglong2(mid[j], z1[j]); },
        [&](int j, uint64_t v) { mid[j] = v; }, scr);
    top -= b;
  } else {
    const uint32_t cc = blk_addsub<false>(
        2 * k, 0u, [&](int j) { return make_ulonglong2(mid[j], z1[j]); },
        [&](int j, uint64_t v) { mid[j] = v; }, scr);
    top += cc;
  }
  if (threadIdx.x == 0) mid[2 * k] = top;
  __syncthreads();
  blk_addsub<false>(
      3 * k, 0u,
      [&](int j) { return make_ulonglong2(o[k + j], j <= 2 * k ? mid[j] : 0ull); },
      [&](int j, uint64_t v) { o[k + j] = v; }, scr);
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Workspace bytes of `count` instances for `levels` levels on n-limb
// operands: per level |x0 - x1| and |y1 - y0| (k limbs each), z1 (2k limbs)
// and the signs, then the next level's (reused by its three products one
// after the other).
size_t chunk_bytes(int64_t count, int n, int levels) {
  if (levels <= 0) return 0;
  const int k = n / 2;
  return 2 * align256(8 * (size_t)count * k) + align256(8 * (size_t)count * 2 * k) +
         align256((size_t)count) + chunk_bytes(count, k, levels - 1);
}

int post_smem_ok(int k) {
  static int optin = -1;
  if (optin < 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      return 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, k_kara_post) != cudaSuccess) return 0;
    optin = v - (int)fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(k_kara_post, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) !=
        cudaSuccess)
      return 0;
  }
  return (size_t)8 * (2 * k + 1) <= (size_t)optin;
}

int run(const uint64_t *x, int64_t sx, const uint64_t *y, int64_t sy, uint64_t *out, int64_t so,
        int64_t count, int n, int levels, char *ws, cudaStream_t st) {
  if (levels <= 0)
    return launch_mul_ex(x, sx, y, sy, out, so, count, n, n, 2 * n, 0, nullptr, st, TC_LEAF_MIN,
                         nullptr, 0);
  const int k = n / 2;
  uint64_t *DA = reinterpret_cast<uint64_t *>(ws);
  char *p = ws + align256(8 * (size_t)count * k);
  uint64_t *DB = reinterpret_cast<uint64_t *>(p);
  p += align256(8 * (size_t)count * k);
  uint64_t *Z1 = reinterpret_cast<uint64_t *>(p);
  p += align256(8 * (size_t)count * 2 * k);
  int8_t *neg = reinterpret_cast<int8_t *>(p);
  p += align256((size_t)count);
  k_kara_pre<<<(unsigned)count, PRE_THREADS, 0, st>>>(x, sx, y, sy, k, DA, DB, k, neg);
  int rc = bigint_launch_status();
  if (rc != BIGINT_OK) return rc;
  if ((rc = run(x, sx, y, sy, out, so, count, k, levels - 1, p, st)) != BIGINT_OK) return rc;
  if ((rc = run(x + k, sx, y + k, sy, out + 2 * k, so, count, k, levels - 1, p, st)) != BIGINT_OK)
    return rc;
  if ((rc = run(DA, k, DB, k, Z1, 2 * k, count, k, levels - 1, p, st)) != BIGINT_OK) return rc;
  k_kara_post<<<(unsigned)count, POST_THREADS, 8 * (size_t)(2 * k + 1), st>>>(out, so, Z1, 2 * k,
                                                                             neg, k);
  return bigint_launch_status();
}

}  // namespace kara

// Levels of Karatsuba for square n-limb products (levels < 0: by size, as
// measured on GB300: two from 8192 limbs, one from 4096, none below).
int kara_levels(int n, int levels) {
  if (levels < 0) levels = n >= 8192 ? 2 : (n >= 4096 ? 1 : 0);
  while (levels > 0 && (n % (1 << levels) != 0)) levels--;  // each level halves exactly
  return levels;
}

bool kara_valid(int n, int levels) {
  if (n < 1 || n > BIGINT_MUL_MAX_LIMBS || levels > 3) return false;
  const int L = kara_levels(n, levels);
  for (int l = 1; l <= L; l++)
    if (!kara::post_smem_ok((n >> l))) return false;
  return true;
}

size_t mul_kara_workspace(int64_t count, int n, int levels) {
  if (count < 0 || !kara_valid(n, levels)) return 0;
  return kara::chunk_bytes(count, n, kara_levels(n, levels));
}

// Batches whose workspace would exceed `bytes` run in chunks of as many
// instances as fit (at least one).
int launch_mul_kara(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int n,
                    int levels, void *ws, size_t bytes, cudaStream_t st) {
  if (count < 0 || !kara_valid(n, levels)) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  const int L = kara_levels(n, levels);
  if (L == 0) return launch_mul(a, b, out, count, n, n, 2 * n, st);  // bigint_mul's own choice
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) % 256) != 0) return BIGINT_EINVAL;
  int64_t chunk = count;
  while (chunk > 1 && kara::chunk_bytes(chunk, n, L) > bytes) chunk = (chunk + 1) / 2;
  if (kara::chunk_bytes(chunk, n, L) > bytes) return BIGINT_ENOMEM;
  for (int64_t i0 = 0; i0 < count; i0 += chunk) {
    const int64_t c = count - i0 < chunk ? count - i0 : chunk;
    const int rc = kara::run(a + i0 * n, n, b + i0 * n, n, out + i0 * 2 * n, 2 * n, c, n, L,
                             static_cast<char *>(ws), st);
    if (rc != BIGINT_OK) return rc;
  }
  return BIGINT_OK;
}

}  // namespace bigint
