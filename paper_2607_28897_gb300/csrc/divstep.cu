// divstep.cu -- division of a uniform batch with every step batched across
// the instances (Sec. V-C, Fig. 6).
//
// The one-CTA-per-division kernel (divmod.cu) runs the whole algorithm of a
// division on one SM, as the paper's intragroup kernel does.  Its products
// are as fast as the SM allows, but the Newton loop is sequential: the early
// steps are tiny, every linear step waits at block barriers, and a batch
// smaller than a few waves of SMs leaves most of the GPU idle.  Here the
// division is instead cut at its steps, and each step runs for ALL instances
// of the batch at once: the products as batched launches of the multiply
// kernels (tensor-core products from 256 limbs: tcmul.cu, each filling every
// SM), the linear steps as one small kernel with one CTA per instance.  The
// arithmetic is that of divmod.cu; only the schedule differs.
//
// Every instance of a batch has the same shape (nu, nv), and for the usual
// operands (top limb of v nonzero, "regular") the same precision k = nv - 1
// and the exponent h = nu, so the Newton schedule (l, m, t per step) is
// known on the host.  Instances whose divisor has a zero top limb
// (including v = 0) take the one-CTA-per-division kernel in a last launch;
// the step kernels run over them too (their values are never used, and
// every size is fixed, so nothing reads out of bounds).
//
// Per step, with the iterate w ~ B^(k+l) / v kept to l + 2 limbs,
// m = min(l - 2, L - l), t = min(k, l + m + 2), vt = top t + 1 limbs of v:
//   P  = vt w mod B^(t+2)                    (low product, exact)
//   d  = B^(t+l) - vt w: |d| = P if P < B^(t+2)/2 (d <= 0), else B^(t+2) - P
//   P2 = w |d|, banded from limb s - 2, s = t + l - m
//   w' = w B^m + floor(P2 / B^s)             (d >= 0)
//   w' = w B^m - floor(P2 / B^s) - 1         (d <  0; the ceiling of Fig. 6
//                                             rounded up by at most one)
// The band makes floor(P2 / B^s) exact or one unit high; so each step lands
// within a few units of B^(k+l+m) / v, and since m <= l - 2 the Newton error
// squared stays below a unit: the error does not grow from step to step.
// Then q^ = floor(u w / B^h) (banded from limb h - 2), r^ = u - q^ v modulo
// B^(nv+1), and the exact correction of divmod.cu settles q and r.  The
// leading steps whose operands all have at most 136 limbs run in one
// launch, a warp per instance (k_ds_small), instead of four launches each.
#include <algorithm>

#include "divcore.cuh"

namespace bigint {

using namespace divc;

int launch_mul_ex(const uint64_t *a, int64_t sa, const uint64_t *b, int64_t sb, uint64_t *out,
                  int64_t so, int64_t count, int na, int nb, int nout, int lo, int *abort_flag,
                  cudaStream_t st, int tc_min, void *sk_ws, size_t sk_bytes);
int launch_divmod_cta(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                      int32_t *status, int64_t count, int nu, int nv, void *ws,
                      const int32_t *list, const int *nlist, cudaStream_t st);
size_t divmod_workspace(int64_t count, int nu, int nv);

namespace dstep {

constexpr int LIN_THREADS = 256;  // CTA of the linear per-instance kernels
// Shorter operand (limbs) from which a step's product runs on the tensor
// cores.  The steps' products are rectangular and come in batches of
// thousands; measured on 2n/n divisions at n = 512 the 132 x 262-limb and
// 68 x 134-limb products of the middle steps took 173 and 90 us on the
// integer pipes for 4096 instances.
constexpr int STEP_TC_MIN = 64;

// The step schedule needs k = prec(v) - 1 = nv - 1.  The dividend may have
// leading zero limbs: with h = nu (not prec(u)) w ~ B^h / v still bounds the
// quotient estimate u w / B^h within a few units of u / v since u < B^h,
// and the banded u w + B^h < B^(nu + nw) still holds, so such instances
// (the zero-padded operands of the batched form's division classes, or a
// short dividend) stay on the step path at the cost of the product work
// above their precision.
__device__ __forceinline__ bool regular(const uint64_t *, int, const uint64_t *v, int nv) {
  return v[nv - 1] != 0;
}

// One thread per instance: lists the irregular instances and writes the
// Newton start w = floor(B^(2 l) / V), V = floor(v / B^(k-l)) + 1, into the
// first l + 2 limbs of the instance's iterate record (zero for irregular
// ones, whose divisor may have a zero top limb).  (Running the first,
// tiny Newton steps in this kernel too, one CTA per instance, was measured
// slower than their batched launches: 579 us for 4096 instances of 512
// limbs, the long chains of block barriers of the one-CTA form again.)
__global__ void k_ds_start(const uint64_t *__restrict__ U, const uint64_t *__restrict__ V, int nu,
                           int nv, int l, uint64_t *W, int64_t sw, int64_t count,
                           int32_t *irregular, int *nirr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  const uint64_t *u = U + i * nu, *v = V + i * nv;
  uint64_t *w = W + i * sw;
  if (!regular(u, nu, v, nv)) {
    irregular[atomicAdd(nirr, 1)] = (int32_t)i;
    for (int j = 0; j < l + 2; j++) w[j] = 0;
    return;
  }
  const int k = nv - 1;
  uint64_t Vt[6] = {0, 0, 0, 0, 0, 0}, Un[8] = {0, 0, 0, 0, 0, 0, 0, 0}, Qt[8];
  for (int j = 0; j <= l; j++) Vt[j] = v[k - l + j];
  int j = 0;
  while (j <= l && ++Vt[j] == 0) j++;  // V + 1, which may carry into limb l + 1
  const int nV = j > l ? l + 2 : l + 1;
  if (j > l) Vt[l + 1] = 1;
  Un[2 * l] = 1;  // B^(2 l)
  small_div(Un, 2 * l + 1, Vt, nV, Qt);
  const int nq = 2 * l + 1 - nV + 1;
  for (int jj = 0; jj < l + 2; jj++) w[jj] = jj < nq ? Qt[jj] : 0;
}

constexpr int WARP_CTA = 256;  // warp-per-instance kernels: 8 instances per CTA

// ---------------------------------------------------------------------------
// The early Newton steps, while every operand of a step has at most
// SMALL_STEP_LIMBS limbs, in one launch with one warp per instance: each
// such step is four small launches otherwise (P, |d|, P2, update), whose
// fixed costs are most of their time.  Per step the warp keeps w, vt, P /
// |d| and P2 in shared memory and runs the same arithmetic as the batched
// kernels, except that P2 = w |d| is computed whole (so floor(P2 / B^s) is
// exact, which the step allows).
// ---------------------------------------------------------------------------
constexpr int SMALL_STEP_LIMBS = 136, SMALL_STEP_WARPS = 4, SMALL_STEP_MAX = 16;

// The steps the fused kernel runs: (l, m, t) of each; N bounds their
// operands (limbs, a multiple of 8): a warp's shared memory holds two
// iterates (N each), vt and |d| (N each), P2 (2 N) and the column sums
// (2 N x 3 words).
struct SmallSteps {
  int n, N;
  int l[SMALL_STEP_MAX], m[SMALL_STEP_MAX], t[SMALL_STEP_MAX];
};
__host__ __device__ constexpr int small_step_warp_limbs(int N) { return 2 * N + 2 * N + 2 * N + 6 * N; }

// Steps S of every instance: the iterate from W0 (its first l + 2 limbs),
// the result (l + m + 2 limbs of the last step) to W0 or W1 as the batched
// steps would leave it (W0 after an even number of steps).
__global__ void __launch_bounds__(32 * SMALL_STEP_WARPS)
    k_ds_small(const uint64_t *__restrict__ V, int nv, uint64_t *W0, uint64_t *W1, int64_t sw,
               int64_t count, SmallSteps S) {
  extern __shared__ __align__(16) uint64_t ssm[];
  const int wi = threadIdx.x >> 5, lane = (int)lane_id();
  const int64_t i = (int64_t)blockIdx.x * SMALL_STEP_WARPS + wi;
  if (i >= count) return;  // the whole warp: no block barrier below
  const int N = S.N;
  uint64_t *base = ssm + (size_t)wi * small_step_warp_limbs(N);
  uint64_t *wb[2] = {base, base + N}, *vts = base + 2 * N, *d = base + 3 * N;
  uint64_t *z = base + 4 * N, *cs = base + 6 * N;
  const uint64_t *v = V + i * nv;
  const int k = nv - 1;
  for (int j = lane; j < S.l[0] + 2; j += 32) wb[0][j] = W0[i * sw + j];
  int cur = 0;
  for (int st = 0; st < S.n; st++) {
    const int l = S.l[st], m = S.m[st], t = S.t[st];
    const int nw = l + 2, nl = t + 2;
    uint64_t *w = wb[cur], *wn = wb[cur ^ 1];
    for (int j = lane; j <= t; j += 32) vts[j] = v[k - t + j];
    __syncwarp();
    // P = vt w mod B^(t+2); |d| = P (top bit clear: d <= 0) or B^(t+2) - P
    warp_mul(vts, t + 1, w, nw, d, nl, cs);
    const bool ng = (d[nl - 1] >> 63) == 0;
    if (!ng) {
      warp_addsub<true>(nl, 0u, [&](int j) { return make_ulonglong2(0ull, d[j]); },
                        [&](int j, uint64_t x) { d[j] = x; });
      __syncwarp();
    }
    // P2 = w |d| (whole); w' = w B^m + floor(P2 / B^s) or w B^m - floor(P2 / B^s) - 1
    warp_mul(w, nw, d, nl, z, nw + nl, cs);
    const int s = t + l - m, ny = nw + nl - s;
    auto load = [&](int j) {
      const uint64_t x = (j >= m && j - m < nw) ? w[j - m] : 0ull;
      return make_ulonglong2(x, j < ny ? z[s + j] : 0ull);
    };
    auto store = [&](int j, uint64_t x) { wn[j] = x; };
    if (ng) warp_addsub<true>(l + m + 2, 1u, load, store);
    else warp_addsub<false>(l + m + 2, 0u, load, store);
    __syncwarp();
    cur ^= 1;
  }
  const int nlast = S.l[S.n - 1] + S.m[S.n - 1] + 2;
  uint64_t *out = (S.n & 1) ? W1 : W0;
  for (int j = lane; j < nlast; j += 32) out[i * sw + j] = wb[cur][j];
}

// One warp per instance: the sign of d from P = vt w mod B^nl and |d| (nl
// limbs): P itself if its top bit is clear (d <= 0), else B^nl - P.
__global__ void __launch_bounds__(WARP_CTA)
    k_ds_mid(const uint64_t *__restrict__ P, int64_t sp, uint64_t *__restrict__ D, int64_t sd,
             int nl, int32_t *neg, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * (WARP_CTA / 32) + (threadIdx.x >> 5);
  if (i >= count) return;
  const uint64_t *p = P + i * sp;
  uint64_t *d = D + i * sd;
  const bool ng = (p[nl - 1] >> 63) == 0;
  if (ng) {
    for (int j = lane_id(); j < nl; j += 32) d[j] = p[j];
  } else {
    warp_addsub<true>(nl, 0u, [&](int j) { return make_ulonglong2(0ull, p[j]); },
                      [&](int j, uint64_t x) { d[j] = x; });
  }
  if (lane_id() == 0) neg[i] = ng ? 1 : 0;
}

// One warp per instance: w' = w B^m + Y (d >= 0) or w B^m - Y - 1 (d < 0),
// Y = floor(P2 / B^s) (ny limbs), into nout limbs of the next iterate record.
__global__ void __launch_bounds__(WARP_CTA)
    k_ds_update(const uint64_t *__restrict__ W, int64_t sw, int nw, const uint64_t *__restrict__ Z,
                int64_t sz, int s, int ny, const int32_t *__restrict__ neg, int m,
                uint64_t *__restrict__ Wn, int nout, int64_t count) {
  const int64_t i = (int64_t)blockIdx.x * (WARP_CTA / 32) + (threadIdx.x >> 5);
  if (i >= count) return;
  const uint64_t *w = W + i * sw, *y = Z + i * sz + s;
  uint64_t *wn = Wn + i * sw;
  auto load = [&](int j) {
    const uint64_t x = (j >= m && j - m < nw) ? w[j - m] : 0ull;
    return make_ulonglong2(x, j < ny ? y[j] : 0ull);
  };
  auto store = [&](int j, uint64_t x) { wn[j] = x; };
  if (neg[i]) warp_addsub<true>(nout, 1u, load, store);
  else warp_addsub<false>(nout, 0u, load, store);
}

// The same two steps with one CTA per instance, for wide records (a warp
// takes its limbs 32 at a time, one round after the other).
__global__ void __launch_bounds__(LIN_THREADS)
    k_ds_mid_cta(const uint64_t *__restrict__ P, int64_t sp, uint64_t *__restrict__ D, int64_t sd,
                 int nl, int32_t *neg) {
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  const int64_t i = blockIdx.x;
  const uint64_t *p = P + i * sp;
  uint64_t *d = D + i * sd;
  const bool ng = (p[nl - 1] >> 63) == 0;
  auto store = [&](int j, uint64_t x) { d[j] = x; };
  if (ng) {
    for (int j = threadIdx.x; j < nl; j += blockDim.x) d[j] = p[j];
  } else {
    auto load = [&](int j) { return make_ulonglong2(0ull, p[j]); };
    blk_addsub<true>(nl, 0u, load, store, scr);
  }
  if (threadIdx.x == 0) neg[i] = ng ? 1 : 0;
}

__global__ void __launch_bounds__(LIN_THREADS)
    k_ds_update_cta(const uint64_t *__restrict__ W, int64_t sw, int nw,
                    const uint64_t *__restrict__ Z, int64_t sz, int s, int ny,
                    const int32_t *__restrict__ neg, int m, uint64_t *__restrict__ Wn, int nout) {
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  const int64_t i = blockIdx.x;
  const uint64_t *w = W + i * sw, *y = Z + i * sz + s;
  uint64_t *wn = Wn + i * sw;
  auto load = [&](int j) {
    const uint64_t x = (j >= m && j - m < nw) ? w[j - m] : 0ull;
    return make_ulonglong2(x, j < ny ? y[j] : 0ull);
  };
  auto store = [&](int j, uint64_t x) { wn[j] = x; };
  if (neg[i]) blk_addsub<true>(nout, 1u, load, store, scr);
  else blk_addsub<false>(nout, 0u, load, store, scr);
}

// Records up to this many limbs take the warp-per-instance kernels.
constexpr int WARP_LIMBS = 1024;

// One CTA per instance: q^ = Z[h .. h + nqh) into its record (zero above).
__global__ void __launch_bounds__(LIN_THREADS)
    k_ds_tail_q(const uint64_t *__restrict__ Z, int64_t sz, int h, int nqh, uint64_t *Qh,
                int64_t sq, int nqcap) {
  const int64_t i = blockIdx.x;
  const uint64_t *z = Z + i * sz + h;
  uint64_t *qh = Qh + i * sq;
  for (int j = threadIdx.x; j < nqcap; j += blockDim.x) qh[j] = j < nqh ? z[j] : 0ull;
}

// One CTA per regular instance: r^ = (u - R) mod B^(nv+1) with R the low
// nv + 1 limbs of q^ v, the exact correction of q^ and r^ (divmod.cu), and
// the results.  Irregular instances are left to the one-CTA-per-division
// kernel.  A tensor-core product of this division that gave up at a wait
// limit (*aborted) voids the results: BIGINT_ETIMEOUT.
__global__ void __launch_bounds__(LIN_THREADS)
    k_ds_finish(const uint64_t *__restrict__ U, int nu, const uint64_t *__restrict__ V, int nv,
                const uint64_t *__restrict__ R, int64_t sp, uint64_t *Rh, int64_t sd, uint64_t *Qh,
                int64_t sq, int nqcap, uint64_t *Qo, int nq, uint64_t *Ro, int32_t *status,
                const int *aborted) {
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  const int64_t i = blockIdx.x;
  const uint64_t *u = U + i * nu, *v = V + i * nv, *rr = R + i * sp;
  if (!regular(u, nu, v, nv)) return;
  uint64_t *rh = Rh + i * sd, *qh = Qh + i * sq;
  {
    auto load = [&](int j) { return make_ulonglong2(j < nu ? u[j] : 0ull, rr[j]); };
    auto store = [&](int j, uint64_t x) { rh[j] = x; };
    blk_addsub<true>(nv + 1, 0u, load, store, scr);
  }
  int st = correct(v, nv, rh, qh, nqcap, scr);
  __syncthreads();
  const int pq = blk_prec(qh, nqcap, scr);
  if (pq > nq && st == BIGINT_OK) st = BIGINT_ERANGE;
  if (*(volatile const int *)aborted) st = BIGINT_ETIMEOUT;
  uint64_t *q = Qo + i * nq, *r = Ro + i * nv;
  for (int j = threadIdx.x; j < nq; j += blockDim.x) q[j] = j < nqcap ? qh[j] : 0ull;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) r[j] = rh[j];
  if (status != nullptr && threadIdx.x == 0) status[i] = st;
}

// The Newton schedule of a regular instance: (l, m, t) per step.
struct Step {
  int l, m, t;
};

int schedule(int k, int h, int l0, Step *steps, int cap) {
  const int L = h - k;
  int l = l0, n = 0;
  while (l < L && n < cap) {
    const int m = (l - 2 < L - l) ? l - 2 : L - l;
    const int t = (k < l + m + 2) ? k : l + m + 2;
    steps[n++] = Step{l, m, t};
    l += m;
  }
  return n;
}

// Per-instance record widths (limbs) and the workspace layout.
struct Layout {
  int64_t sw, sp, sd, sz, sq;  // iterate, low product, |d| / r^, banded product, q^
  size_t w0, w1, p, d, z, qh, neg, total;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

Layout layout(int64_t count, int nu, int nv) {
  Layout Y;
  const int L = nu - nv + 1;
  Y.sw = L + 4;
  Y.sp = nv + 2;
  Y.sd = nv + 2;
  Y.sz = nu + L + 4;
  Y.sq = L + 4;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  Y.w0 = take(8 * count * Y.sw);
  Y.w1 = take(8 * count * Y.sw);
  Y.p = take(8 * count * Y.sp);
  Y.d = take(8 * count * Y.sd);
  Y.z = take(8 * count * Y.sz);
  Y.qh = take(8 * count * Y.sq);
  Y.neg = take(4 * count);
  Y.total = o;
  return Y;
}

}  // namespace dstep

// Smallest divisor (limbs) for which a uniform batch takes the step-batched
// form by default; smaller divisions stay in one CTA each.
constexpr int DIV_STEP_MIN = 128;

// True if divmod_steps can run this shape (with enough workspace).
bool divmod_steps_ok(int64_t count, int nu, int nv, size_t ws_bytes) {
  if (count < 1 || nv < 8 || nu < nv) return false;
  return dstep::layout(count, nu, nv).total <= ws_bytes;
}

bool divmod_steps_default(int nu, int nv) { return nv >= DIV_STEP_MIN && nu >= nv; }

// q = floor(u / v), r = u - q v for a uniform batch, step by step across the
// batch (see the top of this file); irregular instances by the
// one-CTA-per-division kernel at the end.
// ws: ws_bytes for the step records (the one-CTA-per-division kernel's
// per-instance regions, reused); list_and_counters: 4 count bytes rounded to
// 256, then two ints, OUTSIDE those regions (that kernel reads the list
// while it writes its regions); sk: sk_bytes for the column sums of the
// split-K products of a small batch (null: none).
int launch_divmod_steps(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                        int32_t *status, int64_t count, int nu, int nv, void *ws, size_t ws_bytes,
                        void *list_and_counters, void *sk, size_t sk_bytes, cudaStream_t st) {
  using namespace dstep;
  if (!divmod_steps_ok(count, nu, nv, ws_bytes)) return BIGINT_EINVAL;
  const Layout Y = layout(count, nu, nv);
  char *base = static_cast<char *>(ws);
  uint64_t *W[2] = {reinterpret_cast<uint64_t *>(base + Y.w0),
                    reinterpret_cast<uint64_t *>(base + Y.w1)};
  uint64_t *P = reinterpret_cast<uint64_t *>(base + Y.p);
  uint64_t *D = reinterpret_cast<uint64_t *>(base + Y.d);
  uint64_t *Z = reinterpret_cast<uint64_t *>(base + Y.z);
  uint64_t *Qh = reinterpret_cast<uint64_t *>(base + Y.qh);
  int32_t *neg = reinterpret_cast<int32_t *>(base + Y.neg);
  int32_t *list = static_cast<int32_t *>(list_and_counters);
  // [0] irregular instances listed, [1] a tensor-core product gave up
  int *ctr = reinterpret_cast<int *>(static_cast<char *>(list_and_counters) +
                                     ((size_t)4 * count + 255) / 256 * 256);
  const int k = nv - 1, h = nu, L = h - k;
  const int l0 = L < 3 ? L : 3;
  const int nq = nu - nv + 1;
  Step steps[64];
  const int ns = schedule(k, h, l0, steps, 64);
  BIGINT_CUDA_TRY(cudaMemsetAsync(ctr, 0, 8, st));
  k_ds_start<<<(unsigned)((count + 127) / 128), 128, 0, st>>>(u, v, nu, nv, l0, W[0], Y.sw, count,
                                                              list, ctr);
  int rc = bigint_launch_status();
  if (rc != BIGINT_OK) return rc;
  int cur = 0;
  const unsigned gw = (unsigned)((count + WARP_CTA / 32 - 1) / (WARP_CTA / 32));
  // the leading steps whose operands are all small, fused into one launch
  SmallSteps SS;
  SS.n = 0;
  SS.N = 8;
  while (SS.n < ns && SS.n < SMALL_STEP_MAX) {
    const Step &S0 = steps[SS.n];
    // every operand and result of the step within N limbs (w' too)
    const int need = std::max(std::max(S0.l + 2, S0.t + 2), S0.l + S0.m + 2);
    if (need > SMALL_STEP_LIMBS) break;
    SS.N = std::max(SS.N, (need + 7) / 8 * 8);
    SS.l[SS.n] = S0.l;
    SS.m[SS.n] = S0.m;
    SS.t[SS.n] = S0.t;
    SS.n++;
  }
  if (SS.n > 0) {
    const size_t smem = (size_t)8 * SMALL_STEP_WARPS * small_step_warp_limbs(SS.N);
    static bool attr = false;
    if (!attr) {
      BIGINT_CUDA_TRY(cudaFuncSetAttribute(
          k_ds_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
          8 * SMALL_STEP_WARPS * small_step_warp_limbs(SMALL_STEP_LIMBS)));
      attr = true;
    }
    k_ds_small<<<(unsigned)((count + SMALL_STEP_WARPS - 1) / SMALL_STEP_WARPS),
                 32 * SMALL_STEP_WARPS, smem, st>>>(v, nv, W[0], W[1], Y.sw, count, SS);
    if ((rc = bigint_launch_status()) != BIGINT_OK) return rc;
    cur = SS.n & 1;
  }
  for (int i = SS.n; i < ns; i++) {
    const Step S = steps[i];
    const int nw = S.l + 2, nl = S.t + 2;
    // P = vt w mod B^(t+2)
    rc = launch_mul_ex(v + (k - S.t), nv, W[cur], Y.sw, P, Y.sp, count, S.t + 1, nw, nl, 0,
                       ctr + 1, st, STEP_TC_MIN, sk, sk_bytes);
    if (rc != BIGINT_OK) return rc;
    if (nl <= WARP_LIMBS)
      k_ds_mid<<<gw, WARP_CTA, 0, st>>>(P, Y.sp, D, Y.sd, nl, neg, count);
    else
      k_ds_mid_cta<<<(unsigned)count, LIN_THREADS, 0, st>>>(P, Y.sp, D, Y.sd, nl, neg);
    if ((rc = bigint_launch_status()) != BIGINT_OK) return rc;
    // P2 = w |d|, its limbs from s on
    const int s = S.t + S.l - S.m, n2 = nw + nl;
    rc = launch_mul_ex(W[cur], Y.sw, D, Y.sd, Z, Y.sz, count, nw, nl, n2, s - 2, ctr + 1, st, STEP_TC_MIN, sk, sk_bytes);
    if (rc != BIGINT_OK) return rc;
    if (S.l + S.m + 2 <= WARP_LIMBS)
      k_ds_update<<<gw, WARP_CTA, 0, st>>>(W[cur], Y.sw, nw, Z, Y.sz, s, n2 - s, neg, S.m,
                                           W[cur ^ 1], S.l + S.m + 2, count);
    else
      k_ds_update_cta<<<(unsigned)count, LIN_THREADS, 0, st>>>(
          W[cur], Y.sw, nw, Z, Y.sz, s, n2 - s, neg, S.m, W[cur ^ 1], S.l + S.m + 2);
    if ((rc = bigint_launch_status()) != BIGINT_OK) return rc;
    cur ^= 1;
  }
  // q^ = floor(u w / B^h), w of L + 2 limbs
  const int nw = L + 2, nz = nu + nw, nqh = nz - h, nqcap = nqh + 1;
  rc = launch_mul_ex(u, nu, W[cur], Y.sw, Z, Y.sz, count, nu, nw, nz, h - 2, ctr + 1, st, STEP_TC_MIN, sk, sk_bytes);
  if (rc != BIGINT_OK) return rc;
  k_ds_tail_q<<<(unsigned)count, LIN_THREADS, 0, st>>>(Z, Y.sz, h, nqh, Qh, Y.sq, nqcap);
  if ((rc = bigint_launch_status()) != BIGINT_OK) return rc;
  // R = q^ v mod B^(nv+1)
  rc = launch_mul_ex(Qh, Y.sq, v, nv, P, Y.sp, count, nqh, nv, nv + 1, 0, ctr + 1, st, STEP_TC_MIN, sk, sk_bytes);
  if (rc != BIGINT_OK) return rc;
  k_ds_finish<<<(unsigned)count, LIN_THREADS, 0, st>>>(u, nu, v, nv, P, Y.sp, D, Y.sd, Qh, Y.sq,
                                                       nqcap, q, nq, r, status, ctr + 1);
  if ((rc = bigint_launch_status()) != BIGINT_OK) return rc;
  // the irregular instances, one CTA per division (the workspace is free
  // again: everything above is stream-ordered before this launch)
  return launch_divmod_cta(u, v, q, r, status, count, nu, nv, ws, list, ctr, st);
}

size_t divmod_steps_workspace(int64_t count, int nu, int nv) {
  return dstep::layout(count, nu, nv).total;
}

size_t mul_sk_bytes_per_product(int na, int nb, int nout, int lo);

// Batches of at most this many divisions cut their large products over the
// SMs (split-K): a handful of divisions would otherwise run each product on
// a handful of SMs.
constexpr int64_t DIV_SK_MAX_COUNT = 16;

// Column-sum bytes the split-K products of a batch of count 2n/n-shaped
// divisions need (0 for larger batches): the largest over the products of
// the step schedule and of the tail.
size_t divmod_sk_bytes(int64_t count, int nu, int nv) {
  if (count < 1 || count > DIV_SK_MAX_COUNT || nu < nv) return 0;
  const int k = nv - 1, h = nu, L = h - k, l0 = L < 3 ? L : 3;
  dstep::Step steps[64];
  const int ns = dstep::schedule(k, h, l0, steps, 64);
  size_t per = 0;
  auto take = [&](int na, int nb, int nout, int lo) {
    const size_t b = mul_sk_bytes_per_product(na, nb, nout, lo);
    if (b > per) per = b;
  };
  for (int i = 0; i < ns; i++) {
    const dstep::Step S = steps[i];
    const int nw = S.l + 2, nl = S.t + 2;
    take(S.t + 1, nw, nl, 0);
    take(nw, nl, nw + nl, S.t + S.l - S.m - 2);
  }
  const int nw = L + 2;
  take(nu, nw, nu + nw, h - 2);
  take(nw, nv, nv + 1, 0);
  return (size_t)count * per;
}

}  // namespace bigint
