// divmod.cu -- batched division by the shifted inverse (Sec. V-C, Fig. 6).
//
// One CTA per instance runs the whole division, as the paper's Futhark code
// does (one intragroup kernel).  Operands, Newton iterates and products live
// in a per-instance region of the caller's workspace (L2-resident for the
// instance's lifetime); every multiplication is staged through shared memory
// by blk_mul (mulcore.cuh), every linear step is a block-level pass of
// blockops.cuh.
//
// With k = prec(v) - 1 (so B^k <= v < B^(k+1)) and h = prec(u):
//   1. w ~ shinv_h(v) = floor(B^h / v) by Newton steps (A7, A8):
//      * start: l = min(3, h - k) and w = floor(B^(2l) / V), V the top
//        l+1 limbs of v plus one (or v B^(l-k) when v is shorter), so that
//        0 <= B^(k+l)/v - w < 2;
//      * step (Fig. 6): with m = min(l - 2, h - k - l) new limbs and the
//        divisor truncated to its top t+1 limbs, t = min(k, l + m + 2),
//          d  = B^(t+l) - v_t w,
//          w' = w B^m + floor(w d / B^(t+l-m))    if d >= 0,
//          w' = w B^m - ceil(w |d| / B^(t+l-m))   if d <  0,
//        and l grows by m.  The exact Newton update loses v e^2 B^(m-l-k)
//        units for an iterate e units low (the identity the oracle tests
//        pin), so with m <= l - 2 the error stays below 1 + 2^-60 units;
//        the truncation of v costs under B^-2 units per step.
//   2. q^ = floor(u w / B^h) (one product) and r^ = u - q^ v computed
//      modulo B^(k+2) (a low-half product, the varPrecMul of Fig. 6);
//   3. exact correction: while r^ < 0 { r^ += v; q^-- }, while r^ >= v
//      { r^ -= v; q^++ } -- at most a few rounds, capped (BIGINT_EINTERNAL).
// Only q and r are binding; the iterates are this library's reading of the
// refinement loop, which the paper leaves to Watt's algorithm.
#include "divcore.cuh"

namespace bigint {

using namespace divc;


// mode 0: divmod (q, r); mode 1: shinv (w = floor(B^h / v) into q, nq = nw);
// mode 2: divmod (q, r) from a given inverse Wg = floor(B^h / v) (nwg limbs,
// h >= nu): floor(floor(B^h / v) / B^s) = floor(B^(h-s) / v), so the top
// limbs of Wg are the inverse at h - s = prec(u), the one mode 0 computes,
// and the division finishes as mode 0 does without the Newton steps.
// v_stride / w_stride: limbs between the instances' divisors / inverses (0:
// one for the whole batch).
// Thread cap per product variant: 512 gives the wide-chunk variant 128
// registers (no spills in its products); the small variant keeps a 640 cap,
// whose 96-register budget fits two blocks of ~320 threads on one SM.  The
// tensor-core variant (TC) runs exactly tcm::TC_CTA_THREADS threads and holds
// all 512 TMEM columns of its SM: products with a shorter operand of
// TC_DIV_MIN limbs or more run on the tensor cores (tccore.cuh), smaller
// ones on blk_mul.
template <int Q, bool TC> constexpr int div_max_threads() {
  return TC ? tcm::TC_CTA_THREADS : (Q >= 16 ? 512 : 640);
}

// Without a list, CTA b divides instance b (grid = count).  With a list (the
// instances the step-batched form leaves out, divstep.cu), CTA b divides
// instances list[b], list[b + grid], ... of the *nlist listed; CTAs beyond
// *nlist return before they take any tensor memory.
template <int RB, int Q, int F, bool TC>
__global__ void __launch_bounds__(div_max_threads<Q, TC>())
    k_divmod(const uint64_t *__restrict__ U, const uint64_t *__restrict__ V, uint64_t *Qo,
             uint64_t *Ro, int32_t *status, int nu, int nv, int nq, int mode, int h_arg,
             uint64_t *ws, int64_t ws_stride, int smem_words, const uint64_t *Wg, int nwg,
             int64_t v_stride, int64_t w_stride, const int32_t *list, const int *nlist) {
  extern __shared__ __align__(1024) uint32_t smem[];
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  __shared__ tcm::TcShared tsh;
  const int64_t nwork = list != nullptr ? (int64_t)*(volatile const int *)nlist : gridDim.x;
  if ((int64_t)blockIdx.x >= nwork) return;
  tcm::TcCtx tcc;
  tcm::TcCtx *tc = nullptr;
  if constexpr (TC) {
    tcm::tc_init<256>(tcc, reinterpret_cast<uint8_t *>(smem), &tsh, scr);
    tc = &tcc;
  }
  for (int64_t b = blockIdx.x; b < nwork; b += gridDim.x) {
  const int64_t inst = list != nullptr ? (int64_t)list[b] : b;
  const uint64_t *v = V + inst * v_stride;
  uint64_t *q = Qo + inst * (int64_t)nq;
  const int hcap = mode == 1 ? h_arg : nu;
  Work W = carve(ws + inst * ws_stride, nu, nv, hcap);
  int st = BIGINT_OK;

  [&] {
    const int kv = blk_prec(v, nv, scr);
    if (kv == 0) {  // division by zero: q = r = 0
      blk_zero(q, nq);
      if (mode == 0) blk_zero(Ro + inst * (int64_t)nv, nv);
      st = BIGINT_EDIVZERO;
      return;
    }
    const int k = kv - 1;

    if (mode == 1) {
      // ---- shifted inverse: w = floor(B^h / v), h = h_arg >= nv >= kv
      const int h = h_arg;
      int nw = shinv_newton<RB, Q, F, TC>(v, k, h, W, smem, smem_words, scr, tc);
      // R = (B^h - v w) mod B^(kv+1), then exact correction of w
      mul_any<RB, Q, F, TC>(v, kv, W.w, nw, W.p, kv + 1, W.tmp, smem, smem_words, 0, tc);
      {
        uint64_t *P = W.p, *R = W.r;
        auto load = [&](int j) { return make_ulonglong2(j == h ? 1ull : 0ull, P[j]); };
        auto store = [&](int j, uint64_t x) { R[j] = x; };
        blk_addsub<true>(kv + 1, 0u, load, store, scr);
      }
      // w may grow by one limb in the correction
      for (int j = threadIdx.x + nw; j < W.cap_w; j += blockDim.x) W.w[j] = 0;
      st = correct(v, kv, W.r, W.w, nw + 1 < W.cap_w ? nw + 1 : W.cap_w, scr);
      __syncthreads();
      const int pw = blk_prec(W.w, W.cap_w, scr);
      if (pw > nq && st == BIGINT_OK) st = BIGINT_ERANGE;
      for (int j = threadIdx.x; j < nq; j += blockDim.x) q[j] = j < W.cap_w ? W.w[j] : 0;
      return;
    }

    if (mode == 2) {
      // ---- division from the given inverse
      const uint64_t *u = U + inst * (int64_t)nu;
      uint64_t *r = Ro + inst * (int64_t)nv;
      const int ku = blk_prec(u, nu, scr);
      if (ku < kv) {  // u < v: q = 0, r = u
        blk_zero(q, nq);
        for (int j = threadIdx.x; j < nv; j += blockDim.x) r[j] = j < ku ? u[j] : 0;
        __syncthreads();
        return;
      }
      const uint64_t *wg = Wg + inst * w_stride;
      const int s = h_arg - ku;  // inverse at h = ku: drop the low s limbs
      const int pw = blk_prec(wg, nwg, scr);
      const int nw = pw > s ? pw - s : 0;
      if (nw == 0) {  // floor(B^ku / v) >= 1 for a true inverse: this w is not one
        blk_zero(q, nq);
        blk_zero(r, nv);
        st = BIGINT_EINTERNAL;
        return;
      }
      st = divmod_tail<RB, Q, F, TC>(u, ku, v, kv, wg + s, nw, ku, q, nq, r, nv, W, smem,
                                     smem_words, scr, tc);
      return;
    }

    // ---- division
    st = divmod_one<RB, Q, F, TC>(U + inst * (int64_t)nu, nu, v, nv, q, nq,
                                  Ro + inst * (int64_t)nv, ws + inst * ws_stride, smem,
                                  smem_words, scr, tc);
  }();

  if constexpr (TC) {
    if (tcc.aborted) st = BIGINT_ETIMEOUT;
  }
  if (status && threadIdx.x == 0) status[inst] = st;
  __syncthreads();
  }
  if constexpr (TC) tcm::tc_release<256>(tcc);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// Division kernels for H >= DIV_SMALL_LIMBS run their large products on the
// tensor cores unless switched off (bigint_set_variant(1, ...)).
static int g_div_tc = 1;
// Uniform divisions: the step-batched form (divstep.cu) for divisors of
// DIV_STEP_MIN limbs and more (0), never (1, 2: one CTA per division), or
// for every divisor of 8 limbs and more (3).
static int g_div_steps = 0;

int div_set_variant(int v) {
  if (v < 0 || v > 3) return BIGINT_EINVAL;
  g_div_tc = v != 2;
  g_div_steps = v == 0 ? 0 : (v == 3 ? 2 : 1);
  return BIGINT_OK;
}

// BIGINT_ETIMEOUT if a division kernel's tensor-core product hit a wait
// limit since the last call (synchronises the device), else BIGINT_OK.
int div_take_timeout() { return tcm::take_timeout_here(); }
int div_set_wait_limit(long long cycles) { return tcm::set_wait_limit_here(cycles); }

static int div_smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return v;
}

// Per-instance regions of the one-CTA-per-division kernel, then (for the
// step-batched form) the list of instances it leaves to that kernel and two
// counters; the step-batched form's own records fit inside the regions.
static size_t cta_regions_bytes(int64_t count, int nu, int nv) {
  return (size_t)count * (size_t)ws_limbs(nu, nv, nu) * sizeof(uint64_t);
}

size_t divmod_sk_bytes(int64_t count, int nu, int nv);

// ... and, for a small batch, the column sums of its split-K products.
static size_t list_end(int64_t count, int nu, int nv) {
  return cta_regions_bytes(count, nu, nv) + ((size_t)4 * count + 255) / 256 * 256 + 256;
}

size_t divmod_workspace(int64_t count, int nu, int nv) {
  return list_end(count, nu, nv) + divmod_sk_bytes(count, nu, nv);
}

size_t shinv_workspace(int64_t count, int nv, int h) {
  return (size_t)count * (size_t)ws_limbs(nv, nv, h) * sizeof(uint64_t);
}

// Operands of one launch beyond those of divmod: the given inverses of
// mode 2 and the distance between the instances' divisors and inverses.
struct DivExtra {
  const uint64_t *w = nullptr;
  int nw = 0;
  int64_t v_stride = -1;  // -1: nv
  int64_t w_stride = 0;
  const int32_t *list = nullptr;  // instances to divide (device), *nlist of them
  const int *nlist = nullptr;
};

template <int RB, int Q, int F, bool TC>
static int launch_div_variant(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                              int32_t *status, int64_t count, int nu, int nv, int nq, int mode,
                              int h, void *ws, cudaStream_t st, const DivExtra &x) {
  const int optin = div_smem_optin();
  if (optin == 0) return BIGINT_ECUDA;
  static int dyn_max = -1;  // opt-in limit minus the kernel's static shared memory
  if (dyn_max < 0) {
    cudaFuncAttributes fa;
    BIGINT_CUDA_TRY(cudaFuncGetAttributes(&fa, k_divmod<RB, Q, F, TC>));
    dyn_max = optin - (int)fa.sharedSizeBytes;
    BIGINT_CUDA_TRY(cudaFuncSetAttribute(k_divmod<RB, Q, F, TC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max));
  }
  int smem_words = dyn_max / 4;
  // the largest product a division performs is about (2 H) x H limbs;
  // ask for no more shared memory than one such product needs
  const int H = (mode == 1 ? h : nu);
  int need = blk_mul_smem_words<RB, Q>(H, H);
  if (TC) {  // tensor-core products: shorter operand up to max(H - nv, nv) + a few limbs
    const int ns = (H - nv > nv ? H - nv : nv) + 8;
    const tcm::Layout L8 = tcm::layout<256, 8>(ns, H + 8);
    const tcm::Layout L4 = tcm::layout<256, 4>(ns, H + 8);
    const int w8 = (int)(L8.total / 4), w4 = (int)(L4.total / 4);
    const int tcw = w8 <= smem_words ? w8 : w4;
    if (tcw > need) need = tcw;
  }
  if (need < smem_words) smem_words = need;
  int T;
  if (TC) {
    T = tcm::TC_CTA_THREADS;
  } else {
    const int units = blk_mul_units<RB, Q>(H < 8192 ? H : 8192, H < 8192 ? H : 8192);
    constexpr int TMAX = div_max_threads<Q, TC>();
    T = (units + TMAX - 1) / TMAX;
    T = (units + T - 1) / T;
    T = (T + 31) / 32 * 32;
    if (T < 64) T = 64;
    if (T > TMAX) T = TMAX;
  }
  const int hcap = mode == 1 ? h : nu;
  const int64_t stride = ws_limbs(nu, nv, hcap);
  int64_t grid = count;
  if (x.list != nullptr) {  // a listed subset: a few CTAs per SM loop over it
    static int sms = 0;
    if (sms == 0) {
      int dev = 0;
      BIGINT_CUDA_TRY(cudaGetDevice(&dev));
      BIGINT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int64_t slots = (int64_t)sms * (TC ? 1 : 2);
    if (grid > slots) grid = slots;
  }
  k_divmod<RB, Q, F, TC><<<(unsigned)grid, T, (size_t)smem_words * 4, st>>>(
      u, v, q, r, status, nu, nv, nq, mode, h, reinterpret_cast<uint64_t *>(ws), stride,
      smem_words, x.w, x.nw, x.v_stride < 0 ? nv : x.v_stride, x.w_stride, x.list, x.nlist);
  return bigint_launch_status();
}

static int launch_div_common(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                             int32_t *status, int64_t count, int nu, int nv, int nq, int mode,
                             int h, void *ws, cudaStream_t st, const DivExtra &x = DivExtra()) {
  const int H = (mode == 1 ? h : nu);
  if (H < DIV_SMALL_LIMBS)
    return launch_div_variant<SRB, SQ, SF, false>(u, v, q, r, status, count, nu, nv, nq, mode, h,
                                                  ws, st, x);
  if (g_div_tc)
    return launch_div_variant<DRB, DQ, DF, true>(u, v, q, r, status, count, nu, nv, nq, mode, h,
                                                 ws, st, x);
  return launch_div_variant<DRB, DQ, DF, false>(u, v, q, r, status, count, nu, nv, nq, mode, h,
                                                ws, st, x);
}

bool divmod_steps_ok(int64_t count, int nu, int nv, size_t ws_bytes);
bool divmod_steps_default(int nu, int nv);
int launch_divmod_steps(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                        int32_t *status, int64_t count, int nu, int nv, void *ws, size_t ws_bytes,
                        void *list_and_counters, void *sk, size_t sk_bytes, cudaStream_t st);

// One CTA per division for the listed instances (or all, list = null).
int launch_divmod_cta(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                      int32_t *status, int64_t count, int nu, int nv, void *ws,
                      const int32_t *list, const int *nlist, cudaStream_t st) {
  const int nq = nu - nv + 1 > 1 ? nu - nv + 1 : 1;
  DivExtra x;
  x.list = list;
  x.nlist = nlist;
  return launch_div_common(u, v, q, r, status, count, nu, nv, nq, 0, nu, ws, st, x);
}

// The step-batched form (divstep.cu) where it applies, else one CTA per
// division.
int launch_divmod(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                  int32_t *status, int64_t count, int nu, int nv, void *ws, size_t ws_bytes,
                  cudaStream_t st) {
  const size_t regions = cta_regions_bytes(count, nu, nv);
  const bool steps = g_div_steps == 2 ? true : (g_div_steps == 0 && divmod_steps_default(nu, nv));
  if (steps && ws_bytes >= divmod_workspace(count, nu, nv) &&
      divmod_steps_ok(count, nu, nv, regions)) {
    const size_t skb = divmod_sk_bytes(count, nu, nv);
    char *w = static_cast<char *>(ws);
    return launch_divmod_steps(u, v, q, r, status, count, nu, nv, ws, regions, w + regions,
                               skb ? w + list_end(count, nu, nv) : nullptr, skb, st);
  }
  return launch_divmod_cta(u, v, q, r, status, count, nu, nv, ws, nullptr, nullptr, st);
}

// q, r of u / v from w = floor(B^h / v) (h >= nu, h >= nv), per instance or
// shared (strides 0); the workspace of launch_divmod.
int launch_divmod_inv(const uint64_t *u, const uint64_t *v, const uint64_t *w, uint64_t *q,
                      uint64_t *r, int32_t *status, int64_t count, int nu, int nv, int nw, int h,
                      int64_t v_stride, int64_t w_stride, void *ws, cudaStream_t st) {
  const int nq = nu - nv + 1 > 1 ? nu - nv + 1 : 1;
  DivExtra x;
  x.w = w;
  x.nw = nw;
  x.v_stride = v_stride;
  x.w_stride = w_stride;
  return launch_div_common(u, v, q, r, status, count, nu, nv, nq, 2, h, ws, st, x);
}

int launch_shinv(const uint64_t *v, uint64_t *w, int32_t *status, int64_t count, int nv, int h,
                 int nw, void *ws, size_t, cudaStream_t st) {
  return launch_div_common(nullptr, v, w, nullptr, status, count, nv, nv, nw, 1, h, ws, st);
}

}  // namespace bigint
