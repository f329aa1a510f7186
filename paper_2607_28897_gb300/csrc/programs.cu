// programs.cu -- fused multi-operation programs per instance (Sec. VI,
// Tables I and II): the whole program runs in one launch, intermediates stay
// on chip (registers) or in a per-CTA scratch region that stays in L2, so
// global-memory traffic is that of one operation.
//
//   add chain:  r = a + b + ... + b  (k additions, k = 6 is Table I's 6-Add),
//               each a full carry-propagating addition mod B^n; carry_out is
//               the number of wrap-arounds, floor((a + k b) / B^n).
//   poly:       r = (a a + b) (b b + b) + a b  mod B^n  (Table II's Poly: four
//               multiplications and three additions, every value kept to n
//               limbs as the paper's same-width multiply and add do).
#include "divcore.cuh"

namespace bigint {

// ---------------------------------------------------------------------------
// Carry into this thread's segment when every thread holds a segment of
// consecutive limbs in thread order with (generate, propagate) = (g, p) and
// the block gets carry cin; *cout = carry out of the last thread.  The scan
// of Fig. 3 with warp ballots, then across warps (blk_addsub's resolve).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t blk_segment_carry(uint32_t g, uint32_t p, uint32_t cin,
                                                      uint32_t *sm, uint32_t *cout) {
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const WarpCarry wc = warp_gp(g, p);
  if (lane == 0) {
    sm[warp] = warp_carry_out(wc, 0);
    sm[32 + warp] = warp_all_propagate(wc);
  }
  __syncthreads();
  const uint32_t gw = (int)lane < nwarps ? sm[lane] : 0;
  const uint32_t pw = (int)lane < nwarps ? sm[32 + lane] : 1;
  const uint64_t cm = warp_carries(warp_gp(gw, pw), cin);
  const uint32_t cwarp = (uint32_t)(cm >> warp) & 1u;
  *cout = (uint32_t)(cm >> nwarps) & 1u;
  const uint64_t lc = warp_carries(wc, cwarp);
  __syncthreads();  // sm is reused by the next call
  return (uint32_t)(lc >> lane) & 1u;
}

// One CTA per instance; thread t holds limbs [t L, t L + L) of the running
// sum and of b in registers for all k additions.
template <int L>
__global__ void __launch_bounds__(1024)
    k_add_chain(const uint64_t *__restrict__ A, const uint64_t *__restrict__ Bm,
                uint64_t *__restrict__ Out, uint8_t *carry_out, int n, int k) {
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  const int64_t inst = blockIdx.x;
  const uint64_t *a = A + inst * (int64_t)n, *b = Bm + inst * (int64_t)n;
  uint64_t *o = Out + inst * (int64_t)n;
  const int base = (int)threadIdx.x * L;
  int nv = n - base;
  nv = nv < 0 ? 0 : (nv > L ? L : nv);
  uint64_t r[L], y[L];
#pragma unroll
  for (int j = 0; j < L; j++) {
    r[j] = j < nv ? a[base + j] : 0ull;
    y[j] = j < nv ? b[base + j] : 0ull;
  }
  uint32_t total = 0;
  for (int it = 0; it < k; it++) {
    uint32_t c = 0, all_ones = 1;
#pragma unroll
    for (int j = 0; j < L; j++) {
      if (j < nv) {
        const uint64_t t = r[j] + y[j];
        const uint64_t t2 = t + c;
        c = (uint32_t)(t < r[j]) | (uint32_t)(t2 < t);
        r[j] = t2;
        all_ones &= (uint32_t)(t2 == ~0ull);
      }
    }
    // a segment past the end passes carries through
    const uint32_t g = nv > 0 ? c : 0u, p = nv > 0 ? (c == 0u && all_ones) : 1u;
    uint32_t cout;
    uint32_t cin = blk_segment_carry(g, p, 0u, scr, &cout);
#pragma unroll
    for (int j = 0; j < L; j++) {
      if (j < nv && cin) {
        r[j] += 1;
        cin = r[j] == 0 ? 1u : 0u;
      }
    }
    total += cout;
  }
#pragma unroll
  for (int j = 0; j < L; j++)
    if (j < nv) o[base + j] = r[j];
  if (carry_out && threadIdx.x == 0) carry_out[inst] = (uint8_t)total;
}

// ---------------------------------------------------------------------------
// Poly: persistent CTAs; per instance four low-part products (tensor cores
// when n >= TC_DIV_MIN, with the tile of NT columns that holds the n / 16
// columns of a low n x n product, so that small programs run several CTAs
// per SM; else blk_mul) and three in-place additions through a per-CTA
// scratch of 3n limbs.
// ---------------------------------------------------------------------------
template <bool TC, int NT, int G>
__global__ void __launch_bounds__(TC ? 2 * NT + 32 : 512, TC ? 256 / NT : 1)
    k_poly(const uint64_t *__restrict__ A, const uint64_t *__restrict__ Bm,
           uint64_t *__restrict__ Out, int n, int64_t count, uint64_t *scratch, int smem_words) {
  extern __shared__ __align__(1024) uint32_t smem[];
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  __shared__ tcm::TcShared tsh;
  tcm::TcCtx tcc;
  if constexpr (TC) tcm::tc_init<NT>(tcc, reinterpret_cast<uint8_t *>(smem), &tsh, scr);
  uint64_t *T1 = scratch + (int64_t)blockIdx.x * 3 * n, *T2 = T1 + n, *T3 = T2 + n;
  auto prod = [&](const uint64_t *x, const uint64_t *y, uint64_t *out) {
    if constexpr (TC) {
      tcm::tc_product<NT, G, true>(tcc, x, n, y, n, out, n, 0);
    } else {
      blk_mul_call<divc::DRB, divc::DQ, divc::DF>(x, n, y, n, out, n, smem, 0);
    }
  };
  auto add_into = [&](uint64_t *t, const uint64_t *u) {  // t = t + u mod B^n
    auto load = [&](int j) { return make_ulonglong2(t[j], u[j]); };
    auto store = [&](int j, uint64_t v) { t[j] = v; };
    blk_addsub<false>(n, 0u, load, store, scr);
  };
  for (int64_t inst = blockIdx.x; inst < count; inst += gridDim.x) {
    const uint64_t *a = A + inst * (int64_t)n, *b = Bm + inst * (int64_t)n;
    uint64_t *o = Out + inst * (int64_t)n;
    prod(a, a, T1);
    add_into(T1, b);
    prod(b, b, T2);
    add_into(T2, b);
    prod(T1, T2, T3);
    prod(a, b, o);
    add_into(o, T3);
    __syncthreads();
    if constexpr (TC) {
      if (tcc.aborted) break;
    }
  }
  if constexpr (TC) tcm::tc_release<NT>(tcc);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int launch_add_chain(const uint64_t *a, const uint64_t *b, uint64_t *out, uint8_t *carry,
                     int64_t count, int n, int k, cudaStream_t st) {
  if (count == 0) return BIGINT_OK;
  if (n <= 8 * 1024) {
    const int T = ((n + 7) / 8 + 31) / 32 * 32;
    k_add_chain<8><<<(unsigned)count, T, 0, st>>>(a, b, out, carry, n, k);
  } else {
    const int T = ((n + 15) / 16 + 31) / 32 * 32;
    k_add_chain<16><<<(unsigned)count, T, 0, st>>>(a, b, out, carry, n, k);
  }
  return bigint_launch_status();
}

namespace {

template <bool TC, int NT, int G>
int poly_dyn_max() {
  static int dyn = -1;
  if (dyn < 0) {
    int dev = 0, optin = 0;
    BIGINT_CUDA_TRY(cudaGetDevice(&dev));
    BIGINT_CUDA_TRY(
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    BIGINT_CUDA_TRY(cudaFuncGetAttributes(&fa, k_poly<TC, NT, G>));
    const int d = optin - (int)fa.sharedSizeBytes;
    BIGINT_CUDA_TRY(cudaFuncSetAttribute(k_poly<TC, NT, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, d));
    dyn = d;
  }
  return dyn;
}

// CTAs of k_poly<TC, NT, G> resident on one SM with `smem` bytes of dynamic
// shared memory (the tensor memory allows 256 / NT of them), 0 on error.
template <bool TC, int NT, int G>
int poly_per_sm(size_t smem) {
  int dev = 0, smem_sm = 0, reserved = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
          cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
          cudaSuccess)
    return 0;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, k_poly<TC, NT, G>) != cudaSuccess) return 0;
  int per = smem_sm / (int)(smem + fa.sharedSizeBytes + reserved);
  const int cap = TC ? 256 / NT : 1;
  if (per > cap) per = cap;
  return per < 1 ? 1 : per;
}

int sm_count(int *sms) {
  int dev = 0;
  BIGINT_CUDA_TRY(cudaGetDevice(&dev));
  BIGINT_CUDA_TRY(cudaDeviceGetAttribute(sms, cudaDevAttrMultiProcessorCount, dev));
  return BIGINT_OK;
}

// The launch of Poly for n-limb operands: which k_poly, its dynamic shared
// memory and CTAs per SM.  Tensor cores from TC_DIV_MIN limbs with the
// smallest tile holding the n / 16 columns of a low n x n product.
struct PolyPlan {
  int form;  // 0: integer, 1: NT 64, 2: NT 128, 3: NT 256 G 8, 4: NT 256 G 4
  size_t smem;
  int per_sm;
};

template <bool TC, int NT, int G>
bool poly_try(int form, size_t smem, PolyPlan &P) {
  const int dyn = poly_dyn_max<TC, NT, G>();
  if (dyn <= 0 || smem > (size_t)dyn) return false;
  P.form = form;
  P.smem = smem;
  P.per_sm = poly_per_sm<TC, NT, G>(smem);
  return P.per_sm > 0;
}

bool poly_plan(int n, PolyPlan &P) {
  if (n >= divc::TC_DIV_MIN) {
    const int cols = (n + 15) / 16;
    if (cols <= 64 && poly_try<true, 64, 7>(1, tcm::layout<64, 7>(n, n).total, P)) return true;
    if (cols <= 128 && poly_try<true, 128, 8>(2, tcm::layout<128, 8>(n, n).total, P)) return true;
    if (poly_try<true, 256, 8>(3, tcm::layout<256, 8>(n, n).total, P)) return true;
    if (poly_try<true, 256, 4>(4, tcm::layout<256, 4>(n, n).total, P)) return true;
  }
  return poly_try<false, 256, 8>(0, 4 * (size_t)blk_mul_smem_words<divc::DRB, divc::DQ>(n, n),
                                 P);
}

int64_t poly_grid(const PolyPlan &P, int64_t count) {
  int sms = 0;
  if (sm_count(&sms) != BIGINT_OK) return 0;
  const int64_t slots = (int64_t)sms * P.per_sm;
  return count < slots ? count : slots;
}

template <bool TC, int NT, int G>
int launch_poly_variant(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int n,
                        void *ws, int64_t grid, size_t smem, cudaStream_t st) {
  k_poly<TC, NT, G><<<(unsigned)grid, TC ? 2 * NT + 32 : 512, smem, st>>>(
      a, b, out, n, count, static_cast<uint64_t *>(ws), (int)(smem / 4));
  return bigint_launch_status();
}

}  // namespace

// BIGINT_ETIMEOUT if a Poly launch's tensor-core product hit a wait limit
// since the last call (synchronises the device), else BIGINT_OK.
int programs_take_timeout() { return tcm::take_timeout_here(); }
int programs_set_wait_limit(long long cycles) { return tcm::set_wait_limit_here(cycles); }

size_t poly_workspace(int64_t count, int n) {
  PolyPlan P;
  if (n < 1 || !poly_plan(n, P)) return 0;
  const int64_t grid = poly_grid(P, count);
  return (size_t)(grid > 0 ? grid : 1) * 3 * (size_t)n * 8;
}

int launch_poly(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int n,
                void *ws, size_t bytes, cudaStream_t st) {
  if (count == 0) return BIGINT_OK;
  PolyPlan P;
  if (!poly_plan(n, P)) return BIGINT_EINVAL;
  const int64_t grid = poly_grid(P, count);
  if (grid <= 0) return BIGINT_ECUDA;
  if (bytes < (size_t)grid * 3 * n * 8) return BIGINT_ENOMEM;
  switch (P.form) {
    case 1: return launch_poly_variant<true, 64, 7>(a, b, out, count, n, ws, grid, P.smem, st);
    case 2: return launch_poly_variant<true, 128, 8>(a, b, out, count, n, ws, grid, P.smem, st);
    case 3: return launch_poly_variant<true, 256, 8>(a, b, out, count, n, ws, grid, P.smem, st);
    case 4: return launch_poly_variant<true, 256, 4>(a, b, out, count, n, ws, grid, P.smem, st);
    default: return launch_poly_variant<false, 256, 8>(a, b, out, count, n, ws, grid, P.smem, st);
  }
}

}  // namespace bigint
