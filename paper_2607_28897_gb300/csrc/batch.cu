// batch.cu -- ragged batches of mixed operations (add, sub, mul, divmod).
//
// A batch is a list of operation descriptors (bigint_op, include/bigint.h)
// over one input pool and one output pool of limbs.  Two ways to run it:
//
//   * persistent: ONE launch of grid = SMs x resident CTAs; every CTA takes
//     the next operation from a device-side work queue (one atomicAdd on a
//     counter per operation) until the queue is empty.  The queue order is
//     the operations sorted by estimated cost, largest first, so the tail of
//     the launch is made of small operations.  The launch (counter reset +
//     kernel) contains no host-side step and can be captured in a CUDA graph.
//   * per class: one launch per (operation, size class) with size classes
//     [2^k, 2^(k+1)) limbs, each launch striding over its class -- the
//     plain form the persistent one is compared against.
//
// Each operation is executed by the whole CTA with the block-level routines
// of the uniform kernels (blk_addsub, blk_mul, divc::divmod_one), so a
// result is bit-identical whichever form, CTA size or batch it runs in.
// Workspace: the division scratch of one operation per CTA.
#include <algorithm>
#include <vector>

#include "divcore.cuh"

namespace bigint {

using namespace divc;

struct OpDev {
  int32_t op, na, nb, pad;
  int64_t a, b, o1, o2;
};
static_assert(sizeof(OpDev) == sizeof(bigint_op), "descriptor layout");

// Product variant used by batch kernels (both operands in shared memory).
constexpr int BRB = 29, BQ = 16, BF = 32;
constexpr int BATCH_MAX_THREADS = 512;

template <bool TC>
__device__ __forceinline__ int op_status(const OpDev &o, const uint64_t *in, uint64_t *out,
                                         uint64_t *ws, uint32_t *smem, int smem_words,
                                         uint32_t *scr, tcm::TcCtx *tc) {
  switch (o.op) {
    case BIGINT_OP_ADD:
    case BIGINT_OP_SUB: {
      // operands of different lengths (BIGINT_ZEXT) are zero-extended to
      // the longer one, which is the result's length
      const uint64_t *a = in + o.a, *b = in + o.b;
      uint64_t *r = out + o.o1;
      const int n = o.na > o.nb ? o.na : o.nb;
      auto load = [&](int j) {
        return make_ulonglong2(j < o.na ? a[j] : 0ull, j < o.nb ? b[j] : 0ull);
      };
      auto store = [&](int j, uint64_t x) { r[j] = x; };
      return o.op == BIGINT_OP_ADD ? (int)blk_addsub<false>(n, 0u, load, store, scr)
                                   : (int)blk_addsub<true>(n, 0u, load, store, scr);
    }
    case BIGINT_OP_MUL:
      if constexpr (TC) {
        if (tc_mul(tc, in + o.a, o.na, in + o.b, o.nb, out + o.o1, o.na + o.nb, smem_words, 0))
          return 0;
      }
      blk_mul_call<BRB, BQ, BF>(in + o.a, o.na, in + o.b, o.nb, out + o.o1, o.na + o.nb, smem, 0);
      return 0;
    case BIGINT_OP_DIVMOD: {
      const int nq = o.na - o.nb + 1 > 1 ? o.na - o.nb + 1 : 1;
      return divmod_one<DRB, DQ, DF, TC>(in + o.a, o.na, in + o.b, o.nb, out + o.o1, nq,
                                         out + o.o2, ws, smem, smem_words, scr, tc);
    }
    default:
      return BIGINT_EINVAL;
  }
}

// TC: tcm::TC_CTA_THREADS threads holding the SM's tensor memory; products
// with a shorter operand of TC_DIV_MIN limbs or more (multiplications, and
// the products inside divisions) run on the tensor cores.
template <bool TC>
__global__ void __launch_bounds__(TC ? tcm::TC_CTA_THREADS : BATCH_MAX_THREADS)
    k_batch(const OpDev *__restrict__ ops, const int32_t *__restrict__ order, int first,
            int count, const uint64_t *in, uint64_t *out, int32_t *status, uint64_t *ws,
            int64_t ws_per_cta, int *queue, int smem_words) {
  extern __shared__ __align__(1024) uint32_t smem[];
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  __shared__ int s_idx;
  __shared__ tcm::TcShared tsh;
  uint64_t *my_ws = ws + (int64_t)blockIdx.x * ws_per_cta;
  tcm::TcCtx tcc;
  tcm::TcCtx *tc = nullptr;
  if constexpr (TC) {
    tcm::tc_init<256>(tcc, reinterpret_cast<uint8_t *>(smem), &tsh, scr);
    tc = &tcc;
  }
  int stride_idx = blockIdx.x;
  for (;;) {
    int idx;
    if (queue != nullptr) {  // persistent: take the next operation
      if (threadIdx.x == 0) s_idx = atomicAdd(queue, 1);
      __syncthreads();
      idx = s_idx;
      __syncthreads();
    } else {  // per class: static stride over the class
      idx = stride_idx;
      stride_idx += gridDim.x;
    }
    if (idx >= count) break;
    const int opi = order[first + idx];
    const OpDev o = ops[opi];
    int st = op_status<TC>(o, in, out, my_ws, smem, smem_words, scr, tc);
    if constexpr (TC) {
      if (tcc.aborted) st = BIGINT_ETIMEOUT;
    }
    if (status != nullptr && threadIdx.x == 0) status[opi] = st;
    __syncthreads();
  }
  if constexpr (TC) tcm::tc_release<256>(tcc);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

double op_cost(const bigint_op &o) {
  switch (o.op) {
    case BIGINT_OP_ADD:
    case BIGINT_OP_SUB: return (double)(o.na > o.nb ? o.na : o.nb);
    case BIGINT_OP_MUL: return (double)o.na * o.nb;
    case BIGINT_OP_DIVMOD: {
      const double nq = o.na - o.nb + 1 > 1 ? o.na - o.nb + 1 : 1;
      return 2.0 * nq * o.nb + 1.4 * (double)o.nb * std::min<double>(o.nb, nq) + o.na;
    }
    default: return 0;
  }
}

int size_class(const bigint_op &o) {
  const int n = o.na > o.nb ? o.na : o.nb;
  int c = 0;
  while ((2 << c) <= n) c++;
  return c;
}

int op_smem_words(const bigint_op &o) {
  if (o.op == BIGINT_OP_MUL) return blk_mul_smem_words<BRB, BQ>(o.na, o.nb);
  if (o.op == BIGINT_OP_DIVMOD) return blk_mul_smem_words<DRB, DQ>(o.na, o.na);
  return BLK_SCRATCH_WORDS;
}

// Operations that use the tensor cores in a TC launch, and the shared
// memory (words) their largest tensor-core product needs.
bool op_tc(const bigint_op &o) {
  if (o.op == BIGINT_OP_MUL) return std::min(o.na, o.nb) >= TC_DIV_MIN;
  if (o.op == BIGINT_OP_DIVMOD) return o.nb >= TC_DIV_MIN || o.na - o.nb >= TC_DIV_MIN;
  return false;
}

int op_tc_words(const bigint_op &o, int max_words) {
  int ns, nl;
  if (o.op == BIGINT_OP_MUL) {
    ns = std::min(o.na, o.nb);
    nl = std::max(o.na, o.nb);
  } else if (o.op == BIGINT_OP_DIVMOD) {
    ns = std::max(o.na - o.nb, o.nb) + 8;
    nl = o.na + 8;
  } else {
    return 0;
  }
  const int w8 = (int)(tcm::layout<256, 8>(ns, nl).total / 4);
  const int w4 = (int)(tcm::layout<256, 4>(ns, nl).total / 4);
  return w8 <= max_words ? w8 : w4;
}

int op_units(const bigint_op &o) {
  const int a = std::min(o.na, 8192), b = std::min(o.nb, 8192);
  if (o.op == BIGINT_OP_MUL) return blk_mul_units<BRB, BQ>(a, b);
  if (o.op == BIGINT_OP_DIVMOD) return blk_mul_units<DRB, DQ>(a, a);
  return std::min(std::max(o.na, o.nb) / 8 + 32, 512);
}

int threads_for_units(int units) {
  int rounds = (units + BATCH_MAX_THREADS - 1) / BATCH_MAX_THREADS;
  int T = (units + rounds - 1) / rounds;
  T = (T + 31) / 32 * 32;
  return std::max(64, std::min(T, BATCH_MAX_THREADS));
}

int g_batch_threads = 0;  // tuned CTA size of persistent launches (0: from the sizes)

struct Launch {
  int first, count, threads, ctas, smem_words;
  bool tc;  // k_batch<true>: TC_CTA_THREADS threads, one CTA per SM, tensor-core products
};

}  // namespace

int g_batch_tc = 1;  // tensor-core launches for new batches (bigint_set_variant(2, ...))

int batch_set_variant(int v) {
  if (v < 0 || v > 2) return BIGINT_EINVAL;
  g_batch_tc = v != 2;
  return BIGINT_OK;
}

int batch_set_threads(int t) {
  if (t != 0 && (t < 64 || t > BATCH_MAX_THREADS || t % 32)) return BIGINT_EINVAL;
  g_batch_threads = t;
  return BIGINT_OK;
}
int batch_get_threads() { return g_batch_threads; }

// A class of divisions of nearby shapes run together in the step-batched
// form: every member u (nu limbs) / v (nv limbs) is padded to u' = u B^s
// (H limbs) and v' = v B^s (NV limbs), s = NV - nv, so floor(u'/v') =
// floor(u/v) and u' mod v' = (u mod v) B^s (same quotient, the remainder
// shifted by s limbs); the quotient has LQ = H - NV + 1 limbs.
struct DivClass {
  int H, NV, LQ, first, count;
};

// One CTA per member of a class: the padded operands.
__global__ void __launch_bounds__(256)
    k_cls_gather(const OpDev *__restrict__ ops, const int32_t *__restrict__ order, int first,
                 const uint64_t *__restrict__ in, uint64_t *Uc, uint64_t *Vc, int H, int NV) {
  const OpDev o = ops[order[first + blockIdx.x]];
  const int s = NV - o.nb;
  const uint64_t *a = in + o.a, *b = in + o.b;
  uint64_t *u = Uc + (int64_t)blockIdx.x * H, *v = Vc + (int64_t)blockIdx.x * NV;
  for (int j = threadIdx.x; j < H; j += blockDim.x)
    u[j] = (j >= s && j - s < o.na) ? a[j - s] : 0ull;
  for (int j = threadIdx.x; j < NV; j += blockDim.x) v[j] = j >= s ? b[j - s] : 0ull;
}

// One CTA per member: q (its max(nu - nv + 1, 1) limbs) and r (nv limbs,
// the padded remainder shifted back by s) into the output pool; status
// BIGINT_ERANGE where the quotient does not fit its limbs (a divisor with
// zero top limbs), else the class division's status.
__global__ void __launch_bounds__(256)
    k_cls_scatter(const OpDev *__restrict__ ops, const int32_t *__restrict__ order, int first,
                  const uint64_t *__restrict__ Qc, const uint64_t *__restrict__ Rc,
                  const int32_t *__restrict__ stc, uint64_t *out, int32_t *status, int LQ, int NV) {
  const int opi = order[first + blockIdx.x];
  const OpDev o = ops[opi];
  const int s = NV - o.nb, nq = o.na - o.nb + 1 > 1 ? o.na - o.nb + 1 : 1;
  const uint64_t *q = Qc + (int64_t)blockIdx.x * LQ, *r = Rc + (int64_t)blockIdx.x * NV;
  int high = 0;
  for (int j = threadIdx.x; j < LQ; j += blockDim.x) {
    if (j < nq) out[o.o1 + j] = q[j];
    else if (q[j] != 0) high = 1;
  }
  for (int j = threadIdx.x; j < o.nb; j += blockDim.x) out[o.o2 + j] = r[s + j];
  high = __syncthreads_or(high);
  if (status != nullptr && threadIdx.x == 0) {
    int st = stc[blockIdx.x];
    if (st == BIGINT_OK && high) st = BIGINT_ERANGE;
    status[opi] = st;
  }
}

}  // namespace bigint

// The opaque batch handle of include/bigint.h.
struct bigint_batch {
  std::vector<bigint_op> ops;
  std::vector<int32_t> order_persistent;  // cost-sorted, largest first
  std::vector<int32_t> order_classes;     // grouped by (op, size class)
  std::vector<bigint::Launch> classes;    // one launch per class
  bigint::Launch persistent;
  // BIGINT_BATCH_STEPS: divisions grouped into shape classes (each run
  // step-batched on padded operands), the other operations persistent
  std::vector<int32_t> order_rest;        // order_persistent without the class divisions
  std::vector<int32_t> order_div;         // the class divisions, class by class
  std::vector<bigint::DivClass> div_classes;
  int64_t ws_limbs_per_cta = 0;
  int max_ctas = 0;
  size_t desc_off = 0, order_p_off = 0, order_c_off = 0, queue_off = 0, scratch_off = 0;
  size_t order_r_off = 0, order_d_off = 0, cls_off = 0, cls_ws_off = 0, cls_ws_bytes = 0;
  size_t workspace_bytes = 0;
  int sms = 0, optin = 0;
  int threads_override = 0;  // set by the tuner for this batch
  bool use_tc = true;        // tensor-core launches for large products (batch_set_tc)
};

namespace bigint {
namespace {

// Largest dynamic shared memory (words) of a k_batch<TC> launch.
template <bool TC>
int max_dyn_words() {
  static int words = -1;
  if (words < 0) {
    int dev = 0, optin = 0;
    BIGINT_CUDA_TRY(cudaGetDevice(&dev));
    BIGINT_CUDA_TRY(
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    BIGINT_CUDA_TRY(cudaFuncGetAttributes(&fa, k_batch<TC>));
    const int bytes = optin - (int)fa.sharedSizeBytes;
    BIGINT_CUDA_TRY(cudaFuncSetAttribute(k_batch<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         bytes));
    words = bytes / 4;
  }
  return words;
}

int occupancy(bool tc, int threads, int smem_words, int *per_sm) {
  if (tc) {  // all 512 TMEM columns: one CTA per SM
    *per_sm = 1;
    return max_dyn_words<true>() < 0 ? BIGINT_ECUDA : BIGINT_OK;
  }
  if (max_dyn_words<false>() < 0) return BIGINT_ECUDA;
  BIGINT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_batch<false>, threads,
                                                                (size_t)smem_words * 4));
  if (*per_sm < 1) *per_sm = 1;
  return BIGINT_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

size_t divmod_workspace(int64_t count, int nu, int nv);

namespace {

// Divisions with divisors of at least this many limbs join shape classes.
constexpr int CLS_MIN_NV = 128;
// A class keeps divisors within 1/8 and quotient lengths within 1/4 (plus
// 64 limbs) of its smallest, and has at least CLS_MIN_COUNT members (fewer
// stay with the persistent launch: a class costs some 50 small launches).
constexpr int CLS_MIN_COUNT = 8;

// Groups the batch's large divisions into classes of nearby shapes and
// orders the other operations for the persistent launch of the steps form.
void plan_div_classes(bigint_batch *B) {
  B->order_div.clear();
  B->div_classes.clear();
  std::vector<int32_t> cand;
  for (int32_t i = 0; i < (int32_t)B->ops.size(); i++) {
    const bigint_op &o = B->ops[i];
    if (o.op == BIGINT_OP_DIVMOD && o.nb >= CLS_MIN_NV && o.na >= o.nb) cand.push_back(i);
  }
  auto L = [&](int32_t i) { return B->ops[i].na - B->ops[i].nb + 1; };
  std::stable_sort(cand.begin(), cand.end(),
                   [&](int32_t x, int32_t y) { return B->ops[x].nb < B->ops[y].nb; });
  std::vector<char> in_class(B->ops.size(), 0);
  for (size_t i = 0; i < cand.size();) {
    const int nv0 = B->ops[cand[i]].nb;
    size_t j = i;
    while (j < cand.size() && (int64_t)B->ops[cand[j]].nb * 8 <= (int64_t)nv0 * 9) j++;
    std::stable_sort(cand.begin() + i, cand.begin() + j,
                     [&](int32_t x, int32_t y) { return L(x) < L(y); });
    for (size_t a = i; a < j;) {
      const int l0 = L(cand[a]);
      size_t b = a;
      int nv = 0, lq = 0;
      while (b < j && (int64_t)L(cand[b]) * 4 <= (int64_t)l0 * 5 + 256) {
        nv = std::max(nv, (int)B->ops[cand[b]].nb);
        lq = std::max(lq, L(cand[b]));
        b++;
      }
      if (b - a >= (size_t)CLS_MIN_COUNT) {
        DivClass c;
        c.NV = nv;
        c.LQ = lq;
        c.H = nv + lq - 1;
        c.first = (int)B->order_div.size();
        c.count = (int)(b - a);
        for (size_t k = a; k < b; k++) {
          B->order_div.push_back(cand[k]);
          in_class[cand[k]] = 1;
        }
        B->div_classes.push_back(c);
      }
      a = b;
    }
    i = j;
  }
  B->order_rest.clear();
  for (int32_t i : B->order_persistent)
    if (!in_class[i]) B->order_rest.push_back(i);
}

}  // namespace

int batch_configure(bigint_batch *B) {
  const int64_t n = (int64_t)B->ops.size();
  const int max_words = max_dyn_words<false>(), max_words_tc = max_dyn_words<true>();
  if (max_words < 0 || max_words_tc < 0) return BIGINT_ECUDA;
  // persistent launch: one shape for every operation
  int words = BLK_SCRATCH_WORDS, units = 32, tc_words = 0;
  bool tc = false;
  for (const bigint_op &o : B->ops) {
    words = std::max(words, op_smem_words(o));
    units = std::max(units, op_units(o));
    if (B->use_tc && op_tc(o)) {
      tc = true;
      tc_words = std::max(tc_words, op_tc_words(o, max_words_tc));
    }
  }
  Launch &P = B->persistent;
  P.first = 0;
  P.count = (int)n;
  P.tc = tc;
  if (tc) {
    P.smem_words = std::min(std::max(words, tc_words), max_words_tc);
    P.threads = tcm::TC_CTA_THREADS;
  } else {
    P.smem_words = std::min(words, max_words);
    P.threads = B->threads_override
                    ? B->threads_override
                    : (g_batch_threads ? g_batch_threads : threads_for_units(units));
  }
  int per_sm = 1;
  int rc = occupancy(P.tc, P.threads, P.smem_words, &per_sm);
  if (rc != BIGINT_OK) return rc;
  // no more CTAs than operations: each resident CTA holds a division scratch
  // region of the workspace, which a small batch should not pay for
  P.ctas = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)B->sms * per_sm, n));
  B->max_ctas = P.ctas;
  // per-class launches
  B->classes.clear();
  for (size_t i = 0; i < B->order_classes.size();) {
    const bigint_op &o0 = B->ops[B->order_classes[i]];
    size_t j = i;
    int w = BLK_SCRATCH_WORDS, u = 32, tw = 0;
    bool ltc = false;
    while (j < B->order_classes.size()) {
      const bigint_op &o = B->ops[B->order_classes[j]];
      if (o.op != o0.op || size_class(o) != size_class(o0)) break;
      w = std::max(w, op_smem_words(o));
      u = std::max(u, op_units(o));
      if (B->use_tc && op_tc(o)) {
        ltc = true;
        tw = std::max(tw, op_tc_words(o, max_words_tc));
      }
      j++;
    }
    Launch L;
    L.first = (int)i;
    L.count = (int)(j - i);
    L.tc = ltc;
    L.smem_words = ltc ? std::min(std::max(w, tw), max_words_tc) : std::min(w, max_words);
    L.threads = ltc ? tcm::TC_CTA_THREADS : threads_for_units(u);
    rc = occupancy(L.tc, L.threads, L.smem_words, &per_sm);
    if (rc != BIGINT_OK) return rc;
    L.ctas = std::min(L.count, B->sms * per_sm);
    B->max_ctas = std::max(B->max_ctas, L.ctas);
    B->classes.push_back(L);
    i = j;
  }
  // workspace: descriptors | two orders | queue counter | per-CTA scratch
  B->desc_off = 0;
  B->order_p_off = align256(n * sizeof(bigint_op));
  B->order_c_off = B->order_p_off + align256(n * 4);
  B->queue_off = B->order_c_off + align256(n * 4);
  B->scratch_off = B->queue_off + 256;
  // the steps form: the rest's order, the class divisions' order, then one
  // set of padded operands / results / statuses and one division workspace,
  // sized for the largest class (the classes run one after the other)
  B->order_r_off = B->scratch_off + align256((size_t)B->max_ctas * B->ws_limbs_per_cta * 8);
  B->order_d_off = B->order_r_off + align256(B->order_rest.size() * 4);
  B->cls_off = B->order_d_off + align256(B->order_div.size() * 4);
  size_t cls = 0, cls_ws = 0;
  for (const DivClass &c : B->div_classes) {
    const size_t cnt = (size_t)c.count;
    cls = std::max(cls, align256(8 * cnt * c.H) + align256(8 * cnt * c.NV) +
                            align256(8 * cnt * c.LQ) + align256(8 * cnt * c.NV) +
                            align256(4 * cnt));
    cls_ws = std::max(cls_ws, divmod_workspace(c.count, c.H, c.NV));
  }
  B->cls_ws_off = B->cls_off + cls;
  B->cls_ws_bytes = cls_ws;
  B->workspace_bytes = B->div_classes.empty() ? B->order_d_off : B->cls_ws_off + cls_ws;
  return BIGINT_OK;
}

int launch_divmod(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                  int32_t *status, int64_t count, int nu, int nv, void *ws, size_t ws_bytes,
                  cudaStream_t st);

int batch_create(const bigint_op *ops, int64_t nops, bigint_batch **out) {
  if (!out || nops < 0 || nops > 0x7fffffff || (nops > 0 && !ops)) return BIGINT_EINVAL;
  for (int64_t i = 0; i < nops; i++) {
    const bigint_op &o = ops[i];
    if (o.op < BIGINT_OP_ADD || o.op > BIGINT_OP_DIVMOD) return BIGINT_EINVAL;
    if (o.na < 1 || o.nb < 1 || o.na > BIGINT_MAX_LIMBS || o.nb > BIGINT_MAX_LIMBS)
      return BIGINT_EINVAL;
    if ((o.op == BIGINT_OP_ADD || o.op == BIGINT_OP_SUB) && o.na != o.nb &&
        !(o.flags & BIGINT_ZEXT))
      return BIGINT_EINVAL;
    if (o.flags & ~BIGINT_ZEXT) return BIGINT_EINVAL;
    if (o.op == BIGINT_OP_MUL && (o.na > BIGINT_MUL_MAX_LIMBS || o.nb > BIGINT_MUL_MAX_LIMBS))
      return BIGINT_EINVAL;
    if (o.a < 0 || o.b < 0 || o.o1 < 0 || o.o2 < 0) return BIGINT_EINVAL;
  }
  bigint_batch *B = new bigint_batch;
  B->ops.assign(ops, ops + nops);
  B->use_tc = g_batch_tc != 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&B->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&B->optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
          cudaSuccess) {
    delete B;
    return BIGINT_ECUDA;
  }
  B->order_persistent.resize(nops);
  B->order_classes.resize(nops);
  for (int64_t i = 0; i < nops; i++) B->order_persistent[i] = B->order_classes[i] = (int32_t)i;
  std::stable_sort(B->order_persistent.begin(), B->order_persistent.end(),
                   [&](int32_t x, int32_t y) { return op_cost(ops[x]) > op_cost(ops[y]); });
  std::stable_sort(B->order_classes.begin(), B->order_classes.end(), [&](int32_t x, int32_t y) {
    const int kx = ops[x].op * 64 + size_class(ops[x]), ky = ops[y].op * 64 + size_class(ops[y]);
    return kx < ky;
  });
  for (const bigint_op &o : B->ops)
    if (o.op == BIGINT_OP_DIVMOD) B->ws_limbs_per_cta = std::max(B->ws_limbs_per_cta, ws_limbs(o.na, o.nb, o.na));
  plan_div_classes(B);
  const int rc = batch_configure(B);
  if (rc != BIGINT_OK) {
    delete B;
    return rc;
  }
  *out = B;
  return BIGINT_OK;
}

int batch_upload(bigint_batch *B, void *ws, size_t bytes, cudaStream_t st) {
  if (!B || (!ws && B->workspace_bytes) || bytes < B->workspace_bytes) return BIGINT_ENOMEM;
  if (((uintptr_t)ws) % 256) return BIGINT_EINVAL;
  char *w = static_cast<char *>(ws);
  const size_t n = B->ops.size();
  if (n == 0) return BIGINT_OK;
  BIGINT_CUDA_TRY(cudaMemcpyAsync(w + B->desc_off, B->ops.data(), n * sizeof(bigint_op),
                                  cudaMemcpyHostToDevice, st));
  BIGINT_CUDA_TRY(cudaMemcpyAsync(w + B->order_p_off, B->order_persistent.data(), n * 4,
                                  cudaMemcpyHostToDevice, st));
  BIGINT_CUDA_TRY(cudaMemcpyAsync(w + B->order_c_off, B->order_classes.data(), n * 4,
                                  cudaMemcpyHostToDevice, st));
  if (!B->order_rest.empty())
    BIGINT_CUDA_TRY(cudaMemcpyAsync(w + B->order_r_off, B->order_rest.data(),
                                    B->order_rest.size() * 4, cudaMemcpyHostToDevice, st));
  if (!B->order_div.empty())
    BIGINT_CUDA_TRY(cudaMemcpyAsync(w + B->order_d_off, B->order_div.data(),
                                    B->order_div.size() * 4, cudaMemcpyHostToDevice, st));
  return BIGINT_OK;
}

int batch_launch(const bigint_batch *B, const uint64_t *in, uint64_t *out, int32_t *status,
                 void *ws, int mode, cudaStream_t st) {
  if (!B || !in || !out) return BIGINT_EINVAL;
  if (B->ops.empty()) return BIGINT_OK;
  char *w = static_cast<char *>(ws);
  const OpDev *ops = reinterpret_cast<const OpDev *>(w + B->desc_off);
  uint64_t *scratch = reinterpret_cast<uint64_t *>(w + B->scratch_off);
  if (mode == BIGINT_BATCH_PERSISTENT) {
    const Launch &P = B->persistent;
    int *queue = reinterpret_cast<int *>(w + B->queue_off);
    BIGINT_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(int), st));
    auto *kern = P.tc ? k_batch<true> : k_batch<false>;
    kern<<<P.ctas, P.threads, (size_t)P.smem_words * 4, st>>>(
        ops, reinterpret_cast<const int32_t *>(w + B->order_p_off), 0, P.count, in, out, status,
        scratch, B->ws_limbs_per_cta, queue, P.smem_words);
    return bigint_launch_status();
  }
  if (mode == BIGINT_BATCH_STEPS) {
    // the operations outside the division classes: one persistent launch
    const Launch &P = B->persistent;
    const int nrest = (int)B->order_rest.size();
    if (nrest > 0) {
      int *queue = reinterpret_cast<int *>(w + B->queue_off);
      BIGINT_CUDA_TRY(cudaMemsetAsync(queue, 0, sizeof(int), st));
      auto *kern = P.tc ? k_batch<true> : k_batch<false>;
      kern<<<std::min(P.ctas, nrest), P.threads, (size_t)P.smem_words * 4, st>>>(
          ops, reinterpret_cast<const int32_t *>(w + B->order_r_off), 0, nrest, in, out, status,
          scratch, B->ws_limbs_per_cta, queue, P.smem_words);
      const int rc = bigint_launch_status();
      if (rc != BIGINT_OK) return rc;
    }
    // each class of divisions: padded operands, the step-batched division,
    // results back into the pool
    const int32_t *order_d = reinterpret_cast<const int32_t *>(w + B->order_d_off);
    for (const DivClass &c : B->div_classes) {
      const size_t cnt = (size_t)c.count;
      char *p = w + B->cls_off;
      uint64_t *Uc = reinterpret_cast<uint64_t *>(p); p += align256(8 * cnt * c.H);
      uint64_t *Vc = reinterpret_cast<uint64_t *>(p); p += align256(8 * cnt * c.NV);
      uint64_t *Qc = reinterpret_cast<uint64_t *>(p); p += align256(8 * cnt * c.LQ);
      uint64_t *Rc = reinterpret_cast<uint64_t *>(p); p += align256(8 * cnt * c.NV);
      int32_t *stc = reinterpret_cast<int32_t *>(p);
      k_cls_gather<<<(unsigned)c.count, 256, 0, st>>>(ops, order_d, c.first, in, Uc, Vc, c.H,
                                                        c.NV);
      int rc = bigint_launch_status();
      if (rc != BIGINT_OK) return rc;
      rc = launch_divmod(Uc, Vc, Qc, Rc, stc, c.count, c.H, c.NV, w + B->cls_ws_off,
                         B->cls_ws_bytes, st);
      if (rc != BIGINT_OK) return rc;
      k_cls_scatter<<<(unsigned)c.count, 256, 0, st>>>(ops, order_d, c.first, Qc, Rc, stc, out,
                                                         status, c.LQ, c.NV);
      rc = bigint_launch_status();
      if (rc != BIGINT_OK) return rc;
    }
    return BIGINT_OK;
  }
  if (mode != BIGINT_BATCH_PER_CLASS) return BIGINT_EINVAL;
  for (const Launch &L : B->classes) {
    auto *kern = L.tc ? k_batch<true> : k_batch<false>;
    kern<<<L.ctas, L.threads, (size_t)L.smem_words * 4, st>>>(
        ops, reinterpret_cast<const int32_t *>(w + B->order_c_off), L.first, L.count, in, out,
        status, scratch, B->ws_limbs_per_cta, nullptr, L.smem_words);
    const int rc = bigint_launch_status();
    if (rc != BIGINT_OK) return rc;
  }
  return BIGINT_OK;
}

size_t batch_workspace_bytes(const bigint_batch *B) { return B ? B->workspace_bytes : 0; }

// Reconfigures the batch's launches: CTA size of its integer-only persistent
// launch (0: from the sizes) and whether large products run on the tensor
// cores (use_tc: 1 yes, 0 no, -1 unchanged).
int batch_retune(bigint_batch *B, int threads, int use_tc) {
  if (!B) return BIGINT_EINVAL;
  B->threads_override = threads;
  if (use_tc >= 0) B->use_tc = use_tc != 0;
  return batch_configure(B);
}

bool batch_uses_tc(const bigint_batch *B) { return B && B->persistent.tc; }
int batch_threads_of(const bigint_batch *B) { return B ? B->persistent.threads : 0; }

void batch_destroy(bigint_batch *B) { delete B; }

// The batch kernel's own record of tensor-core products that gave up at a
// wait limit, and its wait limit (see tcm::take_timeout_here).
int batch_take_timeout() { return tcm::take_timeout_here(); }
int batch_set_wait_limit(long long cycles) { return tcm::set_wait_limit_here(cycles); }

}  // namespace bigint
