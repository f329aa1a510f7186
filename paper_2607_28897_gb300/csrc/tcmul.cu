// tcmul.cu -- batched full (and low-part) products on the tensor cores.
//
// Persistent CTAs, one per SM (NT = 256), two (NT = 128) or three (NT = 64),
// loop over the instances of a uniform batch, each product computed by tc_product
// (tccore.cuh: the digit convolution as tcgen05 fp16 MMAs with exact fp32
// accumulation, Sec. V-B's schoolbook product on the tensor cores).
#include "tccore.cuh"

namespace bigint {
namespace tcm {

// 2 NT drain threads plus one issuer warp (tc_product<NT, G, true, XC, false,
// KB>).
// Instance i's operands start at X + i sx and Y + i sy, its result at
// Out + i so (limbs); lo > 0 is tc_product's band mode.  A CTA that gives up
// at a wait limit also sets *abort_flag (if given), so that a caller
// chaining products (the step-batched division) can report it per instance.
template <int NT, int G, bool XC, int KB = 128>
__global__ void __launch_bounds__(2 * NT + 32, 256 / NT)
    k_mul_tc(const uint64_t *__restrict__ X, const uint64_t *__restrict__ Y,
             uint64_t *__restrict__ Out, int nx, int ny, int nout, int64_t count, int64_t sx,
             int64_t sy, int64_t so, int lo, int *abort_flag) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ TcShared sh;
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  TcCtx c;
  tc_init<NT>(c, sm, &sh, scr);
  for (int64_t inst = blockIdx.x; inst < count; inst += gridDim.x) {
    const int64_t next = inst + gridDim.x;
    if (threadIdx.x == 0 && next < count) {
      prefetch_l2(X + next * sx, 8 * (size_t)nx);
      prefetch_l2(Y + next * sy, 8 * (size_t)ny);
    }
    if (!tc_product<NT, G, true, XC, false, KB>(c, X + inst * sx, nx, Y + inst * sy, ny,
                                                Out + inst * so, nout, lo))
      break;
  }
  if (c.aborted && abort_flag != nullptr && threadIdx.x == 0) atomicExch(abort_flag, 1);
  tc_release<NT>(c);
}

// Split products: unit u is tile u % T of product u / T (tc_product's split
// mode), its outgoing (high word, carry) at tile_carry[2 u], [2 u + 1].
template <int NT, int G>
__global__ void __launch_bounds__(2 * NT + 32, 1)
    k_mul_tc_split(const uint64_t *__restrict__ X, const uint64_t *__restrict__ Y,
                   uint64_t *__restrict__ Out, int nx, int ny, int nout, int64_t count, int T,
                   uint64_t *tile_carry) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ TcShared sh;
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  TcCtx c;
  tc_init<NT>(c, sm, &sh, scr);
  const int64_t units = count * T;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t inst = u / T;
    if (!tc_product<NT, G, true, true, true>(c, X + inst * (int64_t)nx, nx, Y + inst * (int64_t)ny,
                                             ny, Out + inst * (int64_t)nout, nout, 0,
                                             (int)(u - inst * T), tile_carry + 2 * u))
      break;
  }
  tc_release<NT>(c);
}

// ---- split-K products ---------------------------------------------------------
// A product cut into units of (tile, groups of Toeplitz blocks) so that even
// a single product keeps many SMs busy (tc_partial adds each unit's column
// sums into the product's buffer; k_tc_sk_finish turns them into limbs).
constexpr int SK_MAX_TILES = 8;
struct SkPlan {
  int T;                          // tiles
  int gpc;                        // groups per unit
  int cfirst;                     // first column of the first tile
  int c0[SK_MAX_TILES], W[SK_MAX_TILES];
  int first[SK_MAX_TILES + 1];    // first unit of each tile; first[T] units per product
};

template <int NT, int G>
__global__ void __launch_bounds__(2 * NT + 32, 1)
    k_mul_tc_sk(const uint64_t *__restrict__ X, const uint64_t *__restrict__ Y, int nx, int ny,
                int64_t sx, int64_t sy, int64_t count, SkPlan P, int *colsum, int64_t cs_stride,
                int *abort_flag) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ TcShared sh;
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  TcCtx c;
  tc_init<NT>(c, sm, &sh, scr);
  const int upi = P.first[P.T];
  for (int64_t u = blockIdx.x; u < count * upi; u += gridDim.x) {
    const int64_t inst = u / upi;
    const int r = (int)(u - inst * upi);
    int t = 0;
    while (t + 1 < P.T && P.first[t + 1] <= r) t++;
    const int g0 = (r - P.first[t]) * P.gpc;
    if (!tc_partial<NT, G>(c, X + inst * sx, nx, Y + inst * sy, ny, P.c0[t], P.W[t], g0,
                           g0 + P.gpc, colsum + inst * cs_stride + (P.c0[t] - P.cfirst) * 128))
      break;
  }
  if (c.aborted && abort_flag != nullptr && threadIdx.x == 0) atomicExch(abort_flag, 1);
  tc_release<NT>(c);
}

// One CTA per product: its limbs [L0, nout) from its column sums.
__global__ void __launch_bounds__(512)
    k_tc_sk_finish(const int *colsum, int64_t cs_stride, uint64_t *Out, int64_t so, int L0,
                   int nout, uint64_t margin) {
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  tc_colsum_limbs(colsum + blockIdx.x * cs_stride, L0, nout, margin, Out + blockIdx.x * so, scr);
}

// One CTA per product: tile t (limbs [t L, t L + L), L = tile_limbs) was
// computed without what flows in from tile t - 1, i.e. the high word H of
// that tile's last column sum and its carry out k.  So the product is the
// concatenated tiles plus sum_t (H_t + k_t) B^((t + 1) L), less the bias sum
// of the column sums (as in the unsplit product): two carry passes.
__global__ void __launch_bounds__(512)
    k_tc_split_finish(uint64_t *Out, int nout, int T, int tile_limbs, const uint64_t *tile_carry) {
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  uint64_t *o = Out + (int64_t)blockIdx.x * nout;
  const uint64_t *tc = tile_carry + 2 * (int64_t)blockIdx.x * T;
  auto st = [&](int j, uint64_t v) { o[j] = v; };
  auto ld_links = [&](int j) {
    uint64_t v = 0;
    if (j > 0 && j % tile_limbs == 0) {
      const int t = j / tile_limbs - 1;
      v = tc[2 * t] + tc[2 * t + 1];
    }
    return make_ulonglong2(o[j], v);
  };
  blk_addsub<false>(nout, 0u, ld_links, st, scr);
  auto ld_bias = [&](int j) {
    return make_ulonglong2(o[j], j == 0 ? 0x8080808080000000ull : 0x8080808080808080ull);
  };
  blk_addsub<true>(nout, 0u, ld_bias, st, scr);
}

}  // namespace tcm

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <int NT, int G, bool XC, int KB>
static int tc_dyn_max() {
  static int dyn = -1;
  if (dyn < 0) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
      return 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, tcm::k_mul_tc<NT, G, XC, KB>) != cudaSuccess) return 0;
    const int d = optin - (int)fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(tcm::k_mul_tc<NT, G, XC, KB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, d) != cudaSuccess)
      return 0;
    dyn = d;
  }
  return dyn;
}

// The kernel shapes (tile columns NT, group G, x's carry digit XC, x block
// width KB).  128-digit blocks: the 256-column tile, one CTA per SM, for
// large products; the 128- and 64-column tiles (two and three CTAs per SM)
// for products whose columns fit one such tile, x's carry digit dropped
// (XC = false: one correction addition) where that makes them fit.  Narrow
// blocks (64 or 32 digits, 128-column tiles, two CTAs per SM) give each MMA
// 2 or 4 times the columns for the same 4 KB A operand, which bounds narrow
// MMAs; measured on GB300 they tie with 128-digit blocks at 512-limb
// products and lose from 1024 limbs on (4x the drains and column-sum rows
// per digit), so only the autotuner and the forced variants take them.
enum TcShape {
  TC_64_XC, TC_64_NOXC, TC_128_XC, TC_128_NOXC, TC_256,
  TC_N64_XC, TC_N64_NOXC, TC_N32_XC, TC_N32_NOXC, TC_NSHAPES
};
struct ShapeInfo {
  int nt, g, kb;
  bool xc;
};
static constexpr ShapeInfo SHAPES[TC_NSHAPES] = {
    {64, 7, 128, true},   {64, 7, 128, false},  {128, 8, 128, true}, {128, 8, 128, false},
    {256, 8, 128, true},  {128, 15, 64, true},  {128, 15, 64, false}, {128, 12, 32, true},
    {128, 12, 32, false}};

template <int NT, int G, bool XC, int KB>
static size_t tc_smem(int nx, int ny) {
  const tcm::Layout L = tcm::layout<NT, G, XC, KB>(nx, ny);
  const int d = tc_dyn_max<NT, G, XC, KB>();
  return d > 0 && L.total <= (uint32_t)d ? L.total : 0;
}

// Shared memory of a shape for x of nx and y of ny limbs, 0 if it does not
// fit (the 256-column tile falls back to groups of 4 blocks).
static size_t shape_smem(TcShape sh, int nx, int ny) {
  switch (sh) {
    case TC_64_XC: return tc_smem<64, 7, true, 128>(nx, ny);
    case TC_64_NOXC: return tc_smem<64, 7, false, 128>(nx, ny);
    case TC_128_XC: return tc_smem<128, 8, true, 128>(nx, ny);
    case TC_128_NOXC: return tc_smem<128, 8, false, 128>(nx, ny);
    case TC_N64_XC: return tc_smem<128, 15, true, 64>(nx, ny);
    case TC_N64_NOXC: return tc_smem<128, 15, false, 64>(nx, ny);
    case TC_N32_XC: return tc_smem<128, 12, true, 32>(nx, ny);
    case TC_N32_NOXC: return tc_smem<128, 12, false, 32>(nx, ny);
    default: {
      const size_t s8 = tc_smem<256, 8, true, 128>(nx, ny);
      return s8 ? s8 : tc_smem<256, 4, true, 128>(nx, ny);
    }
  }
}

// Dynamic shared memory the tensor-core product of an na x nb product
// needs with the 256-column tile (which every product that fits any shape
// fits), or 0 if it does not fit (or the shapes are out of range).
size_t mul_tc_smem(int na, int nb) {
  const int nx = na < nb ? na : nb, ny = na < nb ? nb : na;
  if (nx < 1 || nx > 16383 || ny > 32768) return 0;
  return shape_smem(TC_256, nx, ny);
}

// Operands and results of one batched product launch: instance i's x at
// x + i sx, y at y + i sy, result at out + i so (limbs); band start lo (0:
// the low nout limbs exactly); abort_flag as for k_mul_tc (may be null).
struct TcArgs {
  const uint64_t *x, *y;
  uint64_t *out;
  int64_t sx, sy, so;
  int lo;
  int *abort_flag;
};

// CTAs of a shape resident on one SM: TMEM allows 256 / NT, shared memory
// per SM / (dynamic + static + the per-block reservation).
template <int NT, int G, bool XC, int KB>
static int tc_per_sm(size_t smem) {
  static int smem_sm = 0, reserved = 0, static_smem = -1;
  if (static_smem < 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) !=
            cudaSuccess)
      return 1;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, tcm::k_mul_tc<NT, G, XC, KB>) != cudaSuccess) return 1;
    static_smem = (int)fa.sharedSizeBytes;
  }
  int per_sm = smem_sm / (int)(smem + static_smem + reserved);
  if (per_sm > 256 / NT) per_sm = 256 / NT;
  return per_sm < 1 ? 1 : per_sm;
}

static int sm_count() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  }
  return sms;
}

template <int NT, int G, bool XC, int KB>
static int launch_tc(const TcArgs &A, int64_t count, int nx, int ny, int nout, cudaStream_t st) {
  const size_t smem = tc_smem<NT, G, XC, KB>(nx, ny);
  if (smem == 0) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  const int sms = sm_count();
  if (sms == 0) return BIGINT_ECUDA;
  const int64_t slots = (int64_t)sms * tc_per_sm<NT, G, XC, KB>(smem);
  const int64_t grid = count < slots ? count : slots;
  tcm::k_mul_tc<NT, G, XC, KB><<<(unsigned)grid, 2 * NT + 32, smem, st>>>(
      A.x, A.y, A.out, nx, ny, nout, count, A.sx, A.sy, A.so, A.lo, A.abort_flag);
  return bigint_launch_status();
}

static int launch_shape(TcShape sh, const TcArgs &A, int64_t count, int nx, int ny, int nout,
                        cudaStream_t st) {
  switch (sh) {
    case TC_64_XC: return launch_tc<64, 7, true, 128>(A, count, nx, ny, nout, st);
    case TC_64_NOXC: return launch_tc<64, 7, false, 128>(A, count, nx, ny, nout, st);
    case TC_128_XC: return launch_tc<128, 8, true, 128>(A, count, nx, ny, nout, st);
    case TC_128_NOXC: return launch_tc<128, 8, false, 128>(A, count, nx, ny, nout, st);
    case TC_N64_XC: return launch_tc<128, 15, true, 64>(A, count, nx, ny, nout, st);
    case TC_N64_NOXC: return launch_tc<128, 15, false, 64>(A, count, nx, ny, nout, st);
    case TC_N32_XC: return launch_tc<128, 12, true, 32>(A, count, nx, ny, nout, st);
    case TC_N32_NOXC: return launch_tc<128, 12, false, 32>(A, count, nx, ny, nout, st);
    default:
      return tc_smem<256, 8, true, 128>(nx, ny)
                 ? launch_tc<256, 8, true, 128>(A, count, nx, ny, nout, st)
                 : launch_tc<256, 4, true, 128>(A, count, nx, ny, nout, st);
  }
}

// Modelled tensor-core cycles of one product of a shape (x of nx, y of ny
// limbs, low nout limbs, band start lo), following tc_product's tile loop:
// each MMA of N columns costs the larger of its math (128 x N x 16 fp16
// multiply-adds at ~6750 flop/cycle per SM) and its operand reads from
// shared memory (4 KB of A plus 32 N bytes of B at 128 bytes/cycle); the
// tiles (each a fixed cost: its first Hankel build, last drain and column
// sums) count 4000 cycles.  tiles_out: the product's tiles.
static double tc_model(TcShape sh, int nx, int ny, int nout, int lo, int *tiles_out = nullptr) {
  const ShapeInfo &I = SHAPES[sh];
  const int KB = I.kb, S = 128 / KB, R = KB / 8, NT = I.nt;
  const int mx = (8 * nx + (I.xc ? 1 : 0) + KB - 1) / KB, ey = (8 * ny + KB - 1) / 128;
  const int ctot = mx + S * ey + S - 1;
  const int cfirst = lo > 0 ? (lo / R - (S - 1) > 0 ? lo / R - (S - 1) : 0) : 0;
  double cyc = 0;
  int tiles = 0;
  for (int c0 = cfirst; R * c0 < nout; c0 += NT) {
    int W = ctot - c0;
    if (W > NT) W = NT;
    const int need = (nout - R * c0 + R - 1) / R;
    if (W > need) W = need;
    W = (W + 15) & ~15;
    if (R * (c0 + W) <= lo) continue;
    tiles++;
    const int e_lo = c0 - mx + 1 > 0 ? (c0 - mx + S) / S : 0;
    const int e_hi = (c0 + W - 1) / S < ey ? (c0 + W - 1) / S : ey;
    for (int e = e_lo; e <= e_hi; e++) {
      const int ca = (c0 > S * e ? c0 : S * e) - c0, cb = (c0 + W < S * e + mx ? c0 + W : S * e + mx) - c0;
      const int N = ((cb + 15) & ~15) - (ca & ~15);
      const double math = 4096.0 * N / 6750.0, rd = 32.0 + N / 4.0;
      cyc += (KB / 16) * (math > rd ? math : rd);
    }
  }
  if (tiles_out) *tiles_out = tiles;
  return cyc + 4000.0 * tiles;
}

// Whether a shape computes the product at all: the 64- and 128-column tiles
// of 128-digit blocks take products whose columns fit one tile; the others
// any number of tiles.
static bool shape_applies(TcShape sh, int nx, int ny, int nout, int lo) {
  const ShapeInfo &I = SHAPES[sh];
  if (I.kb != 128 || I.nt == 256) return true;
  int tiles = 0;
  tc_model(sh, nx, ny, nout, lo, &tiles);
  return tiles <= 1;
}

// Modelled time of a product on one SM: tensor-core cycles, shared by the
// CTAs resident on it; with one CTA per SM the setup, first Hankel build,
// last drains and column sums of each product do not overlap another CTA's
// MMAs, which the model charges as 15 % more.
static double shape_cost(TcShape sh, int nx, int ny, int nout, int lo) {
  if (!shape_applies(sh, nx, ny, nout, lo)) return -1;
  const size_t smem = shape_smem(sh, nx, ny);
  if (smem == 0) return -1;
  int per_sm = 1;
  switch (sh) {
    case TC_64_XC: per_sm = tc_per_sm<64, 7, true, 128>(smem); break;
    case TC_64_NOXC: per_sm = tc_per_sm<64, 7, false, 128>(smem); break;
    case TC_128_XC: per_sm = tc_per_sm<128, 8, true, 128>(smem); break;
    case TC_128_NOXC: per_sm = tc_per_sm<128, 8, false, 128>(smem); break;
    case TC_N64_XC: per_sm = tc_per_sm<128, 15, true, 64>(smem); break;
    case TC_N64_NOXC: per_sm = tc_per_sm<128, 15, false, 64>(smem); break;
    case TC_N32_XC: per_sm = tc_per_sm<128, 12, true, 32>(smem); break;
    case TC_N32_NOXC: per_sm = tc_per_sm<128, 12, false, 32>(smem); break;
    default: per_sm = 1;
  }
  const double c = tc_model(sh, nx, ny, nout, lo);
  return per_sm > 1 ? c : 1.15 * c;
}

// The cheapest shape by the model for x of nx, y of ny limbs (among those
// whose x block width is in kb_mask: bit 0 128, bit 1 64, bit 2 32, and
// whose tile is NT when nt > 0); cost_out its modelled cost.
static TcShape best_shape(int nx, int ny, int nout, int lo, int kb_mask, int nt,
                          double *cost_out) {
  TcShape best = TC_256;
  double bc = -1;
  for (int i = 0; i < TC_NSHAPES; i++) {
    const TcShape sh = (TcShape)i;
    const int kbit = SHAPES[i].kb == 128 ? 1 : (SHAPES[i].kb == 64 ? 2 : 4);
    if (!(kb_mask & kbit) || (nt > 0 && SHAPES[i].nt != nt)) continue;
    const double c = shape_cost(sh, nx, ny, nout, lo);
    if (c >= 0 && (bc < 0 || c < bc)) {
      bc = c;
      best = sh;
    }
  }
  *cost_out = bc;
  return best;
}

// force: 0 (the 128-digit-block shape by the model, below) or one of the
// autotuner's candidates -- TC_FORCE_64 / _128 / _256 (128-digit blocks,
// that tile) and TC_FORCE_N64 / _N32 (narrow blocks).  The shorter operand
// becomes x.
int launch_mul_tc_ex(const uint64_t *a, int64_t sa, const uint64_t *b, int64_t sb, uint64_t *out,
                     int64_t so, int64_t count, int na, int nb, int nout, int lo, int *abort_flag,
                     cudaStream_t st, int force) {
  TcArgs A{a, b, out, sa, sb, so, lo, abort_flag};
  int nx = na, ny = nb;
  if (nb < na) {
    A.x = b; A.y = a; A.sx = sb; A.sy = sa;
    nx = nb; ny = na;
  }
  if (nx < 1 || nx > 16383 || ny > 32768 || nout < 1 || nout > na + nb || lo < 0 || lo >= nout)
    return BIGINT_EINVAL;
  if (shape_smem(TC_256, nx, ny) == 0) return BIGINT_EINVAL;
  int kb_mask = 1, nt = 0;
  switch (force) {
    case 0: break;
    case TC_FORCE_64: kb_mask = 1; nt = 64; break;
    case TC_FORCE_128: kb_mask = 1; nt = 128; break;
    case TC_FORCE_256: kb_mask = 1; nt = 256; break;
    case TC_FORCE_N64: kb_mask = 2; break;
    case TC_FORCE_N32: kb_mask = 4; break;
    default: return BIGINT_EINVAL;
  }
  // x is the operand stored whole in shared memory (the B side), y the one
  // whose Toeplitz blocks are the A side.  Either may be the shorter: the
  // model often prefers the shorter operand as y (fewer, wider MMAs for a
  // low product whose longer operand has most of the columns), as long as
  // the longer one fits shared memory as x and in a column sum's range.
  double keep = 0, swap = -1;
  TcShape sh = best_shape(nx, ny, nout, lo, kb_mask, nt, &keep);
  if (keep < 0 && force != 0) {  // the forced shape does not take this product
    kb_mask = 1;
    nt = 0;
    sh = best_shape(nx, ny, nout, lo, kb_mask, nt, &keep);
  }
  if (nx != ny && ny <= 16383) {
    const TcShape sw = best_shape(ny, nx, nout, lo, kb_mask, nt, &swap);
    if (swap >= 0 && (keep < 0 || swap < keep)) {
      const uint64_t *tp = A.x; A.x = A.y; A.y = tp;
      const int64_t ts = A.sx; A.sx = A.sy; A.sy = ts;
      const int tn = nx; nx = ny; ny = tn;
      sh = sw;
      keep = swap;
    }
  }
  if (keep < 0) return BIGINT_EINVAL;
  return launch_shape(sh, A, count, nx, ny, nout, st);
}

int launch_mul_tc(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na,
                  int nb, int nout, cudaStream_t st, int force_nt) {
  return launch_mul_tc_ex(a, na, b, nb, out, nout, count, na, nb, nout, 0, nullptr, st, force_nt);
}

// ---- split-K products (host) --------------------------------------------------
namespace {

template <int G>
int sk_dyn_max() {
  static int dyn = -1;
  if (dyn < 0) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
      return 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, tcm::k_mul_tc_sk<256, G>) != cudaSuccess) return 0;
    const int d = optin - (int)fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(tcm::k_mul_tc_sk<256, G>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, d) != cudaSuccess)
      return 0;
    dyn = d;
  }
  return dyn;
}

int sm_count_cached() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  }
  return sms;
}

// Tiles of 256 columns of the low nout limbs of x * y (x with its carry
// digit) from the column of limb lo on, as tc_product computes them; groups
// of G blocks per tile.  Returns false if there are more than SK_MAX_TILES.
bool sk_tiles(int nx, int ny, int nout, int lo, int G, tcm::SkPlan &P, int *groups) {
  const int mx = (8 * nx + 1 + 127) / 128, ey = (8 * ny + 127) / 128, ctot = mx + ey;
  P.cfirst = lo > 0 ? lo / 16 : 0;
  P.T = 0;
  for (int c0 = P.cfirst; 16 * c0 < nout; c0 += 256) {
    if (P.T == tcm::SK_MAX_TILES) return false;
    int W = ctot - c0;
    if (W > 256) W = 256;
    const int need = (nout - 16 * c0 + 15) / 16;
    if (W > need) W = need;
    W = (W + 15) & ~15;
    const int e_lo = c0 - mx + 1 > 0 ? c0 - mx + 1 : 0, e_hi = c0 + W - 1 < ey ? c0 + W - 1 : ey;
    P.c0[P.T] = c0;
    P.W[P.T] = W;
    groups[P.T] = e_hi >= e_lo ? (e_hi - e_lo + G) / G : 0;
    P.T++;
  }
  return P.T > 0;
}

}  // namespace

// Column-sum buffer bytes of one split-K product (0: not splittable).
// (Shared memory bound as for the split products: the opt-in limit per block
// of sm_100 and sm_103 less room for the kernel's static shared memory, so
// that the size does not depend on querying a device.)
constexpr size_t SK_SMEM_CAP = 232448 - 2048;

size_t mul_sk_bytes_per_product(int na, int nb, int nout, int lo) {
  const int nx = na < nb ? na : nb, ny = na < nb ? nb : na;
  tcm::SkPlan P;
  int groups[tcm::SK_MAX_TILES];
  if (nx < 1 || nx > 16383 || ny > 32768 || nout < 1 || nout > na + nb || lo < 0 || lo >= nout)
    return 0;
  if (tcm::layout<256, 4, true>(nx, ny).total > SK_SMEM_CAP) return 0;
  if (!sk_tiles(nx, ny, nout, lo, 8, P, groups)) return 0;
  return (size_t)P.T * 256 * 128 * sizeof(int);
}

// True if the split-K form would run more units than the ordinary launch
// has CTAs busy: few products (count x tiles well below the SMs).
bool mul_sk_worth(int64_t count, int na, int nb, int nout, int lo) {
  const int nx = na < nb ? na : nb, ny = na < nb ? nb : na;
  if (nx < 256 || mul_sk_bytes_per_product(na, nb, nout, lo) == 0) return false;
  tcm::SkPlan P;
  int groups[tcm::SK_MAX_TILES];
  if (!sk_tiles(nx, ny, nout, lo, 8, P, groups)) return false;
  const int sms = sm_count_cached();
  return sms > 0 && count * P.T * 2 <= sms;
}

// The low nout limbs (from limb lo: band mode, as tc_product) of a batch of
// products, each cut into units of (tile, groups) spread over the SMs; the
// units add their column sums into `colsum` (count x
// mul_sk_bytes_per_product bytes, zeroed here), then one CTA per product
// forms the limbs.  Results are those of tc_product (bit-identical).
int launch_mul_tc_sk(const uint64_t *a, int64_t sa, const uint64_t *b, int64_t sb, uint64_t *out,
                     int64_t so, int64_t count, int na, int nb, int nout, int lo, void *colsum,
                     size_t colsum_bytes, int *abort_flag, cudaStream_t st) {
  const uint64_t *x = a, *y = b;
  int64_t sx = sa, sy = sb;
  int nx = na, ny = nb;
  if (nb < na) { x = b; y = a; sx = sb; sy = sa; nx = nb; ny = na; }
  if (count == 0) return BIGINT_OK;
  if (nx < 1 || nx > 16383 || ny > 32768 || nout < 1 || nout > na + nb || lo < 0 || lo >= nout)
    return BIGINT_EINVAL;
  const size_t per = mul_sk_bytes_per_product(na, nb, nout, lo);
  if (per == 0 || colsum == nullptr || colsum_bytes < per * (size_t)count) return BIGINT_EINVAL;
  const int sms = sm_count_cached();
  if (sms == 0) return BIGINT_ECUDA;
  int G = 8;
  size_t smem = tcm::layout<256, 8, true>(nx, ny).total;
  if (sk_dyn_max<8>() <= 0 || smem > (size_t)sk_dyn_max<8>()) {
    G = 4;
    smem = tcm::layout<256, 4, true>(nx, ny).total;
    if (sk_dyn_max<4>() <= 0 || smem > (size_t)sk_dyn_max<4>()) return BIGINT_EINVAL;
  }
  tcm::SkPlan P;
  int groups[tcm::SK_MAX_TILES];
  if (!sk_tiles(nx, ny, nout, lo, G, P, groups)) return BIGINT_EINVAL;
  // groups per unit: about one unit per SM over the whole launch (each unit
  // first stages x and its first Hankel buffer, so units are not cut finer)
  int64_t total = 0;
  for (int t = 0; t < P.T; t++) total += groups[t];
  total *= count;
  int64_t gpc = (total + sms - 1) / sms;
  if (gpc < 1) gpc = 1;
  P.gpc = (int)gpc;
  P.first[0] = 0;
  for (int t = 0; t < P.T; t++) P.first[t + 1] = P.first[t] + (int)((groups[t] + gpc - 1) / gpc);
  const int64_t units = count * P.first[P.T];
  BIGINT_CUDA_TRY(cudaMemsetAsync(colsum, 0, per * (size_t)count, st));
  const int64_t stride = (int64_t)(per / sizeof(int));
  const unsigned grid = (unsigned)(units < sms ? units : sms);
  if (G == 8)
    tcm::k_mul_tc_sk<256, 8><<<grid, 2 * 256 + 32, smem, st>>>(
        x, y, nx, ny, sx, sy, count, P, static_cast<int *>(colsum), stride, abort_flag);
  else
    tcm::k_mul_tc_sk<256, 4><<<grid, 2 * 256 + 32, smem, st>>>(
        x, y, nx, ny, sx, sy, count, P, static_cast<int *>(colsum), stride, abort_flag);
  int rc = bigint_launch_status();
  if (rc != BIGINT_OK) return rc;
  const int L0 = 16 * P.cfirst;
  tcm::k_tc_sk_finish<<<(unsigned)count, 512, 0, st>>>(static_cast<const int *>(colsum), stride,
                                                       out, so, L0, nout,
                                                       lo > 0 ? (1ull << 32) : 0ull);
  return bigint_launch_status();
}

// ---- split products ----------------------------------------------------------
int launch_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na, int nb,
               int nout, cudaStream_t st);

namespace {

constexpr int SPLIT_NT = 256, SPLIT_TILE_LIMBS = 16 * SPLIT_NT;

template <int G>
int split_dyn_max() {
  static int dyn = -1;
  if (dyn < 0) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
      return 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, tcm::k_mul_tc_split<SPLIT_NT, G>) != cudaSuccess) return 0;
    const int d = optin - (int)fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(tcm::k_mul_tc_split<SPLIT_NT, G>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, d) != cudaSuccess)
      return 0;
    dyn = d;
  }
  return dyn;
}

template <int G>
int launch_split(const uint64_t *x, const uint64_t *y, uint64_t *out, int64_t count, int nx, int ny,
                 int T, uint64_t *tile_carry, cudaStream_t st) {
  const size_t smem = tcm::layout<SPLIT_NT, G>(nx, ny).total;
  const int dyn = split_dyn_max<G>();
  if (dyn <= 0 || smem > (size_t)dyn) return BIGINT_EINVAL;
  int dev = 0, sms = 0;
  BIGINT_CUDA_TRY(cudaGetDevice(&dev));
  BIGINT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t units = count * T, grid = units < sms ? units : sms;
  const int nout = nx + ny;
  tcm::k_mul_tc_split<SPLIT_NT, G><<<(unsigned)grid, 2 * SPLIT_NT + 32, smem, st>>>(
      x, y, out, nx, ny, nout, count, T, tile_carry);
  int rc = bigint_launch_status();
  if (rc != BIGINT_OK) return rc;
  tcm::k_tc_split_finish<<<(unsigned)count, 512, 0, st>>>(out, nout, T, SPLIT_TILE_LIMBS,
                                                         tile_carry);
  return bigint_launch_status();
}

// Shared memory a split CTA may take (the opt-in limit per block of sm_100
// and sm_103, less room for the kernel's static shared memory).
constexpr size_t SPLIT_SMEM_CAP = 232448 - 2048;

// Tiles of an nx x ny split product, or 0 if it does not run split (columns
// of 128 digits that fit a 128-column tile, x too large for shared memory,
// or a single tile).
int split_tiles(int nx, int ny) {
  if (nx < 1 || ny > 16383 || (8 * nx + 127) / 128 + (8 * ny + 127) / 128 <= 128) return 0;
  if (tcm::layout<SPLIT_NT, 4>(nx, ny).total > SPLIT_SMEM_CAP) return 0;
  const int T = (nx + ny + SPLIT_TILE_LIMBS - 1) / SPLIT_TILE_LIMBS;
  return T >= 2 ? T : 0;
}

}  // namespace

// Batches of at most this many products take the split-K form in
// bigint_mul_split (its column-sum buffers grow with the batch).
constexpr int64_t SPLIT_SK_MAX_COUNT = 16;

size_t mul_split_workspace(int64_t count, int na, int nb) {
  const int nx = na < nb ? na : nb, ny = na < nb ? nb : na;
  const size_t tiles = (size_t)16 * (size_t)count * (size_t)split_tiles(nx, ny);
  if (count > SPLIT_SK_MAX_COUNT || nx < 256) return tiles;
  const size_t sk = (size_t)count * mul_sk_bytes_per_product(na, nb, na + nb, 0);
  return sk > tiles ? sk : tiles;
}

// The full products of launch_mul spread over CTAs: up to SPLIT_SK_MAX_COUNT
// products in the split-K form (units of tile and groups, about one per SM),
// larger batches with each product's tiles on different CTAs (split_tiles),
// and launch_mul itself where the product has one tile or another shape.
int launch_mul_split(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na,
                     int nb, void *ws, size_t bytes, cudaStream_t st) {
  const size_t need = count > 0 ? mul_split_workspace(count, na, nb) : 0;
  if (need == 0) return launch_mul(a, b, out, count, na, nb, na + nb, st);
  if (bytes < need) return BIGINT_ENOMEM;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % 8) != 0) return BIGINT_EINVAL;
  // a few products: each cut into (tile, groups) units over the SMs
  if (count <= SPLIT_SK_MAX_COUNT && mul_sk_worth(count, na, nb, na + nb, 0))
    return launch_mul_tc_sk(a, na, b, nb, out, na + nb, count, na, nb, na + nb, 0, ws, bytes,
                            nullptr, st);
  const uint64_t *x = a, *y = b;
  int nx = na, ny = nb;
  if (nb < na) { x = b; y = a; nx = nb; ny = na; }
  const int T = split_tiles(nx, ny);
  if (T == 0) return launch_mul(a, b, out, count, na, nb, na + nb, st);
  uint64_t *tcarry = static_cast<uint64_t *>(ws);
  const size_t s8 = tcm::layout<SPLIT_NT, 8>(nx, ny).total;
  const size_t s4 = tcm::layout<SPLIT_NT, 4>(nx, ny).total;
  if (split_dyn_max<8>() > 0 && s8 <= (size_t)split_dyn_max<8>())
    return launch_split<8>(x, y, out, count, nx, ny, T, tcarry, st);
  if (split_dyn_max<4>() > 0 && s4 <= (size_t)split_dyn_max<4>())
    return launch_split<4>(x, y, out, count, nx, ny, T, tcarry, st);
  return launch_mul(a, b, out, count, na, nb, na + nb, st);
}

// BIGINT_ETIMEOUT if a tensor-core product hit a wait limit since the last
// call (synchronises the device), else BIGINT_OK.
int tc_take_timeout() { return tcm::take_timeout_here(); }
int tc_set_wait_limit(long long cycles) { return tcm::set_wait_limit_here(cycles); }

}  // namespace bigint
