// addsub.cu -- batched addition and subtraction (Sec. V-A, Figs. 3 and 4).
//
// One CTA per instance.  The CTA's W warps split the instance into W
// contiguous segments per "super-round"; within its segment a warp reads R
// rounds of 32 lanes x LPL limbs with coalesced 16-byte loads, straight into
// registers (step A1: no shared-memory staging is needed because each limb
// is used by exactly one lane).
//
// Carry propagation (step A2) is the exclusive (generate, propagate) scan of
// Fig. 3 evaluated in three levels:
//   lane   -- each lane folds its LPL limbs sequentially (Fig. 4, f1),
//   warp   -- two ballots per round resolve the carries of 32 lanes
//             (WarpCarry in common.cuh), and the rounds are folded in order,
//   block  -- warp aggregates go through shared memory and are resolved by
//             the same two-ballot trick (Fig. 4, the scan of carry_thds);
// then each lane applies its carry-in and ripples it through its limbs
// (Fig. 4, f2).  Subtraction is the same scan with generate = (a < b) and
// propagate = (a == b), applied as a borrow.
//
// HBM traffic is the algorithmic minimum: 2 limbs read and 1 written per
// limb position (Table I's 3 x NumInsts x NumBits / 8 bytes).
#include "common.cuh"

namespace bigint {

template <bool SUB, int LPL, int R>
__global__ void __launch_bounds__(1024)
    k_addsub(const uint64_t *__restrict__ A, const uint64_t *__restrict__ Bv,
             uint64_t *__restrict__ Out, uint8_t *__restrict__ carry_out, int n) {
  constexpr int SEG = 32 * LPL * R;  // limbs per warp per super-round
  __shared__ uint32_t s_g[32], s_p[32];

  const int64_t inst = blockIdx.x;
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const uint64_t *a = A + inst * (int64_t)n;
  const uint64_t *b = Bv + inst * (int64_t)n;
  uint64_t *out = Out + inst * (int64_t)n;

  uint32_t cin_block = 0;  // carry into the current super-round
  for (int base = 0; base < n; base += SEG * nwarps) {
    const int wbase = base + warp * SEG;
    uint64_t av[R][LPL], bv[R][LPL];
    // ---- A1: all loads of this super-round first (memory-level parallelism)
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int j = wbase + r * 32 * LPL + (int)lane * LPL;
      if constexpr (LPL == 2) {
        if (j + 1 < n) {
          ulonglong2 x = ld_stream2(a + j), y = ld_stream2(b + j);
          av[r][0] = x.x; av[r][1] = x.y; bv[r][0] = y.x; bv[r][1] = y.y;
        } else {
          av[r][0] = j < n ? a[j] : 0; av[r][1] = 0;
          bv[r][0] = j < n ? b[j] : 0; bv[r][1] = 0;
        }
      } else {
        av[r][0] = j < n ? __ldcs(a + j) : 0;
        bv[r][0] = j < n ? __ldcs(b + j) : 0;
      }
    }
    // ---- A2 level 1: per-limb sums and the lane's (g, p) per round
    uint64_t s[R][LPL];
    uint32_t gbits = 0, pbits = 0;  // per-limb generate/propagate, bit r*LPL+l
    WarpCarry wc[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
      uint32_t g = 0, p = 1;
#pragma unroll
      for (int l = 0; l < LPL; l++) {
        uint64_t x = av[r][l], y = bv[r][l];
        uint64_t t = SUB ? x - y : x + y;
        // positions past the end pass carries through, so the carry out of
        // the last real limb reaches the end of the warp and of the block
        const bool in = wbase + r * 32 * LPL + (int)lane * LPL + l < n;
        uint32_t gl = in && (SUB ? (x < y) : (t < x));
        uint32_t pl = !in || (SUB ? (t == 0) : (t == ~0ull));
        s[r][l] = t;
        gbits |= gl << (r * LPL + l);
        pbits |= pl << (r * LPL + l);
        g = gl | (pl & g);  // limb l is more significant than the fold so far
        p = p & pl;
      }
      wc[r] = warp_gp(g, p);
    }
    // ---- A2 level 2: fold the rounds into the warp's (g, p)
    uint32_t wg = 0, wp = 1;
#pragma unroll
    for (int r = 0; r < R; r++) {
      wg = warp_carry_out(wc[r], 0) | (warp_all_propagate(wc[r]) & wg);
      wp = wp & warp_all_propagate(wc[r]);
    }
    if (lane == 0) { s_g[warp] = wg; s_p[warp] = wp; }
    __syncthreads();
    // ---- A2 level 3: resolve the warps of the block
    const uint32_t gw = (int)lane < nwarps ? s_g[lane] : 0;
    const uint32_t pw = (int)lane < nwarps ? s_p[lane] : 0;
    const uint64_t cm = warp_carries(warp_gp(gw, pw), cin_block);
    uint32_t c = (uint32_t)(cm >> warp) & 1u;
    const uint32_t cout_block = (uint32_t)(cm >> nwarps) & 1u;
    // ---- apply the carries (Fig. 4, f2) and store
#pragma unroll
    for (int r = 0; r < R; r++) {
      const uint64_t lc = warp_carries(wc[r], c);
      uint32_t cl = (uint32_t)(lc >> lane) & 1u;
      c = (uint32_t)(lc >> 32) & 1u;
      uint64_t res[LPL];
#pragma unroll
      for (int l = 0; l < LPL; l++) {
        res[l] = SUB ? s[r][l] - cl : s[r][l] + cl;
        const uint32_t gl = (gbits >> (r * LPL + l)) & 1u;
        const uint32_t pl = (pbits >> (r * LPL + l)) & 1u;
        cl = gl | (pl & cl);
      }
      const int j = wbase + r * 32 * LPL + (int)lane * LPL;
      if constexpr (LPL == 2) {
        if (j + 1 < n) {
          st_stream2(out + j, make_ulonglong2(res[0], res[1]));
        } else if (j < n) {
          out[j] = res[0];
        }
      } else {
        if (j < n) __stcs(out + j, res[0]);
      }
    }
    cin_block = cout_block;
    __syncthreads();  // s_g / s_p are rewritten by the next super-round
  }
  if (carry_out != nullptr && threadIdx.x == 0) carry_out[inst] = (uint8_t)cin_block;
}

// Launch shape: R rounds per warp and W warps per CTA, chosen from n so that
// small instances use few rounds (more CTAs in flight) and large ones use
// up to 32 warps x 4 rounds (16 KiB of loads in flight per warp).
template <bool SUB, int LPL>
static int launch_lpl(const uint64_t *a, const uint64_t *b, uint64_t *out,
                      uint8_t *carry, int64_t count, int n, cudaStream_t st) {
  int R = n >= 4096 ? 4 : (n >= 1024 ? 2 : 1);
  int per_warp = 32 * LPL * R;
  int W = (n + per_warp - 1) / per_warp;
  if (W > 32) W = 32;
  if (W < 1) W = 1;
  dim3 grid((unsigned)count), block(32 * W);
  switch (R) {
    case 4: k_addsub<SUB, LPL, 4><<<grid, block, 0, st>>>(a, b, out, carry, n); break;
    case 2: k_addsub<SUB, LPL, 2><<<grid, block, 0, st>>>(a, b, out, carry, n); break;
    default: k_addsub<SUB, LPL, 1><<<grid, block, 0, st>>>(a, b, out, carry, n); break;
  }
  return bigint_launch_status();
}

int launch_addsub(bool sub, const uint64_t *a, const uint64_t *b, uint64_t *out,
                  uint8_t *carry, int64_t count, int n, cudaStream_t st) {
  const bool vec = (n % 2 == 0) && (((uintptr_t)a | (uintptr_t)b | (uintptr_t)out) % 16 == 0);
  if (sub) {
    return vec ? launch_lpl<true, 2>(a, b, out, carry, count, n, st)
               : launch_lpl<true, 1>(a, b, out, carry, count, n, st);
  }
  return vec ? launch_lpl<false, 2>(a, b, out, carry, count, n, st)
             : launch_lpl<false, 1>(a, b, out, carry, count, n, st);
}

}  // namespace bigint
