// blockops.cuh -- block-level linear operations on limb arrays.
//
// Every routine here is executed by ALL threads of a CTA together (it
// contains __syncthreads) and works for any blockDim.x that is a multiple of
// 32 (up to 1024).  They are the building blocks of the multiply's final
// addition (Sec. V-B, Fig. 5 bmulReg's baddReg) and of the division's linear
// steps (Sec. V-C, Fig. 6: baddReg', bsubReg', baddOne, prec, shift,
// nullUpToInd), which the paper pads to full precision.
#pragma once
#include "common.cuh"

namespace bigint {

// Shared scratch (32-bit words) the routines below need.
constexpr int BLK_SCRATCH_WORDS = 72;

// ---------------------------------------------------------------------------
// out(j) = x(j) + y(j) (+carry) or x(j) - y(j) (-borrow), j in [0, n), in
// limb order, with the carry/borrow scan of Fig. 3.  `load(j)` returns the
// pair (x_j, y_j); `store(j, r)` writes the result.  Warps take contiguous
// segments of R*32 limbs (one limb per lane per round); successive
// super-rounds hand their carry on through shared memory.  Returns the carry
// (borrow) out of limb n-1.  load() may read what store() wrote earlier only
// for the same j.
// ---------------------------------------------------------------------------
template <bool SUB, class Load, class Store>
__device__ uint32_t blk_addsub(int n, uint32_t cin, Load load, Store store, uint32_t *sm) {
  constexpr int R = 4;
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  uint32_t *s_g = sm, *s_p = sm + 32;
  uint32_t c_super = cin;
  for (int base = 0; base < n; base += nwarps * R * 32) {
    const int wb = base + warp * R * 32;
    uint64_t s[R];
    uint32_t gb = 0, pb = 0;
    WarpCarry wc[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int j = wb + r * 32 + (int)lane;
      uint32_t g = 0, p = 1;  // past the end: pass carries through
      s[r] = 0;
      if (j < n) {
        const ulonglong2 xy = load(j);
        const uint64_t t = SUB ? xy.x - xy.y : xy.x + xy.y;
        g = SUB ? (xy.x < xy.y) : (t < xy.x);
        p = SUB ? (t == 0) : (t == ~0ull);
        s[r] = t;
      }
      gb |= g << r;
      pb |= p << r;
      wc[r] = warp_gp(g, p);
    }
    uint32_t wg = 0, wp = 1;
#pragma unroll
    for (int r = 0; r < R; r++) {
      wg = warp_carry_out(wc[r], 0) | (warp_all_propagate(wc[r]) & wg);
      wp &= warp_all_propagate(wc[r]);
    }
    if (lane == 0) { s_g[warp] = wg; s_p[warp] = wp; }
    __syncthreads();
    const uint32_t gw = (int)lane < nwarps ? s_g[lane] : 0;
    const uint32_t pw = (int)lane < nwarps ? s_p[lane] : 1;
    const uint64_t cm = warp_carries(warp_gp(gw, pw), c_super);
    uint32_t c = (uint32_t)(cm >> warp) & 1u;
    const uint32_t cout = (uint32_t)(cm >> nwarps) & 1u;
#pragma unroll
    for (int r = 0; r < R; r++) {
      const uint64_t lc = warp_carries(wc[r], c);
      const uint32_t cl = (uint32_t)(lc >> lane) & 1u;
      c = (uint32_t)(lc >> 32) & 1u;
      const int j = wb + r * 32 + (int)lane;
      if (j < n) store(j, SUB ? s[r] - cl : s[r] + cl);
    }
    c_super = cout;
    __syncthreads();
  }
  return c_super;
}

// ---------------------------------------------------------------------------
// r_j = (x_j + y_j + carry) - z_j - borrow, j in [0, n), in one pass over the
// data: blk_addsub's carry scan for the sum, then the same scan as a borrow
// chain for the difference on the sums held in registers.  `load(j)` gives
// (x_j, y_j), `sub(j)` z_j.  *c / *b carry the carry / borrow in and out
// (out of limb n - 1), so a long operand can be processed in pieces.
// ---------------------------------------------------------------------------
template <class Load, class Sub, class Store>
__device__ void blk_add_then_sub(int n, uint32_t *c, uint32_t *b, Load load, Sub sub, Store store,
                                 uint32_t *sm) {
  constexpr int R = 4;
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  uint32_t *s_g = sm, *s_p = sm + 32;
  uint32_t c_super = *c, b_super = *b;
  // carry (borrow) into this warp's segment and out of the block from the
  // per-warp (generate, propagate) of wc[]
  auto resolve = [&](const WarpCarry (&wc)[R], uint32_t cin, uint32_t *cw, uint32_t *cout) {
    uint32_t wg = 0, wp = 1;
#pragma unroll
    for (int r = 0; r < R; r++) {
      wg = warp_carry_out(wc[r], 0) | (warp_all_propagate(wc[r]) & wg);
      wp &= warp_all_propagate(wc[r]);
    }
    if (lane == 0) { s_g[warp] = wg; s_p[warp] = wp; }
    __syncthreads();
    const uint32_t gw = (int)lane < nwarps ? s_g[lane] : 0;
    const uint32_t pw = (int)lane < nwarps ? s_p[lane] : 1;
    const uint64_t cm = warp_carries(warp_gp(gw, pw), cin);
    *cw = (uint32_t)(cm >> warp) & 1u;
    *cout = (uint32_t)(cm >> nwarps) & 1u;
    __syncthreads();  // s_g, s_p are reused
  };
  for (int base = 0; base < n; base += nwarps * R * 32) {
    const int wb = base + warp * R * 32;
    uint64_t s[R];
    WarpCarry wc[R];
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int j = wb + r * 32 + (int)lane;
      uint32_t g = 0, p = 1;
      s[r] = 0;
      if (j < n) {
        const ulonglong2 xy = load(j);
        const uint64_t t = xy.x + xy.y;
        g = t < xy.x;
        p = t == ~0ull;
        s[r] = t;
      }
      wc[r] = warp_gp(g, p);
    }
    uint32_t cw, cout;
    resolve(wc, c_super, &cw, &cout);
#pragma unroll
    for (int r = 0; r < R; r++) {
      const uint64_t lc = warp_carries(wc[r], cw);
      s[r] += (lc >> lane) & 1u;
      cw = (uint32_t)(lc >> 32) & 1u;
    }
    c_super = cout;
#pragma unroll
    for (int r = 0; r < R; r++) {
      const int j = wb + r * 32 + (int)lane;
      uint32_t g = 0, p = 1;
      if (j < n) {
        const uint64_t z = sub(j), t = s[r] - z;
        g = s[r] < z;
        p = t == 0;
        s[r] = t;
      }
      wc[r] = warp_gp(g, p);
    }
    uint32_t bw, bout;
    resolve(wc, b_super, &bw, &bout);
#pragma unroll
    for (int r = 0; r < R; r++) {
      const uint64_t lb = warp_carries(wc[r], bw);
      const uint32_t bl = (uint32_t)(lb >> lane) & 1u;
      bw = (uint32_t)(lb >> 32) & 1u;
      const int j = wb + r * 32 + (int)lane;
      if (j < n) store(j, s[r] - bl);
    }
    b_super = bout;
  }
  *c = c_super;
  *b = b_super;
}

// ---------------------------------------------------------------------------
// Block-wide maximum of one int per thread (all threads get the result).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int blk_max(int v, uint32_t *sm) {
  const uint32_t lane = lane_id();
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  v = __reduce_max_sync(FULL, v);
  int *s = reinterpret_cast<int *>(sm);
  if (lane == 0) s[warp] = v;
  __syncthreads();
  int w = (int)lane < nwarps ? s[lane] : INT32_MIN;
  w = __reduce_max_sync(FULL, w);
  __syncthreads();
  return w;
}

// Precision of x[0..n): index of the highest nonzero limb plus one, 0 for
// zero (Fig. 6 prec; a block max-reduction instead of atomics).
__device__ __forceinline__ int blk_prec(const uint64_t *x, int n, uint32_t *sm) {
  int p = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    if (x[j] != 0) p = j + 1;
  return blk_max(p, sm);
}

// dst[0..n) = src[0..n)  (no overlap).
__device__ __forceinline__ void blk_copy(uint64_t *dst, const uint64_t *src, int n) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) dst[j] = src[j];
}

__device__ __forceinline__ void blk_zero(uint64_t *dst, int n) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) dst[j] = 0;
}

// 1 if any of x[0..n) is nonzero (Fig. 6 nullUpToInd, negated).
__device__ __forceinline__ int blk_any_nonzero(const uint64_t *x, int n, uint32_t *sm) {
  int f = 0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) f |= (x[j] != 0);
  return blk_max(f, sm);
}

// Three-way comparison of x[0..n) and y[0..n): -1, 0, +1.
__device__ __forceinline__ int blk_cmp(const uint64_t *x, const uint64_t *y, int n,
                                       uint32_t *sm) {
  int top = 0;  // highest differing index + 1
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    if (x[j] != y[j]) top = j + 1;
  top = blk_max(top, sm);
  if (top == 0) return 0;
  return x[top - 1] > y[top - 1] ? 1 : -1;
}

// ---------------------------------------------------------------------------
// One warp per instance.  warp_addsub: r = x +- y (+- cin) over n limbs in
// rounds of 32, the carry of each round from two ballots (the scan of Fig.
// 3, as blk_addsub does across a CTA).  Every lane of the warp calls it.
// ---------------------------------------------------------------------------
template <bool SUB, class Load, class Store>
__device__ __forceinline__ void warp_addsub(int n, uint32_t cin, Load load, Store store) {
  const uint32_t lane = lane_id();
  uint32_t c = cin;
  for (int base = 0; base < n; base += 32) {
    const int j = base + (int)lane;
    uint32_t g = 0, pr = 1;
    uint64_t t = 0;
    if (j < n) {
      const ulonglong2 xy = load(j);
      t = SUB ? xy.x - xy.y : xy.x + xy.y;
      g = SUB ? (xy.x < xy.y) : (t < xy.x);
      pr = SUB ? (t == 0) : (t == ~0ull);
    }
    const uint64_t cm = warp_carries(warp_gp(g, pr), c);
    const uint32_t cl = (uint32_t)(cm >> lane) & 1u;
    if (j < n) store(j, SUB ? t - cl : t + cl);
    c = (uint32_t)(cm >> 32) & 1u;
  }
}

// out[0..nout) = low nout limbs of x y (x, y, out in shared memory, cs
// room for nout columns of 3 words), by one warp: each lane forms whole
// columns of the schoolbook product (column j = sum_i x_i y_(j-i), 128-bit
// limb products summed into lo + hi B + top B^2, two partial sums in
// flight), then the columns' words are added as three shifted numbers --
// lo, hi one limb up, top two limbs up -- with the warp carry scan.
__device__ __forceinline__ void warp_mul(const uint64_t *x, int nx, const uint64_t *y, int ny,
                                         uint64_t *out, int nout, uint64_t *cs) {
  const int lane = (int)lane_id();
  for (int j = lane; j < nout; j += 32) {
    uint64_t lo0 = 0, hi0 = 0, top0 = 0, lo1 = 0, hi1 = 0, top1 = 0;
    const int i0 = j - ny + 1 > 0 ? j - ny + 1 : 0, i1 = j < nx - 1 ? j : nx - 1;
    int i = i0;
    for (; i + 1 <= i1; i += 2) {
      const uint64_t p0 = x[i], q0 = y[j - i], p1 = x[i + 1], q1 = y[j - i - 1];
      const uint64_t l0 = p0 * q0, h0 = __umul64hi(p0, q0);
      const uint64_t l1 = p1 * q1, h1 = __umul64hi(p1, q1);
      lo0 += l0;
      const uint64_t u0 = h0 + (lo0 < l0);  // h <= 2^64 - 2: no overflow
      hi0 += u0;
      top0 += hi0 < u0;
      lo1 += l1;
      const uint64_t u1 = h1 + (lo1 < l1);
      hi1 += u1;
      top1 += hi1 < u1;
    }
    if (i <= i1) {
      const uint64_t p = x[i], q = y[j - i];
      const uint64_t l = p * q, h = __umul64hi(p, q);
      lo0 += l;
      const uint64_t u = h + (lo0 < l);
      hi0 += u;
      top0 += hi0 < u;
    }
    lo0 += lo1;
    const uint64_t u = hi1 + (lo0 < lo1);
    const uint64_t carry_u = u < hi1;  // hi1 + 1 overflowed
    hi0 += u;
    top0 += top1 + carry_u + (hi0 < u);
    cs[3 * j] = lo0;
    cs[3 * j + 1] = hi0;
    cs[3 * j + 2] = top0;
  }
  __syncwarp();
  // lo + hi B (each column's hi one limb up), into the lo words
  warp_addsub<false>(nout, 0u,
                     [&](int j) { return make_ulonglong2(cs[3 * j], j >= 1 ? cs[3 * j - 2] : 0ull); },
                     [&](int j, uint64_t v) { cs[3 * j] = v; });
  __syncwarp();
  // + top B^2
  warp_addsub<false>(nout, 0u,
                     [&](int j) { return make_ulonglong2(cs[3 * j], j >= 2 ? cs[3 * j - 4] : 0ull); },
                     [&](int j, uint64_t v) { out[j] = v; });
  __syncwarp();
}

}  // namespace bigint
