// divcore.cuh -- device-side building blocks of the shifted-inverse division
// (Sec. V-C, Fig. 6), shared by the uniform-batch kernel (divmod.cu) and the
// ragged mixed-op batch kernel (batch.cu).  The algorithm and its reading of
// the paper are described at the top of divmod.cu.
#pragma once
#include "blockops.cuh"
#include "mulcore.cuh"
#include "tccore.cuh"

namespace bigint {
namespace divc {
namespace {  // internal linkage: this header is included by several units

// Product variants used inside division: DRB/DQ/DF for large operands,
// SRB/SQ/SF below DIV_SMALL_LIMBS (measured faster there on GB300).
constexpr int DRB = 29, DQ = 16, DF = 32;
constexpr int SRB = 28, SQ = 8, SF = 128;
// (measured, 2n/n divisions: tensor-core kernel 10.9 / 6.9 / 7.5 ms against
// integer products 5.6 / 7.9 / 12.8 ms at nu = 1024 x 4096, 1536 x 2048,
// 2048 x 2048 instances)
constexpr int DIV_SMALL_LIMBS = 1536;
constexpr int MAX_CORRECTIONS = 8;
// Products whose shorter operand has at least this many limbs run on the
// tensor cores in the division kernels that hold tensor memory (TC = true).
constexpr int TC_DIV_MIN = 256;

// ---------------------------------------------------------------------------
// One-thread long division for the Newton start value (tiny operands:
// u <= 7 limbs, v <= 5 limbs).  Knuth's Algorithm D with 64-bit digits and
// 128-bit intermediates.  q[0 .. nu-nv] receives floor(u / v); v[nv-1] != 0.
// ---------------------------------------------------------------------------
__device__ void small_div(const uint64_t *u, int nu, const uint64_t *v, int nv, uint64_t *q) {
  typedef unsigned __int128 u128;
  for (int j = 0; j <= nu - nv; j++) q[j] = 0;
  if (nu < nv) return;
  if (nv == 1) {
    u128 rem = 0;
    for (int i = nu - 1; i >= 0; i--) {
      const u128 cur = (rem << 64) | u[i];
      q[i] = (uint64_t)(cur / v[0]);
      rem = cur % v[0];
    }
    return;
  }
  uint64_t vn[5], un[8];
  const int s = __clzll(v[nv - 1]);
  for (int i = nv - 1; i > 0; i--) vn[i] = (v[i] << s) | (s ? v[i - 1] >> (64 - s) : 0);
  vn[0] = v[0] << s;
  un[nu] = s ? u[nu - 1] >> (64 - s) : 0;
  for (int i = nu - 1; i > 0; i--) un[i] = (u[i] << s) | (s ? u[i - 1] >> (64 - s) : 0);
  un[0] = u[0] << s;
  const u128 B = (u128)1 << 64;
  for (int j = nu - nv; j >= 0; j--) {
    const u128 num = ((u128)un[j + nv] << 64) | un[j + nv - 1];
    u128 qh = num / vn[nv - 1];
    u128 rh = num % vn[nv - 1];
    while (qh >= B || qh * vn[nv - 2] > ((rh << 64) | un[j + nv - 2])) {
      qh--;
      rh += vn[nv - 1];
      if (rh >= B) break;
    }
    u128 borrow = 0, carry = 0;
    for (int i = 0; i < nv; i++) {
      const u128 p = qh * vn[i] + carry;
      carry = p >> 64;
      const u128 t = (u128)un[i + j] - (uint64_t)p - borrow;
      un[i + j] = (uint64_t)t;
      borrow = (t >> 64) ? 1 : 0;
    }
    const u128 t = (u128)un[j + nv] - carry - borrow;
    un[j + nv] = (uint64_t)t;
    if (t >> 64) {  // estimate one too large: add back
      qh--;
      u128 c = 0;
      for (int i = 0; i < nv; i++) {
        const u128 s2 = (u128)un[i + j] + vn[i] + c;
        un[i + j] = (uint64_t)s2;
        c = s2 >> 64;
      }
      un[j + nv] += (uint64_t)c;
    }
    q[j] = (uint64_t)qh;
  }
}

// Per-instance workspace, in limbs.
struct Work {
  uint64_t *w, *wn, *p, *d, *qh, *r, *tmp;
  int cap_w, cap_p, cap_d;
};

__host__ __device__ inline int ws_cap_w(int nu, int nv, int h) {
  const int H = nu > h ? nu : h;
  return H + 8;
}
__host__ __device__ inline int ws_cap_p(int nu, int nv, int h) {
  const int H = nu > h ? nu : h;
  return 2 * H + nv + 16;
}
__host__ __device__ inline int ws_cap_d(int nu, int nv, int h) {
  const int H = nu > h ? nu : h;
  return H + nv + 16;
}
// limbs per instance (rounded to 32 limbs = 256 bytes)
__host__ __device__ inline int64_t ws_limbs(int nu, int nv, int h) {
  const int64_t t = 4 * (int64_t)ws_cap_w(nu, nv, h) + 2 * (int64_t)ws_cap_p(nu, nv, h) +
                    ws_cap_d(nu, nv, h) + (nv + 8);
  return (t + 31) / 32 * 32;
}

__device__ Work carve(uint64_t *base, int nu, int nv, int h) {
  Work W;
  W.cap_w = ws_cap_w(nu, nv, h);
  W.cap_p = ws_cap_p(nu, nv, h);
  W.cap_d = ws_cap_d(nu, nv, h);
  uint64_t *p = base;
  W.w = p; p += W.cap_w;
  W.wn = p; p += W.cap_w;
  W.qh = p; p += W.cap_w;
  W.p = p; p += W.cap_p;
  W.tmp = p; p += W.cap_p;
  W.d = p; p += W.cap_d;
  W.r = p; p += W.cap_w;
  return W;
}

// ---------------------------------------------------------------------------
// Tensor-core product inside a kernel of tcm::TC_CTA_THREADS threads holding
// 512 TMEM columns (tccore.cuh; the last warp issues the MMAs), as one
// out-of-line copy.
// ---------------------------------------------------------------------------
template <int G>
__device__ __noinline__ bool tc_call(tcm::TcCtx *c, const uint64_t *x, int nx, const uint64_t *y,
                                     int ny, uint64_t *out, int nout, int lo) {
  return tcm::tc_product<256, G, true>(*c, x, nx, y, ny, out, nout, lo);
}

// out[0..nout) = x * y on the tensor cores when the shorter operand has
// TC_DIV_MIN limbs and the product's layout fits smem_words; false (nothing
// written) otherwise.  With lo > 0 the tensor-core band semantics apply
// (tc_product): limbs >= lo + 2 are exact or one unit of limb lo + 2 high,
// limbs below the first computed tile are not written.
// Toeplitz blocks the 256-column tiles of x * y (x of nx limbs with its
// carry digit) issue for the limbs [lo, nout), as tc_product's tile loop.
__device__ __forceinline__ int tc_blocks256(int nx, int ny, int nout, int lo) {
  const int mx = (8 * nx + 1 + 127) / 128, ey = (8 * ny + 127) / 128, ctot = mx + ey;
  int blocks = 0;
  for (int c0 = lo > 0 ? lo / 16 : 0; 16 * c0 < nout; c0 += 256) {
    int W = ctot - c0 < 256 ? ctot - c0 : 256;
    const int need = (nout - 16 * c0 + 15) / 16;
    if (W > need) W = need;
    W = (W + 15) & ~15;
    const int e_lo = c0 - mx + 1 > 0 ? c0 - mx + 1 : 0, e_hi = c0 + W - 1 < ey ? c0 + W - 1 : ey;
    if (e_hi >= e_lo) blocks += e_hi - e_lo + 1;
  }
  return blocks;
}

__device__ __forceinline__ bool tc_mul(tcm::TcCtx *tc, const uint64_t *x, int nx,
                                       const uint64_t *y, int ny, uint64_t *out, int nout,
                                       int smem_words, int lo) {
  int ns = nx < ny ? nx : ny, nl = nx < ny ? ny : nx;
  if (tc == nullptr || tc->aborted || ns < TC_DIV_MIN) return false;
  const uint64_t *xs = nx <= ny ? x : y, *ys = nx <= ny ? y : x;
  const int no = nout < nx + ny ? nout : nx + ny;
  const uint32_t bytes = 4u * (uint32_t)smem_words;
  // the shorter operand as the Toeplitz side (y) where that issues fewer
  // MMAs (a low product whose longer operand has most of the columns: an
  // MMA narrower than ~136 columns costs its A operand's read, so fewer,
  // wider MMAs win) and the longer one fits shared memory as x
  if (ns != nl && tcm::layout<256, 4>(nl, ns).total <= bytes &&
      tc_blocks256(nl, ns, no, lo) < tc_blocks256(ns, nl, no, lo)) {
    const uint64_t *t = xs; xs = ys; ys = t;
    const int tn = ns; ns = nl; nl = tn;
  }
  if (tcm::layout<256, 8>(ns, nl).total <= bytes)
    tc_call<8>(tc, xs, ns, ys, nl, out, no, lo);
  else if (tcm::layout<256, 4>(ns, nl).total <= bytes)
    tc_call<4>(tc, xs, ns, ys, nl, out, no, lo);
  else
    return false;
  for (int j = no + (int)threadIdx.x; j < nout; j += blockDim.x) out[j] = 0;
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// Product of arbitrary (limb) sizes: on the tensor cores (TC, large
// operands), else one blk_mul when both operands fit the shared-memory
// budget, otherwise a sum of slice products, each added into place (out
// must not overlap x, y or tmp).  Writes out[0..nout) (band mode: see
// blk_mul and tc_mul).
// ---------------------------------------------------------------------------
template <int RB, int Q, int F, bool TC = false>
__device__ void mul_any(const uint64_t *x, int nx, const uint64_t *y, int ny, uint64_t *out,
                        int nout, uint64_t *tmp, uint32_t *smem, int smem_words, int lo = 0,
                        tcm::TcCtx *tc = nullptr) {
  if (nx <= 0 || ny <= 0) {
    blk_zero(out, nout);
    __syncthreads();
    return;
  }
  if constexpr (TC) {
    if (tc != nullptr && tc->aborted) {
      // a tensor-core product of this CTA gave up at a wait limit: the
      // result is already void (the caller reports BIGINT_ETIMEOUT), so the
      // remaining products are zero and the division runs to its end on
      // bounded loops
      blk_zero(out, nout);
      __syncthreads();
      return;
    }
    if (tc_mul(tc, x, nx, y, ny, out, nout, smem_words, lo)) return;
  }
  if (blk_mul_smem_words<RB, Q>(nx, ny) <= smem_words) {
    blk_mul_call<RB, Q, F>(x, nx, y, ny, out, nout, smem, lo);
    return;
  }
  // slice both operands into pieces of s limbs whose products fit
  int s = 8192;
  while (s > 64 && blk_mul_smem_words<RB, Q>(s, s) > smem_words) s -= 64;
  uint32_t *scr = smem;  // blk_addsub scratch (the slice product is done)
  blk_zero(out, nout);
  __syncthreads();
  for (int i0 = 0; i0 < nx; i0 += s) {
    const int sx = nx - i0 < s ? nx - i0 : s;
    for (int j0 = 0; j0 < ny; j0 += s) {
      const int sy = ny - j0 < s ? ny - j0 : s;
      const int off = i0 + j0;
      if (off >= nout) continue;
      if (lo > 0 && off + sx + sy + 1 <= lo) continue;  // entirely below the band
      const int len = sx + sy < nout - off ? sx + sy : nout - off;
      blk_mul_call<RB, Q, F>(x + i0, sx, y + j0, sy, tmp, len, smem, lo > off ? lo - off : 0);
      const int n = nout - off;
      uint64_t *o = out + off;
      auto load = [&](int j) { return make_ulonglong2(o[j], j < len ? tmp[j] : 0ull); };
      auto store = [&](int j, uint64_t v) { o[j] = v; };
      blk_addsub<false>(n, 0u, load, store, scr);
    }
  }
}

// ---------------------------------------------------------------------------
// The Newton start value: w = floor(B^(2l) / V) with V = floor(v / B^(k-l))
// + 1 (k >= l) or V = v B^(l-k) (k < l).  Thread 0 computes, all wait.
// ---------------------------------------------------------------------------
__device__ void newton_start(const uint64_t *v, int k, int l, uint64_t *w, int cap_w) {
  if (threadIdx.x == 0) {
    uint64_t V[6] = {0, 0, 0, 0, 0, 0}, U[8] = {0, 0, 0, 0, 0, 0, 0, 0}, Qt[8];
    int nV;
    if (k >= l) {
      for (int i = 0; i <= l; i++) V[i] = v[k - l + i];
      // V + 1 (may carry into limb l+1)
      int i = 0;
      while (i <= l && ++V[i] == 0) i++;
      nV = (i > l) ? l + 2 : l + 1;
      if (i > l) V[l + 1] = 1;
    } else {
      for (int i = 0; i <= k; i++) V[l - k + i] = v[i];
      nV = l + 1;
    }
    U[2 * l] = 1;  // B^(2l)
    small_div(U, 2 * l + 1, V, nV, Qt);
    const int nq = 2 * l + 1 - nV + 1;
    for (int i = 0; i < cap_w; i++) w[i] = i < nq ? Qt[i] : 0;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// One Newton step (Fig. 6 step) with the divisor vt (nvt limbs):
//   e = hp - m;  d = B^e - vt w;  w' = w B^m +- round(w |d| / B^(hp - 2m)),
// floor for d >= 0, ceiling for d < 0.  w is in W.w (prec nw), the result
// goes to W.wn and the two buffers are swapped.  Returns prec(w').
// ---------------------------------------------------------------------------
template <int RB, int Q, int F, bool TC = false>
__device__ int newton_step(int hp, int m, const uint64_t *vt, int nvt, Work &W, int nw,
                           uint32_t *smem, int smem_words, uint32_t *scr,
                           tcm::TcCtx *tc = nullptr) {
  // d = B^e - vt w is small: |d| < 2 vt < B^(t+2) / 2 (t = nvt - 1, the
  // iterate is within two units), and e = t + l >= t + 2.  So d is fixed by
  // vt w modulo B^(t+2) -- the powDiff product "performed modulo a power of
  // the base" of Fig. 6 -- and its sign is the top bit of that residue:
  // L = (-d) mod B^(t+2) is below B^(t+2)/2 exactly when d <= 0.
  const int nl = nvt + 1;
  mul_any<RB, Q, F, TC>(vt, nvt, W.w, nw, W.p, nl, W.tmp, smem, smem_words, 0, tc);
  const bool neg = (W.p[nl - 1] >> 63) == 0;  // d <= 0: vt w >= B^e
  int nd = nl;
  {
    uint64_t *P = W.p, *D = W.d;
    auto store = [&](int j, uint64_t x) { D[j] = x; };
    if (neg) {  // |d| = L
      auto load = [&](int j) { return make_ulonglong2(P[j], 0ull); };
      blk_addsub<false>(nl, 0u, load, store, scr);
    } else {  // |d| = B^(t+2) - L
      auto load = [&](int j) { return make_ulonglong2(0ull, P[j]); };
      blk_addsub<true>(nl, 0u, load, store, scr);
    }
  }
  nd = blk_prec(W.d, nd, scr);
  // P2 = w * D ; y = P2 >> s limbs, s = hp - 2m
  const int s = hp - 2 * m;
  const int n2 = nw + nd;
  uint32_t cin = 0;
  if (nd > 0) {
    mul_any<RB, Q, F, TC>(W.w, nw, W.d, nd, W.p, n2, W.tmp, smem, smem_words, 0, tc);
    if (neg) cin = (uint32_t)blk_any_nonzero(W.p, s < n2 ? s : n2, scr);  // ceiling
  }
  const uint64_t *Y = W.p + s;
  const int ny = nd > 0 ? (n2 - s > 0 ? n2 - s : 0) : 0;
  // w' = w B^m +- (y + cin)
  const int nout = (nw + m > ny ? nw + m : ny) + 1;
  {
    const uint64_t *w = W.w;
    uint64_t *wn = W.wn;
    auto load = [&](int j) {
      const uint64_t x = (j >= m && j - m < nw) ? w[j - m] : 0ull;
      return make_ulonglong2(x, j < ny ? Y[j] : 0ull);
    };
    auto store = [&](int j, uint64_t x) { wn[j] = x; };
    if (neg) blk_addsub<true>(nout, cin, load, store, scr);
    else blk_addsub<false>(nout, 0u, load, store, scr);
  }
  uint64_t *t = W.w;
  W.w = W.wn;
  W.wn = t;
  return blk_prec(W.w, nout, scr);
}

// w ~ B^h / v (0 <= B^h/v - w < 2 before the final correction); returns
// prec(w).  v has precision k+1.
template <int RB, int Q, int F, bool TC = false>
__device__ int shinv_newton(const uint64_t *v, int k, int h, Work &W, uint32_t *smem,
                            int smem_words, uint32_t *scr, tcm::TcCtx *tc = nullptr) {
  const int L = h - k;
  int l = L < 3 ? L : 3;
  newton_start(v, k, l, W.w, W.cap_w);
  int nw = blk_prec(W.w, l + 2, scr);
  while (l < L) {
    const int m = (l - 2 < L - l) ? l - 2 : L - l;
    const int t = (k < l + m + 2) ? k : l + m + 2;
    nw = newton_step<RB, Q, F, TC>(t + l + m, m, v + (k - t), t + 1, W, nw, smem, smem_words,
                                   scr, tc);
    l += m;
  }
  return nw;
}

// R = R mod B^(kv+1) holds x - Q v for some Q in W.qh (prec nq <= cap);
// bring it into [0, v).  Returns 0 or BIGINT_EINTERNAL.
__device__ int correct(const uint64_t *v, int kv, uint64_t *R, uint64_t *Qh, int nqcap,
                       uint32_t *scr) {
  const int nr = kv + 1;
  for (int it = 0; it < 2 * MAX_CORRECTIONS; it++) {
    __syncthreads();
    const bool negative = (R[kv] >> 63) != 0;
    int dir = 0;  // +1: r -= v, q++ ; -1: r += v, q--
    if (negative) {
      dir = -1;
    } else {
      // R >= v ?  (v has kv limbs, R has kv+1)
      int top = 0;
      for (int j = threadIdx.x; j < nr; j += blockDim.x) {
        const uint64_t vj = j < kv ? v[j] : 0ull;
        if (R[j] != vj) top = j + 1;
      }
      top = blk_max(top, scr);
      if (top == 0) dir = 1;  // R == v
      else {
        const uint64_t vj = top - 1 < kv ? v[top - 1] : 0ull;
        dir = R[top - 1] > vj ? 1 : 0;
      }
    }
    if (dir == 0) return BIGINT_OK;
    {
      auto load = [&](int j) { return make_ulonglong2(R[j], j < kv ? v[j] : 0ull); };
      auto store = [&](int j, uint64_t x) { R[j] = x; };
      if (dir > 0) blk_addsub<true>(nr, 0u, load, store, scr);
      else blk_addsub<false>(nr, 0u, load, store, scr);
    }
    {
      auto load = [&](int j) { return make_ulonglong2(Qh[j], j == 0 ? 1ull : 0ull); };
      auto store = [&](int j, uint64_t x) { Qh[j] = x; };
      if (dir > 0) blk_addsub<false>(nqcap, 0u, load, store, scr);
      else blk_addsub<true>(nqcap, 0u, load, store, scr);
    }
  }
  return BIGINT_EINTERNAL;
}


// q = floor(u / v), r = u - q v from the inverse w = floor(B^h / v) (nw
// limbs) at h = ku = prec(u) >= kv = prec(v): q^ = floor(u w / B^h), from a
// product that may drop the columns below limb h - 2, is at most a few units
// low (integer product: it is never high, since w <= B^h / v) or one unit
// high (tensor-core product, whose band mode adds a margin above the dropped
// columns); the final correction absorbs either.  u w + B^h < B^(ku + nw)
// since h = ku, so the banded value never wraps.
template <int RB, int Q, int F, bool TC>
__device__ int divmod_tail(const uint64_t *u, int ku, const uint64_t *v, int kv,
                           const uint64_t *w, int nw, int h, uint64_t *q, int nq, uint64_t *r,
                           int nv, Work &W, uint32_t *smem, int smem_words, uint32_t *scr,
                           tcm::TcCtx *tc) {
  int st = BIGINT_OK;
  const int nz = ku + nw;
  mul_any<RB, Q, F, TC>(u, ku, w, nw, W.p, nz, W.tmp, smem, smem_words, h > 2 ? h - 2 : 0, tc);
  const int nqh = nz - h > 0 ? nz - h : 0;
  const int qcap = nqh + 1 < W.cap_w ? nqh + 1 : W.cap_w;
  for (int j = threadIdx.x; j < qcap; j += blockDim.x) W.qh[j] = j < nqh ? W.p[h + j] : 0;
  __syncthreads();
  const int pq = blk_prec(W.qh, qcap, scr);
  // r^ = (u - q^ v) mod B^(kv+1): the low kv+1 limbs of q^ v only
  if (pq > 0) {
    mul_any<RB, Q, F, TC>(W.qh, pq, v, kv, W.p, kv + 1, W.tmp, smem, smem_words, 0, tc);
  } else {
    blk_zero(W.p, kv + 1);
    __syncthreads();
  }
  {
    uint64_t *P = W.p, *R = W.r;
    auto load = [&](int j) { return make_ulonglong2(j < ku ? u[j] : 0ull, P[j]); };
    auto store = [&](int j, uint64_t x) { R[j] = x; };
    blk_addsub<true>(kv + 1, 0u, load, store, scr);
  }
  st = correct(v, kv, W.r, W.qh, qcap, scr);
  __syncthreads();
  const int pqf = blk_prec(W.qh, qcap, scr);
  if (pqf > nq && st == BIGINT_OK) st = BIGINT_ERANGE;
  for (int j = threadIdx.x; j < nq; j += blockDim.x) q[j] = j < qcap ? W.qh[j] : 0;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) r[j] = j < kv ? W.r[j] : 0;
  __syncthreads();
  return st;
}

// One division q = floor(u / v), r = u - q v by the whole CTA (Sec. V-C):
// the shifted inverse by Newton steps, q^ = floor(u w / B^h), r^ computed
// modulo B^(k+2), exact correction.  ws: this instance's workspace region of
// ws_limbs(nu, nv, nu) limbs.  Returns the status (0, EDIVZERO, ERANGE,
// EINTERNAL).
template <int RB, int Q, int F, bool TC = false>
__device__ int divmod_one(const uint64_t *u, int nu, const uint64_t *v, int nv, uint64_t *q,
                          int nq, uint64_t *r, uint64_t *ws, uint32_t *smem, int smem_words,
                          uint32_t *scr, tcm::TcCtx *tc = nullptr) {
  Work W = carve(ws, nu, nv, nu);
  const int kv = blk_prec(v, nv, scr);
  if (kv == 0) {  // division by zero: q = r = 0
    blk_zero(q, nq);
    blk_zero(r, nv);
    __syncthreads();
    return BIGINT_EDIVZERO;
  }
  const int k = kv - 1;
  const int ku = blk_prec(u, nu, scr);
  if (ku < kv) {  // u < B^(ku) <= B^(kv-1) <= v: q = 0, r = u
    blk_zero(q, nq);
    for (int j = threadIdx.x; j < nv; j += blockDim.x) r[j] = j < ku ? u[j] : 0;
    __syncthreads();
    return BIGINT_OK;
  }
  const int h = ku;
  int nw = shinv_newton<RB, Q, F, TC>(v, k, h, W, smem, smem_words, scr, tc);
  return divmod_tail<RB, Q, F, TC>(u, ku, v, kv, W.w, nw, h, q, nq, r, nv, W, smem, smem_words,
                                   scr, tc);
}


}  // namespace
}  // namespace divc

}  // namespace bigint
