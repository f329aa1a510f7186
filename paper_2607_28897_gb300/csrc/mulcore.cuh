// mulcore.cuh -- block-level product of two limb arrays (Sec. V-B, Fig. 5).
//
// blk_mul<RB, Q, F>(x, nx, y, ny, out, nout, smem) writes the low nout limbs
// of x*y to out (nout = nx + ny gives the full product).  All threads of the
// CTA take part.
//
// Digits.  The operands are re-cut into digits of RB < 32 bits (one digit
// per 32-bit word in shared memory).  A digit product then has 2*RB bits and
// one 32x32->64-bit multiply-add (IMAD.WIDE) accumulates it into a 64-bit
// column accumulator with no carry handling: 2^(64-2RB) products fit before
// the accumulator can overflow.  The carries are deferred: every F row steps
// each accumulator keeps its low RB bits and hands the rest to the next
// column.  This replaces the paper's oneConvMul (a 128-bit product added
// into a (low, high, carry) column triple, Sec. V-B) by one instruction per
// digit product, the cheapest integer multiply form on sm_103a.
//
// Schedule.  The shorter operand is the "row" operand (one digit a_i per
// row step, the same for every lane of a warp), the longer one the "window"
// operand (each thread keeps 2Q consecutive digits of it in registers and
// slides the window down one digit per step).  The columns are cut into
// chunks of Q; a thread owns one unit of work at a time:
//   * unit u < K_R: the balanced pair of chunk u (rising part of the column
//     profile) and chunk K_W + u (falling part), as in Fig. 5 threadConv --
//     their row counts (u+1)Q and (K_R-u)Q add up to (K_R+1)Q;
//   * unit u >= K_R: one chunk of the flat middle part, K_R Q rows (+Q
//     zero rows to keep every unit at exactly K_R+1 groups of Q steps).
// Zero padding of Q digits on both sides of the window operand (and after
// the row operand) lets the triangular ends of the chunks (Fig. 5 halfConv's
// second loop) run through the same code.
//
// Combine (Fig. 5 combineQ / manifestShm / bmulReg).  A finished chunk is Q
// normalised digits plus an overflow word X (the chunk's value above its Q
// digits).  The digits are packed into their bit positions of the output
// (limbs shared by two chunks are completed with atomicOr); the overflow
// words go to shared memory ("Hsh").  One block-wide carry-scan addition of
// the output and the overflow words finishes the product.
#pragma once
#include "blockops.cuh"
#include "common.cuh"

namespace bigint {

template <int RB>
struct Digits {
  static constexpr uint32_t MASK = (1u << RB) - 1u;
  // number of RB-bit digits of an n-limb number
  static __host__ __device__ constexpr int count(int nlimbs) { return (64 * nlimbs + RB - 1) / RB; }
  // digit k: bits [RB k, RB k + RB) of the limb array (read as 32-bit words)
  static __device__ __forceinline__ uint32_t get(const uint32_t *w, int nwords, int k) {
    const int bit = RB * k;
    const int i = bit >> 5, s = bit & 31;
    const uint32_t lo = i < nwords ? w[i] : 0u;
    const uint32_t hi = i + 1 < nwords ? w[i + 1] : 0u;
    return __funnelshift_r(lo, hi, s) & MASK;
  }
};

// Shared-memory words blk_mul needs for an nx-by-ny product.
template <int RB, int Q>
__host__ __device__ constexpr int blk_mul_smem_words(int nx, int ny) {
  const int NX = Digits<RB>::count(nx), NY = Digits<RB>::count(ny);
  const int NR = NX < NY ? NX : NY, NW = NX < NY ? NY : NX;
  const int KR = (NR + Q - 1) / Q, KW = (NW + Q - 1) / Q;
  // row [KR Q + Q] | window [-Q, KW Q + Q) | H (64-bit) [KW + KR] | scratch
  return (KR * Q + Q) + (KW * Q + 2 * Q) + 2 * (KW + KR) + BLK_SCRATCH_WORDS;
}

// Units of work (threads x rounds) for an nx-by-ny product.
template <int RB, int Q>
__host__ __device__ constexpr int blk_mul_units(int nx, int ny) {
  const int NX = Digits<RB>::count(nx), NY = Digits<RB>::count(ny);
  const int NW = NX < NY ? NY : NX;
  return (NW + Q - 1) / Q;
}

template <int RB, int Q>
__device__ __forceinline__ void normalise(uint64_t (&acc)[Q], uint64_t &X) {
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const uint64_t c = acc[q] >> RB;
    acc[q] &= Digits<RB>::MASK;
    if (q + 1 < Q) acc[q + 1] += c; else X += c;
  }
}

// Normalise, pack the Q digits of chunk c into the output bits
// [RB Q c, RB Q (c+1)) (limbs < nout), and park the overflow X in sH[c].
template <int RB, int Q>
__device__ __forceinline__ void finish_chunk(uint64_t (&acc)[Q], uint64_t X, int c,
                                             uint64_t *out, int nout, uint64_t *sH) {
  normalise<RB, Q>(acc, X);
  sH[c] = X;
  const int o = RB * Q * c;
  int limb = o >> 6, pos = o & 63;
  uint64_t cur = 0;
#pragma unroll
  for (int q = 0; q < Q; q++) {
    const uint64_t d = acc[q];
    cur |= d << pos;
    pos += RB;
    if (pos >= 64) {
      if (limb < nout && cur) atomicOr(reinterpret_cast<unsigned long long *>(out + limb), cur);
      limb++;
      pos -= 64;
      cur = pos > 0 ? d >> (RB - pos) : 0;
    }
  }
  if (pos > 0 && limb < nout && cur)
    atomicOr(reinterpret_cast<unsigned long long *>(out + limb), cur);
}

// Row steps with the window split in two register buffers (lo = digits
// [base-Q, base), hi = [base, base+Q)); the caller swaps the roles of the two
// buffers from one group to the next, so the window slides with no register
// moves at all.
template <int Q, int T0>
__device__ __forceinline__ void row_steps_pp(uint64_t (&acc)[Q], const uint32_t (&lo)[Q],
                                             const uint32_t (&hi)[Q], const uint32_t *a) {
  if constexpr (T0 < Q) {
    const uint4 av = *reinterpret_cast<const uint4 *>(a + T0);
    const uint32_t a4[4] = {av.x, av.y, av.z, av.w};
#pragma unroll
    for (int t = 0; t < 4; t++) {
#pragma unroll
      for (int q = 0; q < Q; q++) {
        constexpr int dummy = 0;
        (void)dummy;
        const int x = Q - (T0 + t) + q;  // window index in [1, 2Q)
        const uint32_t w = x < Q ? lo[x] : hi[x - Q];
        acc[q] += (uint64_t)a4[t] * (uint64_t)w;  // one IMAD.WIDE.U32
      }
    }
    row_steps_pp<Q, T0 + 4>(acc, lo, hi, a);
  }
}

template <int Q>
__device__ __forceinline__ void load_q(uint32_t (&r)[Q], const uint32_t *p) {
#pragma unroll
  for (int q = 0; q < Q; q += 4) {
    const uint4 v = *reinterpret_cast<const uint4 *>(p + q);
    r[q] = v.x; r[q + 1] = v.y; r[q + 2] = v.z; r[q + 3] = v.w;
  }
}

// conv_unit with ping-pong window buffers (see row_steps_pp).  Band limits:
// a chunk that starts at or above output bit 64 nout contributes nothing to
// out[0, nout) and is skipped (exact); with lo > 0 a chunk whose digits and
// overflow word all lie below bit 64 lo is skipped too, which drops its
// contribution -- callers that pass lo > 0 only use limbs well above lo and
// correct the result afterwards.
template <int RB, int Q, int F, bool BAND>
__device__ __forceinline__ void conv_unit_pp(int u, int KR, int KW, const uint32_t *sRow,
                                             const uint32_t *sW, uint64_t *out, int nout,
                                             uint64_t *sH, int lo) {
  static_assert(F % Q == 0, "flush interval must be a whole number of groups");
  static_assert(F < (1 << (64 - 2 * RB)), "flush interval too long for this digit size");
  constexpr int FG = F / Q;
  constexpr int64_t CB = (int64_t)RB * Q;  // bits per chunk
  const int NWp = KW * Q;
  const bool pair = u < KR;
  auto skip_chunk = [&](int c) {
    if constexpr (!BAND) return false;
    const int64_t b0 = CB * c;
    return b0 >= 64 * (int64_t)nout || b0 + CB + 64 <= 64 * (int64_t)lo;
  };
  const bool f_skip = skip_chunk(u);
  const bool m_skip = pair ? skip_chunk(KW + u) : true;
  if (f_skip && (!pair || m_skip)) return;
  const int switch_g = pair ? u + 1 : -1;
  const int g_begin = (pair && f_skip) ? u + 1 : 0;
  const int g_end = (pair && m_skip) ? u : KR;
  uint64_t acc[Q], X = 0;
  uint32_t A[Q], Bf[Q];
#pragma unroll
  for (int q = 0; q < Q; q++) acc[q] = 0;
  if (g_begin == 0) load_q<Q>(A, sW + u * Q);  // hi half of group 0
  bool fwd = g_begin == 0;
  // one group: hi/lo are the buffer roles for this group's parity
  auto group = [&](int g, uint32_t (&hi)[Q], uint32_t (&lo)[Q]) {
    if (g == switch_g) {  // low chunk done: continue with its partner
      if (!f_skip) finish_chunk<RB, Q>(acc, X, u, out, nout, sH);
#pragma unroll
      for (int q = 0; q < Q; q++) { acc[q] = 0; hi[q] = 0; }  // window[NWp..) is padding
      X = 0;
      fwd = false;
    }
    const int base = fwd ? (u - g) * Q : NWp + (u + 1 - g) * Q;
    const int i0 = fwd ? g * Q : (g - 1) * Q;
    load_q<Q>(lo, sW + base - Q);
    row_steps_pp<Q, 0>(acc, lo, hi, sRow + i0);
    if ((g + 1) % FG == 0) normalise<RB, Q>(acc, X);
  };
  // The first group of the range always takes hi = A: A holds the window's
  // high half of group 0, or is zeroed at the switch when the range starts
  // with the partner chunk.
  int g = g_begin;
#pragma unroll 1
  for (; g + 1 <= g_end; g += 2) {
    group(g, A, Bf);      // hi = A, lo = B
    group(g + 1, Bf, A);  // hi = B (the previous lo), lo = A
  }
  if (g <= g_end) group(g, A, Bf);
  if (g_end == KR) {
    if (!pair || !m_skip) finish_chunk<RB, Q>(acc, X, pair ? KW + u : u, out, nout, sH);
  } else if (!f_skip) {
    finish_chunk<RB, Q>(acc, X, u, out, nout, sH);  // partner chunk skipped
  }
}

// Low nout limbs of x[0..nx) * y[0..ny) into out[0..nout) (out must not
// overlap x or y).  With BAND, chunks at or above limb nout are skipped, and lo > 0 allows the result to miss the products of chunks
// below limb lo (see conv_unit_pp): limbs >= lo + 2 are then at most a few
// units of limb lo below the exact value.  smem: blk_mul_smem_words<RB,Q>(nx, ny) words, 16-byte
// aligned.  Returns the carry out of limb nout-1 of the final addition
// (0 whenever nout >= nx + ny).
template <int RB, int Q, int F, bool BAND = false>
__device__ uint32_t blk_mul(const uint64_t *x, int nx, const uint64_t *y, int ny, uint64_t *out,
                            int nout, uint32_t *smem, int lo = 0) {
  const int NX = Digits<RB>::count(nx), NY = Digits<RB>::count(ny);
  const bool x_is_row = NX <= NY;
  const uint32_t *rw = reinterpret_cast<const uint32_t *>(x_is_row ? x : y);
  const uint32_t *ww = reinterpret_cast<const uint32_t *>(x_is_row ? y : x);
  const int NR = x_is_row ? NX : NY, NW = x_is_row ? NY : NX;
  const int rwords = 2 * (x_is_row ? nx : ny), wwords = 2 * (x_is_row ? ny : nx);
  const int KR = (NR + Q - 1) / Q, KW = (NW + Q - 1) / Q;
  // Every region starts on a multiple of Q >= 4 words: 16-byte aligned.
  uint32_t *sRow = smem;                                             // [KR Q + Q]
  uint32_t *sW = smem + (KR * Q + Q) + Q;                            // [-Q, KW Q + Q)
  uint64_t *sH = reinterpret_cast<uint64_t *>(sW + KW * Q + Q);      // [KW + KR]
  uint32_t *scr = reinterpret_cast<uint32_t *>(sH + (KW + KR));      // scratch
  const int T = blockDim.x, t = threadIdx.x;

  // ---- A1: stage both operands as RB-bit digits, zero padded; clear out
  for (int k = t; k < KR * Q + Q; k += T) sRow[k] = k < NR ? Digits<RB>::get(rw, rwords, k) : 0u;
  for (int k = t - Q; k < KW * Q + Q; k += T) sW[k] = (k >= 0 && k < NW) ? Digits<RB>::get(ww, wwords, k) : 0u;
  for (int j = t; j < nout; j += T) out[j] = 0;
  __syncthreads();

  // ---- A3: convolution, one unit at a time per thread
  for (int u = t; u < KW; u += T) {
    conv_unit_pp<RB, Q, F, BAND>(u, KR, KW, sRow, sW, out, nout, sH, lo);
  }
  __syncthreads();

  // ---- A4: out += overflow words, one carry-scan addition
  const int CB = RB * Q;  // bits per chunk
  const int nch = KW + KR;
  auto load = [&](int j) -> ulonglong2 {
    const int c1 = (64 * j) / CB - 1;  // last chunk whose overflow starts at or below bit 64j
    uint64_t add = 0;
    if (c1 >= 0 && c1 < nch) {
      const int d = 64 * j - CB * (c1 + 1);
      if (d < 64) add |= sH[c1] >> d;
    }
    const int c2 = c1 + 1;
    if (c2 >= 0 && c2 < nch) {
      const int o2 = CB * (c2 + 1) - 64 * j;  // > 0
      if (o2 < 64) add |= sH[c2] << o2;
    }
    return make_ulonglong2(out[j], add);
  };
  auto store = [&](int j, uint64_t v) { out[j] = v; };
  return blk_addsub<false>(nout, 0u, load, store, scr);
}

// blk_mul (band-limited) as one out-of-line function: the division and batch
// kernels call products from many places, and one shared copy keeps their
// code (and register pressure) small; the call costs nothing next to a
// product.
template <int RB, int Q, int F>
__device__ __noinline__ uint32_t blk_mul_call(const uint64_t *x, int nx, const uint64_t *y,
                                              int ny, uint64_t *out, int nout, uint32_t *smem,
                                              int lo) {
  return blk_mul<RB, Q, F, true>(x, nx, y, ny, out, nout, smem, lo);
}

// ---------------------------------------------------------------------------
// One level of Karatsuba for a square product (both operands n limbs):
// with x = x1 B^h + x0 and y = y1 B^h + y0 (h = floor(n/2)),
//   x y = z2 B^(2h) + (z1 - z0 - z2) B^h + z0,
//   z0 = x0 y0, z2 = x1 y1, z1 = (x0 + x1)(y0 + y1),
// three half-size products (each by blk_mul) instead of four: 3/4 of the
// digit products of the schoolbook full product.  Sec. VII names faster
// multiplication as the next step after the quadratic one; this is its
// exact-integer form.  The sums x0 + x1 and y0 + y1 are parked in the output
// (free until z0 is written), z1 lives in shared memory.
// smem: blk_kara_smem_words(n) words.  out: 2n limbs.
// ---------------------------------------------------------------------------
template <int RB, int Q>
__host__ __device__ constexpr int blk_kara_smem_words(int n) {
  const int hh = n - n / 2;
  return 2 * (2 * hh + 2) + blk_mul_smem_words<RB, Q>(hh + 1, hh + 1);
}

template <int RB, int Q>
__host__ __device__ constexpr int blk_kara_units(int n) {
  const int hh = n - n / 2;
  return blk_mul_units<RB, Q>(hh + 1, hh + 1);
}

template <int RB, int Q, int F>
__device__ void blk_mul_kara(const uint64_t *x, const uint64_t *y, int n, uint64_t *out,
                             uint32_t *smem) {
  const int h = n / 2, hh = n - h;  // x0, y0: h limbs; x1, y1: hh limbs
  const int nz1 = 2 * hh + 2;
  uint64_t *z1 = reinterpret_cast<uint64_t *>(smem);  // [nz1] limbs
  uint32_t *msm = smem + 2 * nz1;                     // blk_mul's region
  uint32_t *scr = msm;                                // scratch between products
  uint64_t *s1 = out, *s2 = out + (hh + 1);
  __shared__ uint32_t carries[2];
  {  // s1 = x0 + x1, s2 = y0 + y1 (hh + 1 limbs each)
    auto lx = [&](int j) { return make_ulonglong2(j < h ? x[j] : 0ull, x[h + j]); };
    auto sx = [&](int j, uint64_t v) { s1[j] = v; };
    const uint32_t c1 = blk_addsub<false>(hh, 0u, lx, sx, scr);
    auto ly = [&](int j) { return make_ulonglong2(j < h ? y[j] : 0ull, y[h + j]); };
    auto sy = [&](int j, uint64_t v) { s2[j] = v; };
    const uint32_t c2 = blk_addsub<false>(hh, 0u, ly, sy, scr);
    if (threadIdx.x == 0) {
      carries[0] = c1;
      carries[1] = c2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s1[hh] = carries[0];
      s2[hh] = carries[1];
    }
    __syncthreads();
  }
  // z1 = s1 s2 (into shared memory)
  blk_mul<RB, Q, F>(s1, hh + 1, s2, hh + 1, z1, nz1, msm);
  // z0 = x0 y0 -> out[0, 2h); z2 = x1 y1 -> out[2h, 2n)
  blk_mul<RB, Q, F>(x, h, y, h, out, 2 * h, msm);
  blk_mul<RB, Q, F>(x + h, hh, y + h, hh, out + 2 * h, 2 * hh, msm);
  {  // z1 -= z0; z1 -= z2 (the difference x0 y1 + x1 y0 is nonnegative)
    auto l0 = [&](int j) { return make_ulonglong2(z1[j], j < 2 * h ? out[j] : 0ull); };
    auto st = [&](int j, uint64_t v) { z1[j] = v; };
    blk_addsub<true>(nz1, 0u, l0, st, scr);
    auto l2 = [&](int j) { return make_ulonglong2(z1[j], j < 2 * hh ? out[2 * h + j] : 0ull); };
    blk_addsub<true>(nz1, 0u, l2, st, scr);
  }
  {  // out[h ..] += z1
    auto la = [&](int j) { return make_ulonglong2(out[h + j], j < nz1 ? z1[j] : 0ull); };
    auto sa = [&](int j, uint64_t v) { out[h + j] = v; };
    blk_addsub<false>(2 * n - h, 0u, la, sa, scr);
  }
}

}  // namespace bigint
