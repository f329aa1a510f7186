// common.cuh -- shared device helpers of libbigint (sm_103a).
//
// Digits: every kernel works on 32-bit digits.  A little-endian array of
// 64-bit limbs is, byte for byte, a little-endian array of 32-bit digits
// (limb i = digit 2i + 2^32 * digit 2i+1), so device code may reinterpret a
// limb pointer as a digit pointer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "bigint.h"

namespace bigint {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------------------
// Carry resolution over 32 lanes with two ballots.
//
// Each lane holds a (generate, propagate) pair for its digits: g = the lane's
// digits produce a carry by themselves, p = they pass an incoming carry
// through (all result digits are at their maximum).  g and p are never both
// set.  With G and P the warp's ballots and X = G | P, the binary sum
// X + G + cin carries into bit i exactly when the digit-level carry reaches
// lane i: a generate lane has X_i = G_i = 1 (always carries out), a propagate
// lane has X_i = 1, G_i = 0 (carries out iff a carry comes in), any other
// lane has X_i = G_i = 0 (never carries out).  So the carry INTO every lane
// is bit i of (X + G + cin) ^ X ^ G, and the carry out of the warp is bit 32.
// This evaluates the exclusive scan with the operator of Fig. 3,
//   (g1,p1) o (g2,p2) = (g2 | (g1 & p2), p1 & p2),
// in a handful of integer instructions.
// ---------------------------------------------------------------------------
struct WarpCarry {
  uint32_t G, X;
};

__device__ __forceinline__ WarpCarry warp_gp(uint32_t g, uint32_t p) {
  WarpCarry w;
  w.G = __ballot_sync(FULL, g);
  w.X = w.G | __ballot_sync(FULL, p);
  return w;
}

// 64-bit word whose bit i (i < 32) is the carry into lane i and whose bit 32
// is the carry out of lane 31.
__device__ __forceinline__ uint64_t warp_carries(WarpCarry w, uint32_t cin) {
  const uint64_t s = (uint64_t)w.X + w.G + cin;
  return s ^ w.X ^ w.G;
}

// Carry out of the whole warp for a given carry in.
__device__ __forceinline__ uint32_t warp_carry_out(WarpCarry w, uint32_t cin) {
  return (uint32_t)(((uint64_t)w.X + w.G + cin) >> 32);
}

// (g, p) of a whole warp: generate = carry out with carry-in 0,
// propagate = every lane propagates.
__device__ __forceinline__ uint32_t warp_all_propagate(WarpCarry w) {
  return (w.X == FULL) && (w.G == 0);
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }

// Streaming global accesses (each limb is touched once).
__device__ __forceinline__ ulonglong2 ld_stream2(const uint64_t *p) {
  return __ldcs(reinterpret_cast<const ulonglong2 *>(p));
}
__device__ __forceinline__ void st_stream2(uint64_t *p, ulonglong2 v) {
  __stcs(reinterpret_cast<ulonglong2 *>(p), v);
}

}  // namespace bigint

// Host-side helpers --------------------------------------------------------
#define BIGINT_CUDA_TRY(expr)                   \
  do {                                          \
    cudaError_t e__ = (expr);                   \
    if (e__ != cudaSuccess) return BIGINT_ECUDA; \
  } while (0)

namespace bigint {
// Counts the kernel launches the library enqueues (bigint_kernel_launches).
void count_launch();

// Shapes the tensor-core product can be forced to (the autotuner's
// candidates; 0 = chosen by the cost model): 128-digit x blocks with the
// 64-, 128- or 256-column tile, or narrow x blocks of 64 or 32 digits.
constexpr int TC_FORCE_64 = 64, TC_FORCE_128 = 128, TC_FORCE_256 = 256;
constexpr int TC_FORCE_N64 = 1064, TC_FORCE_N32 = 1032;
}  // namespace bigint

// Called right after every kernel launch of the library: counts it and
// reports a launch error.
static inline int bigint_launch_status() {
  bigint::count_launch();
  return cudaPeekAtLastError() == cudaSuccess ? BIGINT_OK : BIGINT_ECUDA;
}
