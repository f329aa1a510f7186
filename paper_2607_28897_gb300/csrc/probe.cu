// probe.cu -- integer-pipe throughput probe for the multiply roofline.
//
// The multiply is bound by the SM's integer multiply-add issue rate, a
// number NVIDIA does not publish per instruction form for sm_103.  This probe
// measures it: every SM runs register-only loops of one instruction form with
// eight independent dependency chains per thread at full occupancy, and each
// block times itself with the SM cycle counter.  The result is thread-level
// operations per SM per SM clock cycle.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace bigint {

constexpr int PROBE_ITERS = 4096;

template <int VARIANT>
__global__ void __launch_bounds__(256) k_probe(uint32_t seed, uint64_t *sink, long long *cycles) {
  __shared__ long long t0;
  uint32_t x[8];
  uint64_t y[8];
#pragma unroll
  for (int k = 0; k < 8; k++) {
    x[k] = seed * (threadIdx.x + 7 * k + 1) | 1u;
    y[k] = x[k] ^ 0x9e3779b9u;
  }
  const uint32_t m = seed | 3u;
  __syncthreads();
  if (threadIdx.x == 0) t0 = clock64();
  __syncthreads();
  if constexpr (VARIANT == 0) {
#pragma unroll 1
    for (int it = 0; it < PROBE_ITERS; it++) {
#pragma unroll
      for (int k = 0; k < 8; k++)
        asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(y[k]) : "r"(x[k]), "r"(m));
    }
  } else if constexpr (VARIANT == 1) {
#pragma unroll 1
    for (int it = 0; it < PROBE_ITERS; it++) {
#pragma unroll
      for (int k = 0; k < 8; k++)
        asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[k]) : "r"(m), "r"(m));
    }
  } else if constexpr (VARIANT == 2) {
#pragma unroll 1
    for (int it = 0; it < PROBE_ITERS; it++) {
#pragma unroll
      for (int k = 0; k < 8; k++)
        asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[k]) : "r"(m), "r"(m));
    }
  } else {
    // the multiply kernel's inner step: 8 column accumulators, a sliding
    // window of 16 digits, one mad.wide.u32 per digit product
    uint64_t acc[8];
    uint32_t W[16];
#pragma unroll
    for (int q = 0; q < 8; q++) acc[q] = x[q];
#pragma unroll
    for (int q = 0; q < 16; q++) W[q] = x[(q + 3) & 7] + q;
#pragma unroll 1
    for (int it = 0; it < PROBE_ITERS / 8; it++) {
#pragma unroll
      for (int t = 0; t < 8; t++) {
        const uint32_t a = x[t] ^ (uint32_t)it;
#pragma unroll
        for (int q = 0; q < 8; q++)
          asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc[q]) : "r"(a), "r"(W[8 - t + q]));
      }
#pragma unroll
      for (int q = 0; q < 8; q++) W[8 + q] = W[q] + (uint32_t)it;
    }
#pragma unroll
    for (int q = 0; q < 8; q++) y[q] += acc[q];
  }
  __syncthreads();
  if (threadIdx.x == 0) cycles[blockIdx.x] = clock64() - t0;
  uint64_t s = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) s += y[k] + x[k];
  if (s == 0x1234567ull) sink[0] = s;  // keeps the loops alive
}

// Operations per thread for one probe launch.
static double probe_ops_per_thread(int variant) {
  if (variant == 3) return (double)(PROBE_ITERS / 8) * 64;
  return (double)PROBE_ITERS * 8;
}

template <int V>
static int run_probe(double *ops_per_clk_sm, double *sm_mhz) {
  int dev = 0, sms = 0, per_sm = 0;
  BIGINT_CUDA_TRY(cudaGetDevice(&dev));
  BIGINT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BIGINT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe<V>, 256, 0));
  if (per_sm < 1) return BIGINT_EINTERNAL;
  const int blocks = sms * per_sm;
  uint64_t *sink = nullptr;
  long long *cycles = nullptr;
  BIGINT_CUDA_TRY(cudaMalloc(&sink, 8));
  BIGINT_CUDA_TRY(cudaMalloc(&cycles, sizeof(long long) * blocks));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  k_probe<V><<<blocks, 256>>>(12345u, sink, cycles);  // warm-up
  cudaEventRecord(e0);
  k_probe<V><<<blocks, 256>>>(54321u, sink, cycles);
  cudaEventRecord(e1);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  std::vector<long long> cyc(blocks);
  if (err == cudaSuccess)
    err = cudaMemcpy(cyc.data(), cycles, sizeof(long long) * blocks, cudaMemcpyDeviceToHost);
  cudaFree(sink);
  cudaFree(cycles);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return BIGINT_ECUDA;
  std::sort(cyc.begin(), cyc.end());
  const double med = (double)cyc[blocks / 2];
  const double ops_block = probe_ops_per_thread(V) * 256.0;
  *ops_per_clk_sm = ops_block * per_sm / med;
  *sm_mhz = (double)cyc[blocks - 1] / (ms * 1e3);
  return BIGINT_OK;
}

int probe_int_throughput(int variant, double *ops, double *mhz) {
  switch (variant) {
    case 0: return run_probe<0>(ops, mhz);
    case 1: return run_probe<1>(ops, mhz);
    case 2: return run_probe<2>(ops, mhz);
    case 3: return run_probe<3>(ops, mhz);
    default: return BIGINT_EINVAL;
  }
}

}  // namespace bigint
