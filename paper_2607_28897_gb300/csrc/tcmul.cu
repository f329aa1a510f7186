// tcmul.cu -- batched full (and low-part) products on the tensor cores.
//
// One persistent CTA per SM (NT = 256) or two (NT = 128) loops over the
// instances of a uniform batch, each product computed by tc_product
// (tccore.cuh: the digit convolution as tcgen05 fp16 MMAs with exact fp32
// accumulation, Sec. V-B's schoolbook product on the tensor cores).
#include "tccore.cuh"

namespace bigint {
namespace tcm {

// 2 NT drain threads plus one issuer warp (tc_product<NT, G, true>).
template <int NT, int G>
__global__ void __launch_bounds__(2 * NT + 32, 256 / NT)
    k_mul_tc(const uint64_t *__restrict__ X, const uint64_t *__restrict__ Y,
             uint64_t *__restrict__ Out, int nx, int ny, int nout, int64_t count) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ TcShared sh;
  __shared__ uint32_t scr[BLK_SCRATCH_WORDS];
  TcCtx c;
  tc_init<NT>(c, sm, &sh, scr);
  for (int64_t inst = blockIdx.x; inst < count; inst += gridDim.x)
    if (!tc_product<NT, G, true>(c, X + inst * (int64_t)nx, nx, Y + inst * (int64_t)ny, ny,
                           Out + inst * (int64_t)nout, nout, 0))
      break;
  tc_release<NT>(c);
}

}  // namespace tcm

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
template <int NT, int G>
static int tc_dyn_max() {
  static int dyn = -1;
  if (dyn < 0) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
      return 0;
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, tcm::k_mul_tc<NT, G>) != cudaSuccess) return 0;
    const int d = optin - (int)fa.sharedSizeBytes;
    if (cudaFuncSetAttribute(tcm::k_mul_tc<NT, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             d) != cudaSuccess)
      return 0;
    dyn = d;
  }
  return dyn;
}

// Tile width for an nx x ny product (nx <= ny): 128 columns while the
// output has at most 128 columns of 128 digits (n up to ~1000 limbs for
// square products), else 256.
static int tc_tile(int nx, int ny) {
  return (8 * nx + 1 + 127) / 128 + (8 * ny + 127) / 128 <= 128 ? 128 : 256;
}

template <int NT, int G>
static size_t tc_smem(int nx, int ny) {
  const tcm::Layout L = tcm::layout<NT, G>(nx, ny);
  const int d = tc_dyn_max<NT, G>();
  return d > 0 && L.total <= (uint32_t)d ? L.total : 0;
}

// Group size: 8 Toeplitz blocks per drain where the Hankel buffers fit,
// else 4 (0: the product does not fit at all).
template <int NT>
static int tc_group(int nx, int ny) {
  if (tc_smem<NT, 8>(nx, ny)) return 8;
  if (tc_smem<NT, 4>(nx, ny)) return 4;
  return 0;
}

// Dynamic shared memory the tensor-core product of an na x nb product
// needs, or 0 if it does not fit (or the shapes are out of range).
size_t mul_tc_smem(int na, int nb) {
  const int nx = na < nb ? na : nb, ny = na < nb ? nb : na;
  if (nx < 1 || ny > 16383) return 0;
  if (tc_tile(nx, ny) == 128)
    return tc_group<128>(nx, ny) == 8 ? tc_smem<128, 8>(nx, ny) : tc_smem<128, 4>(nx, ny);
  return tc_group<256>(nx, ny) == 8 ? tc_smem<256, 8>(nx, ny) : tc_smem<256, 4>(nx, ny);
}

template <int NT, int G>
static int launch_tc(const uint64_t *x, const uint64_t *y, uint64_t *out, int64_t count, int nx,
                     int ny, int nout, cudaStream_t st) {
  const size_t smem = tc_smem<NT, G>(nx, ny);
  if (smem == 0) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  int dev = 0, sms = 0;
  BIGINT_CUDA_TRY(cudaGetDevice(&dev));
  BIGINT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t slots = (int64_t)sms * (256 / NT);  // CTAs resident at once
  const int64_t grid = count < slots ? count : slots;
  tcm::k_mul_tc<NT, G><<<(unsigned)grid, 2 * NT + 32, smem, st>>>(x, y, out, nx, ny, nout, count);
  return bigint_launch_status();
}

int launch_mul_tc(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na,
                  int nb, int nout, cudaStream_t st) {
  const uint64_t *x = a, *y = b;
  int nx = na, ny = nb;
  if (nb < na) { x = b; y = a; nx = nb; ny = na; }
  if (nx < 1 || ny > 16383 || nout < 1 || nout > na + nb) return BIGINT_EINVAL;
  if (tc_tile(nx, ny) == 128)
    return tc_group<128>(nx, ny) == 8 ? launch_tc<128, 8>(x, y, out, count, nx, ny, nout, st)
                                      : launch_tc<128, 4>(x, y, out, count, nx, ny, nout, st);
  return tc_group<256>(nx, ny) == 8 ? launch_tc<256, 8>(x, y, out, count, nx, ny, nout, st)
                                    : launch_tc<256, 4>(x, y, out, count, nx, ny, nout, st);
}

// BIGINT_ETIMEOUT if a tensor-core product hit a wait limit since the last
// call (synchronises the device), else BIGINT_OK.
int tc_take_timeout() {
  BIGINT_CUDA_TRY(cudaDeviceSynchronize());
  int v = 0;
  BIGINT_CUDA_TRY(cudaMemcpyFromSymbol(&v, tcm::g_timeout, sizeof(int)));
  if (v) {
    const int zero = 0;
    BIGINT_CUDA_TRY(cudaMemcpyToSymbol(tcm::g_timeout, &zero, sizeof(int)));
    return BIGINT_ETIMEOUT;
  }
  return BIGINT_OK;
}

}  // namespace bigint
