// noalloc.cu -- bigint_divmod for callers that cannot allocate device memory.
//
// bigint_divmod needs a scratch workspace that the caller allocates.  Some
// callers cannot do that: code that must not call cudaMalloc (for example a
// host application that hands this library a fixed memory budget, or a
// latency-critical loop that cannot afford cudaMalloc's implicit device
// synchronisation).  bigint_divmod_noalloc serves them: its scratch is one
// file-scope __device__ array of NOALLOC_SCRATCH_BYTES that every GPU loading
// this library holds until the process exits.  The entry point itself calls
// no cudaMalloc, cudaFree or any allocating library routine.
//
// In host code the array's name is only a host-side stand-in, not a device
// address, so the address is looked up with cudaGetSymbolAddress once per
// device (again only if that device's context was destroyed and created
// anew, which can move the array) and then passed to the existing division
// kernels.
// Batches whose scratch does not fit the array are processed in consecutive
// launches on the caller's stream, as many instances per launch as fit.
#include <mutex>

#include "common.cuh"

namespace bigint {
int launch_divmod(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                  int32_t *status, int64_t count, int nu, int nv, void *ws, size_t ws_bytes,
                  cudaStream_t st);
size_t divmod_workspace(int64_t count, int nu, int nv);
}  // namespace bigint

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;  // 32 MiB per device
static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_SCRATCH_BYTES / 8];

constexpr int MAX_DEVICES = 64;
// Per device: the scratch array's device address and the id of the context
// it was looked up in.  The array lives in the library's module, which is
// loaded once per context: after cudaDeviceReset (or any other way the
// device's context is destroyed and created again) the module is loaded
// again and the array may sit at another address, so a lookup is valid only
// for the context it was made in.
struct ScratchEntry {
  unsigned long long ctx_id;
  void *addr;
};
ScratchEntry g_scratch[MAX_DEVICES] = {};
std::mutex g_scratch_mutex;

typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// Unique id of the context current on this thread (0 if none), through the
// driver entry points the runtime hands out (no link against libcuda).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (get_current == nullptr || get_id == nullptr) {
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess)
      return 0;
    get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (get_current(&ctx) != 0 || ctx == nullptr || get_id(ctx, &id) != 0) return 0;
  return id;
}

// Device address of the scratch array in the current context of device
// `dev` (current on this thread), looked up with cudaGetSymbolAddress the
// first time the library meets that context; nullptr if the lookup failed.
void *scratch_address(int dev) {
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  // makes the device's primary context current (and creates it if needed),
  // so that there is a context whose id identifies the lookup
  if (cudaSetDevice(dev) != cudaSuccess) return nullptr;
  const unsigned long long id = current_context_id();
  ScratchEntry &e = g_scratch[dev];
  if (e.addr == nullptr || id == 0 || e.ctx_id != id) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return nullptr;
    e.addr = p;
    e.ctx_id = id;
  }
  return e.addr;
}

}  // namespace

extern "C" size_t bigint_divmod_noalloc_scratch_bytes(void) { return NOALLOC_SCRATCH_BYTES; }

extern "C" int bigint_divmod_noalloc(const uint64_t *u, const uint64_t *v, uint64_t *q,
                                     uint64_t *r, int32_t *status, int64_t count, int32_t nu,
                                     int32_t nv, void *stream) {
  if (count < 0 || count > 0x7fffffff || nu < 1 || nv < 1) return BIGINT_EINVAL;
  if (nu > BIGINT_MAX_LIMBS || nv > BIGINT_MAX_LIMBS) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  if (!u || !v || !q || !r) return BIGINT_EINVAL;
  const size_t per = bigint::divmod_workspace(1, nu, nv);
  if (per == 0 || per > NOALLOC_SCRATCH_BYTES) return BIGINT_ENOMEM;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return BIGINT_ECUDA;
  void *scratch = scratch_address(dev);
  if (scratch == nullptr) return BIGINT_ECUDA;
  const int nq = nu - nv + 1 > 1 ? nu - nv + 1 : 1;
  const int64_t chunk = (int64_t)(NOALLOC_SCRATCH_BYTES / per);
  for (int64_t i0 = 0; i0 < count; i0 += chunk) {
    const int64_t c = count - i0 < chunk ? count - i0 : chunk;
    const int rc = bigint::launch_divmod(u + i0 * nu, v + i0 * nv, q + i0 * nq, r + i0 * nv,
                                         status ? status + i0 : nullptr, c, nu, nv, scratch,
                                         NOALLOC_SCRATCH_BYTES,
                                         reinterpret_cast<cudaStream_t>(stream));
    if (rc != BIGINT_OK) return rc;
  }
  return BIGINT_OK;
}
