// tune.cu -- the autotuner and its persistent table.
//
// Two knobs are tuned by timing on the caller's own data:
//   * the multiply variant (digit size RB, chunk width Q -- the "limbs per
//     thread" of the paper's sequentialisation factor -- and the carry
//     interval) per operand size class;
//   * the CTA size ("threads per instance") of persistent batch launches.
// The table is saved as a small JSON file keyed by the GPU name.
#include <cstdio>
#include <cstring>
#include <string>

#include "common.cuh"

struct bigint_batch;

namespace bigint {
int launch_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na,
               int nb, int nout, cudaStream_t st);
int mul_set_variant(int v);
int mul_size_class(int na, int nb);
extern int g_mul_tuned[32];
int batch_set_threads(int t);
int batch_get_threads();
int batch_configure(bigint_batch *B);
int batch_launch(const bigint_batch *B, const uint64_t *in, uint64_t *out, int32_t *status,
                 void *ws, int mode, cudaStream_t st);
size_t batch_workspace_bytes(const bigint_batch *B);
int batch_retune(bigint_batch *B, int threads);

namespace {

// Time of fn() on stream st: best of `reps` runs, after one warm-up.
template <class F>
int time_best(F fn, cudaStream_t st, int reps, float *best_ms) {
  cudaEvent_t e0, e1;
  BIGINT_CUDA_TRY(cudaEventCreate(&e0));
  BIGINT_CUDA_TRY(cudaEventCreate(&e1));
  int rc = fn();
  *best_ms = 1e30f;
  for (int i = 0; i < reps && rc == BIGINT_OK; i++) {
    cudaEventRecord(e0, st);
    rc = fn();
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) rc = BIGINT_ECUDA;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < *best_ms) *best_ms = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}

std::string gpu_name() {
  int dev = 0;
  cudaDeviceProp p;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&p, dev) != cudaSuccess)
    return "unknown";
  return std::string(p.name);
}

}  // namespace

int tune_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na, int nb,
             cudaStream_t st, int *best_variant) {
  int best = 0;
  float best_ms = 1e30f;
  for (int v = 1; v <= 6; v++) {
    mul_set_variant(v);
    float ms = 0;
    const int rc = time_best([&] { return launch_mul(a, b, out, count, na, nb, na + nb, st); },
                             st, 2, &ms);
    if (rc == BIGINT_OK && ms < best_ms) {
      best_ms = ms;
      best = v;
    }
  }
  mul_set_variant(0);
  if (best == 0) return BIGINT_EINTERNAL;
  g_mul_tuned[mul_size_class(na, nb)] = best;
  if (best_variant) *best_variant = best;
  return BIGINT_OK;
}

int tune_batch(bigint_batch *B, const uint64_t *in, uint64_t *out, int32_t *status, void *ws,
               size_t bytes, cudaStream_t st, int *best_threads) {
  if (bytes < batch_workspace_bytes(B)) return BIGINT_ENOMEM;
  static const int cand[] = {256, 384, 512};
  int best = 0;
  float best_ms = 1e30f;
  for (int T : cand) {
    int rc = batch_retune(B, T);
    if (rc != BIGINT_OK) return rc;
    if (batch_workspace_bytes(B) > bytes) continue;  // needs more resident CTAs than budgeted
    float ms = 0;
    rc = time_best([&] { return batch_launch(B, in, out, status, ws, BIGINT_BATCH_PERSISTENT, st); },
                   st, 2, &ms);
    if (rc != BIGINT_OK) return rc;
    if (ms < best_ms) {
      best_ms = ms;
      best = T;
    }
  }
  if (best == 0) return BIGINT_EINTERNAL;
  batch_set_threads(best);
  const int rc = batch_retune(B, best);
  if (best_threads) *best_threads = best;
  return rc;
}

int tuning_save(const char *path) {
  FILE *f = std::fopen(path, "w");
  if (!f) return BIGINT_EINVAL;
  std::fprintf(f, "{\n  \"gpu\": \"%s\",\n  \"batch_threads\": %d,\n  \"mul_variant_by_class\": [",
               gpu_name().c_str(), batch_get_threads());
  for (int c = 0; c < 32; c++) std::fprintf(f, "%s%d", c ? ", " : "", g_mul_tuned[c]);
  std::fprintf(f, "]\n}\n");
  std::fclose(f);
  return BIGINT_OK;
}

int tuning_load(const char *path) {
  FILE *f = std::fopen(path, "r");
  if (!f) return BIGINT_EINVAL;
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = std::fread(buf, 1, sizeof buf, f)) > 0) text.append(buf, n);
  std::fclose(f);
  auto find_after = [&](const char *key) -> size_t {
    const size_t k = text.find(key);
    if (k == std::string::npos) return std::string::npos;
    const size_t c = text.find(':', k);
    return c == std::string::npos ? c : c + 1;
  };
  const size_t g = find_after("\"gpu\"");
  if (g == std::string::npos) return BIGINT_EINVAL;
  const size_t q0 = text.find('"', g), q1 = text.find('"', q0 + 1);
  if (q0 == std::string::npos || q1 == std::string::npos) return BIGINT_EINVAL;
  if (text.substr(q0 + 1, q1 - q0 - 1) != gpu_name()) return BIGINT_EINVAL;
  int threads = 0, classes[32] = {};
  const size_t t = find_after("\"batch_threads\"");
  if (t == std::string::npos || std::sscanf(text.c_str() + t, "%d", &threads) != 1)
    return BIGINT_EINVAL;
  size_t m = find_after("\"mul_variant_by_class\"");
  if (m == std::string::npos) return BIGINT_EINVAL;
  m = text.find('[', m);
  for (int c = 0; c < 32; c++) {
    int v = 0, used = 0;
    if (m == std::string::npos || std::sscanf(text.c_str() + m + 1, " %d%n", &v, &used) != 1)
      return BIGINT_EINVAL;
    if (v < 0 || v > 6) return BIGINT_EINVAL;
    classes[c] = v;
    m = text.find(c < 31 ? ',' : ']', m + 1);
  }
  if (batch_set_threads(threads) != BIGINT_OK) return BIGINT_EINVAL;
  for (int c = 0; c < 32; c++) g_mul_tuned[c] = classes[c];
  return BIGINT_OK;
}

}  // namespace bigint
