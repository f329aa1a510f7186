// tune.cu -- the autotuner and its persistent table.
//
// Two knobs are tuned by timing on the caller's own data:
//   * the multiply variant per operand size class: the tensor-core product's
//     tile (64, 128 or 256 output columns per tile, i.e. three, two or one
//     CTAs per SM) or an integer product (digit size RB and chunk width Q --
//     the "limbs per thread" of the paper's sequentialisation factor);
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
bool mul_variant_valid(int v);
size_t mul_tc_smem(int na, int nb);
int mul_size_class(int na, int nb);
extern int g_mul_tuned[32];
int batch_set_threads(int t);
int batch_get_threads();
int batch_configure(bigint_batch *B);
int batch_launch(const bigint_batch *B, const uint64_t *in, uint64_t *out, int32_t *status,
                 void *ws, int mode, cudaStream_t st);
size_t batch_workspace_bytes(const bigint_batch *B);
int batch_retune(bigint_batch *B, int threads, int use_tc);
bool batch_uses_tc(const bigint_batch *B);
int batch_threads_of(const bigint_batch *B);

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

// Candidates of the multiply tuner for an na x nb product: the tensor-core
// product with its shape chosen by the cost model (12), forced to 128-digit
// x blocks with 64, 128 and 256 output columns (13, 14, 15) -- the tile also
// sets how many CTAs share an SM -- and to narrow x blocks of 64 and 32
// digits (16, 17), and the integer products with 29-bit digits / 16-column
// chunks (8) and 28-bit digits / 8-column chunks (9), plus one level of
// Karatsuba (10) for square products.
int tune_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na, int nb,
             cudaStream_t st, int *best_variant) {
  int cand[10], nc = 0;
  if ((na < nb ? na : nb) >= 64 && mul_tc_smem(na, nb) > 0) {
    cand[nc++] = 12; cand[nc++] = 13; cand[nc++] = 14; cand[nc++] = 15;
    cand[nc++] = 16; cand[nc++] = 17;
  }
  cand[nc++] = 8;
  cand[nc++] = 9;
  if (na == nb && na >= 64) cand[nc++] = 10;
  int best = 0;
  float best_ms = 1e30f;
  for (int i = 0; i < nc; i++) {
    if (mul_set_variant(cand[i]) != BIGINT_OK) continue;
    float ms = 0;
    const int rc = time_best([&] { return launch_mul(a, b, out, count, na, nb, na + nb, st); },
                             st, 2, &ms);
    if (rc == BIGINT_OK && ms < best_ms) {
      best_ms = ms;
      best = cand[i];
    }
    if (rc != BIGINT_OK) cudaGetLastError();  // a candidate that does not fit this shape
  }
  mul_set_variant(0);
  if (best == 0) return BIGINT_EINTERNAL;
  g_mul_tuned[mul_size_class(na, nb)] = best;
  if (best_variant) *best_variant = best;
  return BIGINT_OK;
}

// Candidates of the batch tuner: the launch whose CTAs hold their SM's
// tensor memory and run the large products on the tensor cores (when the
// batch has such products), and launches on the integer pipes alone with
// 256, 384 or 512 threads per CTA (threads per instance).  *best_threads
// receives the chosen CTA size (tcm::TC_CTA_THREADS for the tensor-core
// form).
int tune_batch(bigint_batch *B, const uint64_t *in, uint64_t *out, int32_t *status, void *ws,
               size_t bytes, cudaStream_t st, int *best_threads) {
  if (bytes < batch_workspace_bytes(B)) return BIGINT_ENOMEM;
  struct Cand { bool tc; int threads; };
  const Cand cand[] = {{true, 0}, {false, 256}, {false, 384}, {false, 512}};
  int best = -1;
  float best_ms = 1e30f;
  for (int i = 0; i < 4; i++) {
    int rc = batch_retune(B, cand[i].threads, cand[i].tc ? 1 : 0);
    if (rc != BIGINT_OK) return rc;
    if (cand[i].tc && !batch_uses_tc(B)) continue;  // nothing for the tensor cores
    if (batch_workspace_bytes(B) > bytes) continue;  // needs more resident CTAs than budgeted
    float ms = 0;
    rc = time_best([&] { return batch_launch(B, in, out, status, ws, BIGINT_BATCH_PERSISTENT, st); },
                   st, 2, &ms);
    if (rc != BIGINT_OK) return rc;
    if (ms < best_ms) {
      best_ms = ms;
      best = i;
    }
  }
  if (best < 0) return BIGINT_EINTERNAL;
  if (!cand[best].tc) batch_set_threads(cand[best].threads);
  const int rc = batch_retune(B, cand[best].threads, cand[best].tc ? 1 : 0);
  if (best_threads) *best_threads = batch_threads_of(B);
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
    if (!mul_variant_valid(v)) return BIGINT_EINVAL;
    classes[c] = v;
    m = text.find(c < 31 ? ',' : ']', m + 1);
  }
  if (batch_set_threads(threads) != BIGINT_OK) return BIGINT_EINVAL;
  for (int c = 0; c < 32; c++) g_mul_tuned[c] = classes[c];
  return BIGINT_OK;
}

}  // namespace bigint
