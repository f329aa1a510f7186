// capi.cu -- the extern "C" entry points of libbigint (include/bigint.h).
//
// Host-side argument checks and dispatch only; every arithmetic step runs in
// the kernels of addsub.cu, mul.cu and divmod.cu.
#include <atomic>
#include <cstdio>

#include "common.cuh"

namespace bigint {
static std::atomic<unsigned long long> g_kernel_launches{0};
void count_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace bigint

namespace bigint {
int launch_addsub(bool sub, const uint64_t *a, const uint64_t *b, uint64_t *out,
                  uint8_t *carry, int64_t count, int n, cudaStream_t st);
int launch_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na,
               int nb, int nout, cudaStream_t st);
int mul_max_limbs();
size_t mul_split_workspace(int64_t count, int na, int nb);
int launch_mul_split(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na,
                     int nb, void *ws, size_t bytes, cudaStream_t st);
size_t mul_kara_workspace(int64_t count, int n, int levels);
int launch_mul_kara(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int n,
                    int levels, void *ws, size_t bytes, cudaStream_t st);
int mul_set_variant(int v);
int mul_variant_for(int na, int nb, int nout);
int tc_take_timeout();
int programs_take_timeout();
int div_take_timeout();
int batch_take_timeout();
int tc_set_wait_limit(long long cycles);
int div_set_wait_limit(long long cycles);
int programs_set_wait_limit(long long cycles);
int batch_set_wait_limit(long long cycles);
int launch_add_chain(const uint64_t *a, const uint64_t *b, uint64_t *out, uint8_t *carry,
                     int64_t count, int n, int k, cudaStream_t st);
size_t poly_workspace(int64_t count, int n);
int launch_poly(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int n,
                void *ws, size_t bytes, cudaStream_t st);
size_t host_workspace(int op, int64_t chunk, int na, int nb);
int host_run(int op, const uint64_t *in0, const uint64_t *in1, uint64_t *out0, uint64_t *out1,
             void *aux, int64_t count, int na, int nb, void *workspace, size_t bytes, bool sync);
int host_sync();
int div_set_variant(int v);
int batch_set_variant(int v);
int probe_int_throughput(int variant, double *ops, double *mhz);
int launch_divmod(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                  int32_t *status, int64_t count, int nu, int nv, void *ws, size_t ws_bytes,
                  cudaStream_t st);
size_t divmod_workspace(int64_t count, int nu, int nv);
int launch_shinv(const uint64_t *v, uint64_t *w, int32_t *status, int64_t count, int nv,
                 int h, int nw, void *ws, size_t ws_bytes, cudaStream_t st);
size_t shinv_workspace(int64_t count, int nv, int h);
int launch_divmod_inv(const uint64_t *u, const uint64_t *v, const uint64_t *w, uint64_t *q,
                      uint64_t *r, int32_t *status, int64_t count, int nu, int nv, int nw, int h,
                      int64_t v_stride, int64_t w_stride, void *ws, cudaStream_t st);
int batch_create(const bigint_op *ops, int64_t nops, bigint_batch **out);
size_t batch_workspace_bytes(const bigint_batch *B);
int batch_upload(bigint_batch *B, void *ws, size_t bytes, cudaStream_t st);
int batch_launch(const bigint_batch *B, const uint64_t *in, uint64_t *out, int32_t *status,
                 void *ws, int mode, cudaStream_t st);
void batch_destroy(bigint_batch *B);
int tune_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na, int nb,
             cudaStream_t st, int *best_variant);
int tune_batch(bigint_batch *B, const uint64_t *in, uint64_t *out, int32_t *status, void *ws,
               size_t bytes, cudaStream_t st, int *best_threads);
int tuning_save(const char *path);
int tuning_load(const char *path);
}  // namespace bigint

using namespace bigint;

static inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" {

const char *bigint_strerror(int status) {
  switch (status) {
    case BIGINT_OK: return "ok";
    case BIGINT_EINVAL: return "invalid argument";
    case BIGINT_EDIVZERO: return "division by zero";
    case BIGINT_ENOMEM: return "workspace too small";
    case BIGINT_ETIMEOUT: return "device wait limit reached";
    case BIGINT_EINTERNAL: return "internal correction limit exceeded";
    case BIGINT_ECUDA: return "CUDA runtime error";
    case BIGINT_ERANGE: return "quotient does not fit in the output";
    default: return "unknown status";
  }
}

int bigint_version(void) { return 100; }

static int check_addsub(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count,
                        int32_t n) {
  if (count < 0 || n < 1 || n > BIGINT_MAX_LIMBS) return BIGINT_EINVAL;
  if (count > 0 && (!a || !b || !out)) return BIGINT_EINVAL;
  if (count > 0x7fffffff) return BIGINT_EINVAL;
  return BIGINT_OK;
}

int bigint_add(const uint64_t *a, const uint64_t *b, uint64_t *out, uint8_t *carry_out,
               int64_t count, int32_t n, void *stream) {
  int rc = check_addsub(a, b, out, count, n);
  if (rc != BIGINT_OK || count == 0) return rc;
  return launch_addsub(false, a, b, out, carry_out, count, n, as_stream(stream));
}

int bigint_sub(const uint64_t *a, const uint64_t *b, uint64_t *out, uint8_t *borrow_out,
               int64_t count, int32_t n, void *stream) {
  int rc = check_addsub(a, b, out, count, n);
  if (rc != BIGINT_OK || count == 0) return rc;
  return launch_addsub(true, a, b, out, borrow_out, count, n, as_stream(stream));
}

int bigint_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int32_t na,
               int32_t nb, void *stream) {
  if (count < 0 || count > 0x7fffffff || na < 1 || nb < 1) return BIGINT_EINVAL;
  if (na > mul_max_limbs() || nb > mul_max_limbs()) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  if (!a || !b || !out) return BIGINT_EINVAL;
  return launch_mul(a, b, out, count, na, nb, na + nb, as_stream(stream));
}

int bigint_mul_lo(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count,
                  int32_t na, int32_t nb, int32_t m, void *stream) {
  if (count < 0 || count > 0x7fffffff || na < 1 || nb < 1) return BIGINT_EINVAL;
  if (na > mul_max_limbs() || nb > mul_max_limbs()) return BIGINT_EINVAL;
  if (m < 1 || m > na + nb) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  if (!a || !b || !out) return BIGINT_EINVAL;
  return launch_mul(a, b, out, count, na, nb, m, as_stream(stream));
}

size_t bigint_mul_split_workspace(int64_t count, int32_t na, int32_t nb) {
  if (count < 0 || na < 1 || nb < 1) return 0;
  return mul_split_workspace(count, na, nb);
}

int bigint_mul_split(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count,
                     int32_t na, int32_t nb, void *workspace, size_t workspace_bytes,
                     void *stream) {
  if (count < 0 || count > 0x7fffffff || na < 1 || nb < 1) return BIGINT_EINVAL;
  if (na > mul_max_limbs() || nb > mul_max_limbs()) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  if (!a || !b || !out) return BIGINT_EINVAL;
  return launch_mul_split(a, b, out, count, na, nb, workspace, workspace_bytes,
                          as_stream(stream));
}

size_t bigint_mul_kara_workspace(int64_t count, int32_t n, int32_t levels) {
  return mul_kara_workspace(count, n, levels);
}

int bigint_mul_kara(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int32_t n,
                    int32_t levels, void *workspace, size_t workspace_bytes, void *stream) {
  if (count < 0 || count > 0x7fffffff || n < 1 || n > mul_max_limbs()) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  if (!a || !b || !out) return BIGINT_EINVAL;
  return launch_mul_kara(a, b, out, count, n, levels, workspace, workspace_bytes,
                         as_stream(stream));
}

int bigint_divmod_inv(const uint64_t *u, const uint64_t *v, const uint64_t *w, uint64_t *q,
                      uint64_t *r, int32_t *status, int64_t count, int32_t nu, int32_t nv,
                      int32_t nw, int32_t h, int64_t v_stride, int64_t w_stride,
                      void *workspace, size_t workspace_bytes, void *stream) {
  if (count < 0 || count > 0x7fffffff || nu < 1 || nv < 1 || nw < 1) return BIGINT_EINVAL;
  if (nu > BIGINT_MAX_LIMBS || nv > BIGINT_MAX_LIMBS) return BIGINT_EINVAL;
  if (h < nu || h < nv || h > 2 * BIGINT_MAX_LIMBS || nw > h + 1) return BIGINT_EINVAL;
  if (v_stride != 0 && v_stride != nv) return BIGINT_EINVAL;
  if (w_stride != 0 && w_stride != nw) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  if (!u || !v || !w || !q || !r) return BIGINT_EINVAL;
  if (workspace_bytes < divmod_workspace(count, nu, nv)) return BIGINT_ENOMEM;
  if (workspace_bytes > 0 && (!workspace || ((uintptr_t)workspace % 256) != 0))
    return BIGINT_EINVAL;
  return launch_divmod_inv(u, v, w, q, r, status, count, nu, nv, nw, h, v_stride, w_stride,
                           workspace, as_stream(stream));
}

size_t bigint_divmod_workspace(int64_t count, int32_t nu, int32_t nv) {
  if (count < 0 || nu < 1 || nv < 1) return 0;
  return divmod_workspace(count, nu, nv);
}

int bigint_divmod(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                  int32_t *status, int64_t count, int32_t nu, int32_t nv, void *workspace,
                  size_t workspace_bytes, void *stream) {
  if (count < 0 || count > 0x7fffffff || nu < 1 || nv < 1) return BIGINT_EINVAL;
  if (nu > BIGINT_MAX_LIMBS || nv > BIGINT_MAX_LIMBS) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  if (!u || !v || !q || !r) return BIGINT_EINVAL;
  if (workspace_bytes < divmod_workspace(count, nu, nv)) return BIGINT_ENOMEM;
  if (workspace_bytes > 0 && (!workspace || ((uintptr_t)workspace % 256) != 0))
    return BIGINT_EINVAL;
  return launch_divmod(u, v, q, r, status, count, nu, nv, workspace, workspace_bytes,
                       as_stream(stream));
}

size_t bigint_shinv_workspace(int64_t count, int32_t nv, int32_t h) {
  if (count < 0 || nv < 1 || h < 1) return 0;
  return shinv_workspace(count, nv, h);
}

int bigint_shinv(const uint64_t *v, uint64_t *w, int32_t *status, int64_t count, int32_t nv,
                 int32_t h, int32_t nw, void *workspace, size_t workspace_bytes,
                 void *stream) {
  if (count < 0 || count > 0x7fffffff || nv < 1 || nw < 1) return BIGINT_EINVAL;
  if (nv > BIGINT_MAX_LIMBS || h < nv || h > 2 * BIGINT_MAX_LIMBS) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  if (!v || !w) return BIGINT_EINVAL;
  if (workspace_bytes < shinv_workspace(count, nv, h)) return BIGINT_ENOMEM;
  if (workspace_bytes > 0 && (!workspace || ((uintptr_t)workspace % 256) != 0))
    return BIGINT_EINVAL;
  return launch_shinv(v, w, status, count, nv, h, nw, workspace, workspace_bytes,
                      as_stream(stream));
}

int bigint_batch_create(const bigint_op *ops_host, int64_t nops, bigint_batch **batch) {
  return batch_create(ops_host, nops, batch);
}

size_t bigint_batch_workspace(const bigint_batch *batch) { return batch_workspace_bytes(batch); }

int bigint_batch_upload(bigint_batch *batch, void *workspace, size_t bytes, void *stream) {
  if (!batch) return BIGINT_EINVAL;
  return batch_upload(batch, workspace, bytes, as_stream(stream));
}

int bigint_batch_launch(const bigint_batch *batch, const uint64_t *in_pool, uint64_t *out_pool,
                        int32_t *status, void *workspace, int mode, void *stream) {
  if (!batch) return BIGINT_EINVAL;
  return batch_launch(batch, in_pool, out_pool, status, workspace, mode, as_stream(stream));
}

int bigint_batch_tune(bigint_batch *batch, const uint64_t *in_pool, uint64_t *out_pool,
                      int32_t *status, void *workspace, size_t bytes, void *stream,
                      int *best_threads) {
  if (!batch || !in_pool || !out_pool) return BIGINT_EINVAL;
  return tune_batch(batch, in_pool, out_pool, status, workspace, bytes, as_stream(stream),
                    best_threads);
}

void bigint_batch_destroy(bigint_batch *batch) { batch_destroy(batch); }

int bigint_tune(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count,
                    int32_t na, int32_t nb, void *stream, int *best_variant) {
  if (count < 1 || count > 0x7fffffff || na < 1 || nb < 1) return BIGINT_EINVAL;
  if (na > mul_max_limbs() || nb > mul_max_limbs() || !a || !b || !out) return BIGINT_EINVAL;
  return tune_mul(a, b, out, count, na, nb, as_stream(stream), best_variant);
}

int bigint_save_tuning(const char *path) { return path ? tuning_save(path) : BIGINT_EINVAL; }
int bigint_load_tuning(const char *path) { return path ? tuning_load(path) : BIGINT_EINVAL; }

int bigint_set_variant(int op, int variant) {
  if (op == 0) return mul_set_variant(variant);
  if (op == 1) return div_set_variant(variant);
  if (op == 2) return batch_set_variant(variant);
  return BIGINT_EINVAL;
}

size_t bigint_host_workspace(int op, int64_t chunk, int32_t na, int32_t nb) {
  return host_workspace(op, chunk, na, nb);
}

int bigint_add_host(const uint64_t *a, const uint64_t *b, uint64_t *out, uint8_t *carry_out,
                    int64_t count, int32_t n, void *workspace, size_t bytes) {
  return host_run(BIGINT_OP_ADD, a, b, out, nullptr, carry_out, count, n, n, workspace, bytes,
                  true);
}

int bigint_sub_host(const uint64_t *a, const uint64_t *b, uint64_t *out, uint8_t *borrow_out,
                    int64_t count, int32_t n, void *workspace, size_t bytes) {
  return host_run(BIGINT_OP_SUB, a, b, out, nullptr, borrow_out, count, n, n, workspace, bytes,
                  true);
}

int bigint_mul_host(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count,
                    int32_t na, int32_t nb, void *workspace, size_t bytes) {
  return host_run(BIGINT_OP_MUL, a, b, out, nullptr, nullptr, count, na, nb, workspace, bytes,
                  true);
}

int bigint_divmod_host(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                       int32_t *status, int64_t count, int32_t nu, int32_t nv,
                       void *workspace, size_t bytes) {
  return host_run(BIGINT_OP_DIVMOD, u, v, q, r, status, count, nu, nv, workspace, bytes, true);
}

int bigint_host_async(int op, const uint64_t *a, const uint64_t *b, uint64_t *out0,
                      uint64_t *out1, void *aux, int64_t count, int32_t na, int32_t nb,
                      void *workspace, size_t bytes) {
  return host_run(op, a, b, out0, out1, aux, count, na, nb, workspace, bytes, false);
}

int bigint_host_sync(void) { return host_sync(); }

int bigint_check_timeout(void) {
  // every translation unit that launches tensor-core products keeps its own
  // record: ask them all (each read clears it)
  const int rc[4] = {tc_take_timeout(), div_take_timeout(), programs_take_timeout(),
                     batch_take_timeout()};
  int out = BIGINT_OK;
  for (int x : rc) {
    if (x == BIGINT_ECUDA) return BIGINT_ECUDA;
    if (x != BIGINT_OK) out = x;
  }
  return out;
}

unsigned long long bigint_kernel_launches(void) {
  return g_kernel_launches.load(std::memory_order_relaxed);
}

int bigint_set_wait_limit(long long cycles) {
  const int rc[4] = {tc_set_wait_limit(cycles), div_set_wait_limit(cycles),
                     programs_set_wait_limit(cycles), batch_set_wait_limit(cycles)};
  for (int x : rc)
    if (x != BIGINT_OK) return x;
  return BIGINT_OK;
}

int bigint_add_chain(const uint64_t *a, const uint64_t *b, uint64_t *out, uint8_t *carry_out,
                     int64_t count, int32_t n, int32_t k, void *stream) {
  int rc = check_addsub(a, b, out, count, n);
  if (rc != BIGINT_OK) return rc;
  if (k < 1 || k > 255) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  return launch_add_chain(a, b, out, carry_out, count, n, k, as_stream(stream));
}

size_t bigint_poly_workspace(int64_t count, int32_t n) {
  if (count < 0 || n < 1 || n > BIGINT_MUL_MAX_LIMBS) return 0;
  return poly_workspace(count, n);
}

int bigint_poly(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int32_t n,
                void *workspace, size_t bytes, void *stream) {
  if (count < 0 || count > 0x7fffffff || n < 1 || n > BIGINT_MUL_MAX_LIMBS) return BIGINT_EINVAL;
  if (count == 0) return BIGINT_OK;
  if (!a || !b || !out || !workspace) return BIGINT_EINVAL;
  return launch_poly(a, b, out, count, n, workspace, bytes, as_stream(stream));
}

int bigint_mul_variant_for(int32_t na, int32_t nb) {
  if (na < 1 || nb < 1) return BIGINT_EINVAL;
  return mul_variant_for(na, nb, na + nb);
}

int bigint_probe_int_throughput(int variant, double *ops_per_clk_sm, double *sm_mhz) {
  if (!ops_per_clk_sm || !sm_mhz) return BIGINT_EINVAL;
  return probe_int_throughput(variant, ops_per_clk_sm, sm_mhz);
}

}  // extern "C"
