// views.cu -- the per-operation ragged forms of the boundary
// (bigint_batch_add / _sub / _mul / _divmod over bigint_batch_cview and
// bigint_batch_view) and the one-call mixed-op form (bigint_batch_run).
//
// Host code only: each call turns its views into the operation descriptors
// of the batched form (bigint_op, batch.cu) -- one input and one output pool
// whose offsets are the distances of the instances' limbs from the lowest
// view base -- plans them, copies the plan into the caller's workspace and
// enqueues the persistent launch.  So a ragged call runs exactly the kernels
// (and block routines) of the batched form; its results do not depend on
// which form it came through.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace bigint {
int batch_create(const bigint_op *ops, int64_t nops, bigint_batch **out);
size_t batch_workspace_bytes(const bigint_batch *B);
int batch_upload(bigint_batch *B, void *ws, size_t bytes, cudaStream_t st);
int batch_launch(const bigint_batch *B, const uint64_t *in, uint64_t *out, int32_t *status,
                 void *ws, int mode, cudaStream_t st);
void batch_destroy(bigint_batch *B);

namespace {

// Instance i of a view: offset (limbs from its data) and length.
template <class V>
int64_t v_off(const V &v, int64_t i) {
  return v.offset ? v.offset[i] : i * (int64_t)v.n;
}
template <class V>
int32_t v_len(const V &v, int64_t i) {
  return v.nlimbs ? v.nlimbs[i] : v.n;
}

template <class V>
bool v_valid(const V *v) {
  if (!v || v->count < 0 || !v->data) return false;
  if ((reinterpret_cast<uintptr_t>(v->data) % 8) != 0) return false;
  if (!v->nlimbs && v->n < 1) return false;
  for (int64_t i = 0; i < v->count; i++) {
    const int32_t n = v_len(*v, i);
    if (n < 1 || n > BIGINT_MAX_LIMBS || v_off(*v, i) < 0) return false;
  }
  return true;
}

// Distance in limbs from base to p (both 8-byte aligned device addresses).
int64_t limbs_from(const void *base, const void *p) {
  return (int64_t)((reinterpret_cast<uintptr_t>(p) - reinterpret_cast<uintptr_t>(base)) / 8);
}

// The descriptors of an operation over views; returns BIGINT_OK or
// BIGINT_EINVAL (lengths that do not match the operation, bad views).
int build_ops(int op, const bigint_batch_cview *a, const bigint_batch_cview *b,
              const bigint_batch_view *o1, const bigint_batch_view *o2, int flags,
              std::vector<bigint_op> &ops, const uint64_t **in_base, uint64_t **out_base) {
  if (!v_valid(a) || !v_valid(b) || !v_valid(o1)) return BIGINT_EINVAL;
  if (op == BIGINT_OP_DIVMOD && !v_valid(o2)) return BIGINT_EINVAL;
  if (flags & ~BIGINT_ZEXT) return BIGINT_EINVAL;
  if ((flags & BIGINT_ZEXT) && op != BIGINT_OP_ADD && op != BIGINT_OP_SUB) return BIGINT_EINVAL;
  const int64_t count = a->count;
  if (b->count != count || o1->count != count || (o2 && o2->count != count))
    return BIGINT_EINVAL;
  const uint64_t *ib = std::min(a->data, b->data);
  uint64_t *ob = o2 ? std::min(o1->data, o2->data) : o1->data;
  const int64_t da = limbs_from(ib, a->data), db = limbs_from(ib, b->data);
  const int64_t d1 = limbs_from(ob, o1->data), d2 = o2 ? limbs_from(ob, o2->data) : 0;
  ops.resize(count);
  for (int64_t i = 0; i < count; i++) {
    const int32_t na = v_len(*a, i), nb = v_len(*b, i), n1 = v_len(*o1, i);
    bigint_op &x = ops[i];
    x.op = op;
    x.na = na;
    x.nb = nb;
    x.flags = flags;
    x.a = da + v_off(*a, i);
    x.b = db + v_off(*b, i);
    x.o1 = d1 + v_off(*o1, i);
    x.o2 = 0;
    switch (op) {
      case BIGINT_OP_ADD:
      case BIGINT_OP_SUB:
        if (na != nb && !(flags & BIGINT_ZEXT)) return BIGINT_EINVAL;
        if (n1 != std::max(na, nb)) return BIGINT_EINVAL;
        break;
      case BIGINT_OP_MUL:
        if (na > BIGINT_MUL_MAX_LIMBS || nb > BIGINT_MUL_MAX_LIMBS || n1 != na + nb)
          return BIGINT_EINVAL;
        break;
      default: {  // divmod: q max(nu - nv + 1, 1) limbs, r nv limbs
        const int32_t nq = std::max(na - nb + 1, 1);
        if (n1 != nq || v_len(*o2, i) != nb) return BIGINT_EINVAL;
        x.o2 = d2 + v_off(*o2, i);
      }
    }
  }
  *in_base = ib;
  *out_base = ob;
  return BIGINT_OK;
}

// Plans, uploads and launches a descriptor array (persistent form).
int run_ops(const std::vector<bigint_op> &ops, const uint64_t *in, uint64_t *out,
            int32_t *status, void *ws, size_t bytes, int mode, cudaStream_t st) {
  if (ops.empty()) return BIGINT_OK;
  bigint_batch *B = nullptr;
  int rc = batch_create(ops.data(), (int64_t)ops.size(), &B);
  if (rc != BIGINT_OK) return rc;
  if (bytes < batch_workspace_bytes(B)) {
    batch_destroy(B);
    return BIGINT_ENOMEM;
  }
  rc = batch_upload(B, ws, bytes, st);
  if (rc == BIGINT_OK) rc = batch_launch(B, in, out, status, ws, mode, st);
  // the plan's descriptor copies were staged from host memory by the time
  // upload returned (pageable source), so the plan can go now
  batch_destroy(B);
  return rc;
}

size_t ops_workspace(const std::vector<bigint_op> &ops) {
  if (ops.empty()) return 0;
  bigint_batch *B = nullptr;
  if (batch_create(ops.data(), (int64_t)ops.size(), &B) != BIGINT_OK) return 0;
  const size_t b = batch_workspace_bytes(B);
  batch_destroy(B);
  return b;
}

int views_call(int op, const bigint_batch_cview *a, const bigint_batch_cview *b,
               const bigint_batch_view *o1, const bigint_batch_view *o2, int32_t *status,
               int flags, void *ws, size_t bytes, void *stream) {
  if (a && a->count == 0 && b && b->count == 0) return BIGINT_OK;
  std::vector<bigint_op> ops;
  const uint64_t *in = nullptr;
  uint64_t *out = nullptr;
  const int rc = build_ops(op, a, b, o1, o2, flags, ops, &in, &out);
  if (rc != BIGINT_OK) return rc;
  return run_ops(ops, in, out, status, ws, bytes, BIGINT_BATCH_PERSISTENT,
                 reinterpret_cast<cudaStream_t>(stream));
}

}  // namespace
}  // namespace bigint

using namespace bigint;

extern "C" {

size_t bigint_batch_views_workspace(int op, const bigint_batch_cview *a,
                                    const bigint_batch_cview *b) {
  if (op < BIGINT_OP_ADD || op > BIGINT_OP_DIVMOD || !v_valid(a) || !v_valid(b) ||
      a->count != b->count)
    return 0;
  std::vector<bigint_op> ops(a->count);
  for (int64_t i = 0; i < a->count; i++) {
    bigint_op &x = ops[i];
    x.op = op;
    x.na = v_len(*a, i);
    x.nb = v_len(*b, i);
    x.flags = (op == BIGINT_OP_ADD || op == BIGINT_OP_SUB) && x.na != x.nb ? BIGINT_ZEXT : 0;
    x.a = x.b = x.o1 = x.o2 = 0;
  }
  return ops_workspace(ops);
}

int bigint_batch_add(const bigint_batch_cview *a, const bigint_batch_cview *b,
                     const bigint_batch_view *out, int32_t *carry_out, int flags,
                     void *workspace, size_t bytes, void *stream) {
  return views_call(BIGINT_OP_ADD, a, b, out, nullptr, carry_out, flags, workspace, bytes,
                    stream);
}

int bigint_batch_sub(const bigint_batch_cview *a, const bigint_batch_cview *b,
                     const bigint_batch_view *out, int32_t *borrow_out, int flags,
                     void *workspace, size_t bytes, void *stream) {
  return views_call(BIGINT_OP_SUB, a, b, out, nullptr, borrow_out, flags, workspace, bytes,
                    stream);
}

int bigint_batch_mul(const bigint_batch_cview *a, const bigint_batch_cview *b,
                     const bigint_batch_view *out, void *workspace, size_t bytes, void *stream) {
  return views_call(BIGINT_OP_MUL, a, b, out, nullptr, nullptr, 0, workspace, bytes, stream);
}

int bigint_batch_divmod(const bigint_batch_cview *u, const bigint_batch_cview *v,
                        const bigint_batch_view *q, const bigint_batch_view *r, int32_t *status,
                        void *workspace, size_t bytes, void *stream) {
  return views_call(BIGINT_OP_DIVMOD, u, v, q, r, status, 0, workspace, bytes, stream);
}

size_t bigint_batch_run_workspace(const bigint_op *ops, int64_t nops) {
  if (nops < 0 || (nops > 0 && !ops)) return 0;
  return ops_workspace(std::vector<bigint_op>(ops, ops + nops));
}

int bigint_batch_run(const bigint_op *ops, int64_t nops, const uint64_t *in_pool,
                     uint64_t *out_pool, int32_t *status, void *workspace, size_t bytes, int mode,
                     void *stream) {
  if (nops < 0 || (nops > 0 && (!ops || !in_pool || !out_pool))) return BIGINT_EINVAL;
  if (mode != BIGINT_BATCH_PERSISTENT && mode != BIGINT_BATCH_PER_CLASS &&
      mode != BIGINT_BATCH_STEPS)
    return BIGINT_EINVAL;
  return run_ops(std::vector<bigint_op>(ops, ops + nops), in_pool, out_pool, status, workspace,
                 bytes, mode, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
