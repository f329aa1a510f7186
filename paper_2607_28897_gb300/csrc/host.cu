// host.cu -- operations on operands in host memory, with copies and kernels
// overlapped.
//
// A call splits its batch into chunks and runs three library streams: copy
// in (host -> device), compute (the uniform-batch kernel of the operation)
// and copy out (device -> host).  Chunk i uses staging slot i % 2 of the
// caller's device workspace (as many slots as it holds, up to one per chunk
// and MAX_SLOTS), so chunk i+1 is copied in while chunk i is computed and
// chunk i-1 is copied out; events order the three streams per slot.  The plain call returns when every result is in host memory; the
// _async form only enqueues, so the copies of one call overlap the kernels
// of the next, and bigint_host_sync() waits for everything enqueued.  A
// call's first copy-in waits for every earlier call whose workspace range
// overlaps its own (a ring of the last calls' ranges and completion events),
// so calls may share workspaces in any shapes.  With pinned
// host buffers (cudaHostAlloc / cudaHostRegister) the copies run
// asynchronously on the copy engines; pageable buffers still give correct
// results, without the overlap.
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "bigint.h"
#include "common.cuh"

namespace bigint {

int launch_addsub(bool sub, const uint64_t *a, const uint64_t *b, uint64_t *out,
                  uint8_t *carry_out, int64_t count, int n, cudaStream_t st);
int launch_mul(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int na,
               int nb, int nout, cudaStream_t st);
int launch_divmod(const uint64_t *u, const uint64_t *v, uint64_t *q, uint64_t *r,
                  int32_t *status, int64_t count, int nu, int nv, void *ws, size_t bytes,
                  cudaStream_t st);
size_t divmod_workspace(int64_t count, int nu, int nv);
int kara_levels(int n, int levels);
size_t mul_kara_workspace(int64_t count, int n, int levels);
int launch_mul_kara(const uint64_t *a, const uint64_t *b, uint64_t *out, int64_t count, int n,
                    int levels, void *ws, size_t bytes, cudaStream_t st);
int mul_max_limbs();

namespace {

constexpr size_t ALIGN = 256;
constexpr int MAX_DEVICES = 64;

size_t align_up(size_t x) { return (x + ALIGN - 1) / ALIGN * ALIGN; }

// Per-instance sizes of one operation (limbs, and bytes of the small
// per-instance output: carry or status).
struct Shape {
  int op;             // BIGINT_OP_ADD, _SUB, _MUL, _DIVMOD
  int na, nb;         // input limbs
  int no0, no1;       // output limbs (result / quotient, remainder)
  int aux;            // bytes per instance of carry (add/sub) or status (divmod)
};

Shape shape_of(int op, int na, int nb) {
  Shape s{op, na, nb, 0, 0, 0};
  switch (op) {
    case BIGINT_OP_ADD:
    case BIGINT_OP_SUB: s.no0 = na; s.aux = 1; break;
    case BIGINT_OP_MUL: s.no0 = na + nb; break;
    default: s.no0 = na - nb + 1 > 1 ? na - nb + 1 : 1; s.no1 = nb; s.aux = 4; break;
  }
  return s;
}

// Square products of the sizes where bigint_mul_kara's measured choice runs
// Karatsuba levels take that form here too (with its workspace in the slot).
bool kara_form(const Shape &s) {
  return s.op == BIGINT_OP_MUL && s.na == s.nb && kara_levels(s.na, -1) > 0;
}

// Device bytes of one staging slot for `c` instances.
size_t slot_bytes(const Shape &s, int64_t c) {
  size_t b = align_up(8 * (size_t)c * s.na) + align_up(8 * (size_t)c * s.nb) +
             align_up(8 * (size_t)c * s.no0);
  if (s.no1) b += align_up(8 * (size_t)c * s.no1);
  if (s.aux) b += align_up((size_t)c * s.aux);
  if (s.op == BIGINT_OP_DIVMOD) b += align_up(divmod_workspace(c, s.na, s.nb));
  if (kara_form(s)) b += align_up(mul_kara_workspace(c, s.na, -1));
  return b;
}

struct Slot {
  uint64_t *in0, *in1, *out0, *out1;
  void *aux, *ws;
  size_t ws_bytes;
};

Slot carve_slot(const Shape &s, int64_t c, uint8_t *base) {
  Slot sl{};
  uint8_t *p = base;
  sl.in0 = reinterpret_cast<uint64_t *>(p); p += align_up(8 * (size_t)c * s.na);
  sl.in1 = reinterpret_cast<uint64_t *>(p); p += align_up(8 * (size_t)c * s.nb);
  sl.out0 = reinterpret_cast<uint64_t *>(p); p += align_up(8 * (size_t)c * s.no0);
  if (s.no1) { sl.out1 = reinterpret_cast<uint64_t *>(p); p += align_up(8 * (size_t)c * s.no1); }
  if (s.aux) { sl.aux = p; p += align_up((size_t)c * s.aux); }
  if (s.op == BIGINT_OP_DIVMOD) {
    sl.ws = p;
    sl.ws_bytes = divmod_workspace(c, s.na, s.nb);
  }
  if (kara_form(s)) {
    sl.ws = p;
    sl.ws_bytes = mul_kara_workspace(c, s.na, -1);
  }
  return sl;
}

// The three streams and the per-slot events of one device (created on first
// use, kept for the process), and the workspace ranges of the last calls
// with the events that mark their last copy-out.
constexpr int RING = 16;
constexpr int MAX_SLOTS = 8;
struct Pipe {
  bool ready = false;
  cudaStream_t in, comp, out;
  cudaEvent_t loaded[MAX_SLOTS], done[MAX_SLOTS], freed[MAX_SLOTS];
  cudaEvent_t finished[RING];
  uintptr_t lo[RING] = {}, hi[RING] = {};  // empty range: never recorded
  int next = 0;
};
Pipe g_pipe[MAX_DEVICES];

int get_pipe(Pipe **pp) {
  int dev = 0;
  BIGINT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return BIGINT_EINVAL;
  Pipe &p = g_pipe[dev];
  if (!p.ready) {
    BIGINT_CUDA_TRY(cudaStreamCreateWithFlags(&p.in, cudaStreamNonBlocking));
    BIGINT_CUDA_TRY(cudaStreamCreateWithFlags(&p.comp, cudaStreamNonBlocking));
    BIGINT_CUDA_TRY(cudaStreamCreateWithFlags(&p.out, cudaStreamNonBlocking));
    for (int i = 0; i < MAX_SLOTS; i++) {
      BIGINT_CUDA_TRY(cudaEventCreateWithFlags(&p.loaded[i], cudaEventDisableTiming));
      BIGINT_CUDA_TRY(cudaEventCreateWithFlags(&p.done[i], cudaEventDisableTiming));
      BIGINT_CUDA_TRY(cudaEventCreateWithFlags(&p.freed[i], cudaEventDisableTiming));
    }
    for (int i = 0; i < RING; i++)
      BIGINT_CUDA_TRY(cudaEventCreateWithFlags(&p.finished[i], cudaEventDisableTiming));
    p.ready = true;
  }
  *pp = &p;
  return BIGINT_OK;
}

// Divisions in chunks of fewer instances than this run each Newton step's
// products on too few SMs (measured: 256 divisions of 2^20 by 2^19 bits in
// four chunks of 64 took 9.7 ms through this path against 4.3 ms in one
// launch), so a division chunk holds at least this many (or the batch).
constexpr int64_t MIN_DIV_CHUNK = 1024;

// Instances per chunk: what two slots of the workspace hold, and at most a
// quarter of the batch (so that copies and kernels of different chunks
// overlap) -- for divisions at least MIN_DIV_CHUNK -- at least 1.
int64_t chunk_size(const Shape &s, int64_t count, size_t bytes) {
  int64_t hi = (count + 3) / 4;
  if (s.op == BIGINT_OP_DIVMOD && hi < MIN_DIV_CHUNK) hi = count < MIN_DIV_CHUNK ? count : MIN_DIV_CHUNK;
  if (hi < 1) hi = 1;
  int64_t lo = 0;  // largest c with 2 slot_bytes(c) <= bytes
  int64_t a = 1, b = count;
  while (a <= b) {
    const int64_t m = a + (b - a) / 2;
    if (2 * slot_bytes(s, m) <= bytes) { lo = m; a = m + 1; } else { b = m - 1; }
  }
  return lo < hi ? lo : hi;
}

int run(const Shape &s, const uint64_t *in0, const uint64_t *in1, uint64_t *out0, uint64_t *out1,
        void *aux, int64_t count, void *workspace, size_t bytes, bool sync) {
  if (count == 0) return BIGINT_OK;
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) % ALIGN) != 0) return BIGINT_EINVAL;
  const int64_t c = chunk_size(s, count, bytes);
  if (c < 1) return BIGINT_ENOMEM;
  Pipe *p = nullptr;
  int rc = get_pipe(&p);
  if (rc != BIGINT_OK) return rc;
  uint8_t *ws = static_cast<uint8_t *>(workspace);
  const int64_t nchunks = (count + c - 1) / c;
  const size_t sb = slot_bytes(s, c);
  int64_t ns = (int64_t)(bytes / sb);  // staging slots: >= 2 (chunk_size), <= chunks, <= MAX_SLOTS
  if (ns > nchunks) ns = nchunks;
  if (ns > MAX_SLOTS) ns = MAX_SLOTS;
  if (ns < 1) ns = 1;
  Slot slots[MAX_SLOTS];
  for (int64_t k = 0; k < ns; k++) slots[k] = carve_slot(s, c, ws + k * sb);
  // earlier calls that used any of this call's workspace must be done with it;
  // the ring entry about to be reused is waited for too (its range is dropped)
  const uintptr_t wlo = reinterpret_cast<uintptr_t>(ws), whi = wlo + (size_t)ns * sb;
  for (int e = 0; e < RING; e++)
    if ((p->lo[e] < whi && wlo < p->hi[e]) || (e == p->next && p->hi[e] > p->lo[e]))
      BIGINT_CUDA_TRY(cudaStreamWaitEvent(p->in, p->finished[e], 0));
  for (int64_t i = 0; i < nchunks && rc == BIGINT_OK; i++) {
    const int k = (int)(i % ns);
    const Slot &sl = slots[k];
    const int64_t i0 = i * c, m = count - i0 < c ? count - i0 : c;
    // copy in, once the slot's previous results (this call) have been copied out
    if (i >= ns) BIGINT_CUDA_TRY(cudaStreamWaitEvent(p->in, p->freed[k], 0));
    BIGINT_CUDA_TRY(cudaMemcpyAsync(sl.in0, in0 + i0 * s.na, 8 * (size_t)m * s.na,
                                    cudaMemcpyHostToDevice, p->in));
    BIGINT_CUDA_TRY(cudaMemcpyAsync(sl.in1, in1 + i0 * s.nb, 8 * (size_t)m * s.nb,
                                    cudaMemcpyHostToDevice, p->in));
    BIGINT_CUDA_TRY(cudaEventRecord(p->loaded[k], p->in));
    // compute
    BIGINT_CUDA_TRY(cudaStreamWaitEvent(p->comp, p->loaded[k], 0));
    switch (s.op) {
      case BIGINT_OP_ADD:
      case BIGINT_OP_SUB:
        rc = launch_addsub(s.op == BIGINT_OP_SUB, sl.in0, sl.in1, sl.out0,
                           static_cast<uint8_t *>(sl.aux), m, s.na, p->comp);
        break;
      case BIGINT_OP_MUL:
        rc = kara_form(s) ? launch_mul_kara(sl.in0, sl.in1, sl.out0, m, s.na, -1, sl.ws,
                                            sl.ws_bytes, p->comp)
                          : launch_mul(sl.in0, sl.in1, sl.out0, m, s.na, s.nb, s.na + s.nb,
                                       p->comp);
        break;
      default:
        rc = launch_divmod(sl.in0, sl.in1, sl.out0, sl.out1, static_cast<int32_t *>(sl.aux), m,
                           s.na, s.nb, sl.ws, sl.ws_bytes, p->comp);
        break;
    }
    BIGINT_CUDA_TRY(cudaEventRecord(p->done[k], p->comp));
    // copy out
    BIGINT_CUDA_TRY(cudaStreamWaitEvent(p->out, p->done[k], 0));
    BIGINT_CUDA_TRY(cudaMemcpyAsync(out0 + i0 * s.no0, sl.out0, 8 * (size_t)m * s.no0,
                                    cudaMemcpyDeviceToHost, p->out));
    if (s.no1 && out1)
      BIGINT_CUDA_TRY(cudaMemcpyAsync(out1 + i0 * s.no1, sl.out1, 8 * (size_t)m * s.no1,
                                      cudaMemcpyDeviceToHost, p->out));
    if (s.aux && aux)
      BIGINT_CUDA_TRY(cudaMemcpyAsync(static_cast<uint8_t *>(aux) + i0 * s.aux, sl.aux,
                                      (size_t)m * s.aux, cudaMemcpyDeviceToHost, p->out));
    BIGINT_CUDA_TRY(cudaEventRecord(p->freed[k], p->out));
  }
  if (rc == BIGINT_OK) {  // this call's workspace range is free once its last copy-out is done
    BIGINT_CUDA_TRY(cudaEventRecord(p->finished[p->next], p->out));
    p->lo[p->next] = wlo;
    p->hi[p->next] = whi;
    p->next = (p->next + 1) % RING;
  }
  if (!sync && rc == BIGINT_OK) return BIGINT_OK;
  const cudaError_t e = cudaStreamSynchronize(p->out);
  if (rc != BIGINT_OK) {
    cudaStreamSynchronize(p->comp);
    cudaStreamSynchronize(p->in);
    return rc;
  }
  return e == cudaSuccess ? BIGINT_OK : BIGINT_ECUDA;
}

bool shape_ok(int op, int64_t count, int na, int nb) {
  if (count < 0 || count > 0x7fffffff || na < 1 || nb < 1) return false;
  switch (op) {
    case BIGINT_OP_ADD:
    case BIGINT_OP_SUB: return na == nb && na <= BIGINT_MAX_LIMBS;
    case BIGINT_OP_MUL: return na <= mul_max_limbs() && nb <= mul_max_limbs();
    case BIGINT_OP_DIVMOD: return na <= BIGINT_MAX_LIMBS && nb <= BIGINT_MAX_LIMBS;
    default: return false;
  }
}

}  // namespace

size_t host_workspace(int op, int64_t chunk, int na, int nb) {
  if (!shape_ok(op, chunk, na, nb) || chunk < 1) return 0;
  return 2 * slot_bytes(shape_of(op, na, nb), chunk);
}

int host_run(int op, const uint64_t *in0, const uint64_t *in1, uint64_t *out0, uint64_t *out1,
             void *aux, int64_t count, int na, int nb, void *workspace, size_t bytes, bool sync) {
  if (!shape_ok(op, count, na, nb)) return BIGINT_EINVAL;
  if (count > 0 && (!in0 || !in1 || !out0)) return BIGINT_EINVAL;
  if (op == BIGINT_OP_DIVMOD && count > 0 && !out1) return BIGINT_EINVAL;
  return run(shape_of(op, na, nb), in0, in1, out0, out1, aux, count, workspace, bytes, sync);
}

int host_sync() {
  Pipe *p = nullptr;
  const int rc = get_pipe(&p);
  if (rc != BIGINT_OK) return rc;
  const cudaError_t a = cudaStreamSynchronize(p->in), b = cudaStreamSynchronize(p->comp),
                    c = cudaStreamSynchronize(p->out);
  return (a == cudaSuccess && b == cudaSuccess && c == cudaSuccess) ? BIGINT_OK : BIGINT_ECUDA;
}

}  // namespace bigint
