"""Batched exact arithmetic on midsize unsigned integers on one GB300.

Thin Python binding over the C ABI of ``libbigint.so`` (``include/bigint.h``):
argument marshalling only.  Every arithmetic step runs in the CUDA kernels of
``csrc/``; PyTorch is used for device memory and streams.  There is no CPU
fallback: if the library is missing or no GPU is present, calls raise.

Integers are little-endian arrays of 64-bit limbs.  A batch is a CUDA tensor
of shape ``(count, n)`` and dtype ``torch.uint64`` or ``torch.int64`` (the
bits are what matter), contiguous, instance-major.
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "BigIntError", "load", "add", "sub", "mul", "mul_lo", "mul_split", "mul_split_workspace_bytes",
    "mul_kara", "mul_kara_workspace_bytes",
    "divmod", "divmod_noalloc", "divmod_inv", "shinv",
    "divmod_workspace_bytes", "shinv_workspace_bytes", "probe_int_throughput", "set_variant",
    "set_wait_limit", "check_timeout",
    "host_workspace_bytes", "add_host", "sub_host", "mul_host", "divmod_host", "host_sync",
    "add_chain", "poly", "poly_workspace_bytes",
    "OK", "EINVAL", "EDIVZERO", "ENOMEM", "ETIMEOUT", "EINTERNAL", "ECUDA", "ERANGE",
    "MAX_LIMBS", "MUL_MAX_LIMBS",
]

OK, EINVAL, EDIVZERO, ENOMEM, ETIMEOUT, EINTERNAL, ECUDA, ERANGE = 0, -1, -2, -3, -4, -5, -6, -7
OP_ADD, OP_SUB, OP_MUL, OP_DIVMOD = 1, 2, 3, 4
BATCH_PERSISTENT, BATCH_PER_CLASS, BATCH_STEPS = 0, 1, 2
MAX_LIMBS = 16384
MUL_MAX_LIMBS = 10000

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbigint.so")

# Every symbol include/bigint.h declares, with its ctypes signature.
_P, _I64, _I32, _SZ = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_size_t
SIGNATURES = {
    "bigint_strerror": ([ctypes.c_int], ctypes.c_char_p),
    "bigint_version": ([], ctypes.c_int),
    "bigint_add": ([_P, _P, _P, _P, _I64, _I32, _P], ctypes.c_int),
    "bigint_sub": ([_P, _P, _P, _P, _I64, _I32, _P], ctypes.c_int),
    "bigint_mul": ([_P, _P, _P, _I64, _I32, _I32, _P], ctypes.c_int),
    "bigint_mul_lo": ([_P, _P, _P, _I64, _I32, _I32, _I32, _P], ctypes.c_int),
    "bigint_mul_split": ([_P, _P, _P, _I64, _I32, _I32, _P, _SZ, _P], ctypes.c_int),
    "bigint_mul_kara_workspace": ([_I64, _I32, _I32], ctypes.c_size_t),
    "bigint_mul_kara": ([_P, _P, _P, _I64, _I32, _I32, _P, _SZ, _P], ctypes.c_int),
    "bigint_mul_split_workspace": ([_I64, _I32, _I32], _SZ),
    "bigint_divmod": ([_P, _P, _P, _P, _P, _I64, _I32, _I32, _P, _SZ, _P], ctypes.c_int),
    "bigint_divmod_workspace": ([_I64, _I32, _I32], _SZ),
    "bigint_divmod_noalloc": ([_P, _P, _P, _P, _P, _I64, _I32, _I32, _P], ctypes.c_int),
    "bigint_divmod_noalloc_scratch_bytes": ([], _SZ),
    "bigint_shinv": ([_P, _P, _P, _I64, _I32, _I32, _I32, _P, _SZ, _P], ctypes.c_int),
    "bigint_shinv_workspace": ([_I64, _I32, _I32], _SZ),
    "bigint_divmod_inv": ([_P, _P, _P, _P, _P, _P, _I64, _I32, _I32, _I32, _I32, _I64, _I64, _P,
                           _SZ, _P], ctypes.c_int),
    "bigint_batch_create": ([_P, _I64, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "bigint_batch_workspace": ([_P], _SZ),
    "bigint_batch_upload": ([_P, _P, _SZ, _P], ctypes.c_int),
    "bigint_batch_launch": ([_P, _P, _P, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "bigint_batch_tune": ([_P, _P, _P, _P, _P, _SZ, _P, ctypes.POINTER(ctypes.c_int)],
                          ctypes.c_int),
    "bigint_batch_destroy": ([_P], None),
    "bigint_batch_views_workspace": ([ctypes.c_int, _P, _P], _SZ),
    "bigint_batch_add": ([_P, _P, _P, _P, ctypes.c_int, _P, _SZ, _P], ctypes.c_int),
    "bigint_batch_sub": ([_P, _P, _P, _P, ctypes.c_int, _P, _SZ, _P], ctypes.c_int),
    "bigint_batch_mul": ([_P, _P, _P, _P, _SZ, _P], ctypes.c_int),
    "bigint_batch_divmod": ([_P, _P, _P, _P, _P, _P, _SZ, _P], ctypes.c_int),
    "bigint_batch_run_workspace": ([_P, _I64], _SZ),
    "bigint_batch_run": ([_P, _I64, _P, _P, _P, _P, _SZ, ctypes.c_int, _P], ctypes.c_int),
    "bigint_tune": ([_P, _P, _P, _I64, _I32, _I32, _P, ctypes.POINTER(ctypes.c_int)],
                        ctypes.c_int),
    "bigint_save_tuning": ([ctypes.c_char_p], ctypes.c_int),
    "bigint_load_tuning": ([ctypes.c_char_p], ctypes.c_int),
    "bigint_set_variant": ([ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "bigint_mul_variant_for": ([_I32, _I32], ctypes.c_int),
    "bigint_check_timeout": ([], ctypes.c_int),
    "bigint_set_wait_limit": ([ctypes.c_longlong], ctypes.c_int),
    "bigint_kernel_launches": ([], ctypes.c_ulonglong),
    "bigint_host_workspace": ([ctypes.c_int, _I64, _I32, _I32], _SZ),
    "bigint_add_chain": ([_P, _P, _P, _P, _I64, _I32, _I32, _P], ctypes.c_int),
    "bigint_poly_workspace": ([_I64, _I32], _SZ),
    "bigint_poly": ([_P, _P, _P, _I64, _I32, _P, _SZ, _P], ctypes.c_int),
    "bigint_add_host": ([_P, _P, _P, _P, _I64, _I32, _P, _SZ], ctypes.c_int),
    "bigint_sub_host": ([_P, _P, _P, _P, _I64, _I32, _P, _SZ], ctypes.c_int),
    "bigint_mul_host": ([_P, _P, _P, _I64, _I32, _I32, _P, _SZ], ctypes.c_int),
    "bigint_divmod_host": ([_P, _P, _P, _P, _P, _I64, _I32, _I32, _P, _SZ], ctypes.c_int),
    "bigint_host_async": ([ctypes.c_int, _P, _P, _P, _P, _P, _I64, _I32, _I32, _P, _SZ],
                          ctypes.c_int),
    "bigint_host_sync": ([], ctypes.c_int),
    "bigint_probe_int_throughput": ([ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
}


class BigIntError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


_lib = None


def load(path: str | None = None):
    """Load libbigint.so (built by ``build.py``).  Raises if it is missing."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(
            f"libbigint.so not found at {p}: build it with "
            "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    L = ctypes.CDLL(p)
    for name, (args, res) in SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    if path is None:
        _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return load().bigint_strerror(code).decode()
    except Exception:  # library unavailable: still give a readable message
        return {0: "ok", -1: "invalid argument", -2: "division by zero"}.get(code, "error")


def _check(rc: int, what: str) -> None:
    if rc != OK:
        raise BigIntError(rc, what)


def _torch():
    import torch

    return torch


def _dev_tensor(x, name: str):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if x.dtype not in (torch.uint64, torch.int64):
        raise TypeError(f"{name} must have dtype uint64 or int64")
    if x.dim() != 2 or not x.is_contiguous():
        raise ValueError(f"{name} must be a contiguous (count, n) tensor")
    return x


def _stream_ptr(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _empty_like_limbs(ref, count: int, n: int):
    torch = _torch()
    return torch.empty((count, n), dtype=ref.dtype, device=ref.device)


def add(a, b, out=None, carry=None, stream=None):
    """(a + b) mod B^n and the carry out per instance (uint8)."""
    return _addsub("bigint_add", a, b, out, carry, stream)


def sub(a, b, out=None, borrow=None, stream=None):
    """(a - b) mod B^n and the borrow out per instance (uint8, 1 iff a < b)."""
    return _addsub("bigint_sub", a, b, out, borrow, stream)


def _addsub(fn, a, b, out, flag, stream):
    torch = _torch()
    a, b = _dev_tensor(a, "a"), _dev_tensor(b, "b")
    if a.shape != b.shape:
        raise ValueError("a and b must have the same shape")
    count, n = a.shape
    out = _empty_like_limbs(a, count, n) if out is None else _dev_tensor(out, "out")
    if flag is None:
        flag = torch.empty(count, dtype=torch.uint8, device=a.device)
    rc = getattr(load(), fn)(a.data_ptr(), b.data_ptr(), out.data_ptr(), flag.data_ptr(),
                             count, n, _stream_ptr(stream))
    _check(rc, fn)
    return out, flag


def mul(a, b, out=None, stream=None):
    """Full product, (count, na + nb) limbs."""
    a, b = _dev_tensor(a, "a"), _dev_tensor(b, "b")
    count, na = a.shape
    nb = b.shape[1]
    if b.shape[0] != count:
        raise ValueError("batch sizes differ")
    out = _empty_like_limbs(a, count, na + nb) if out is None else _dev_tensor(out, "out")
    rc = load().bigint_mul(a.data_ptr(), b.data_ptr(), out.data_ptr(), count, na, nb,
                           _stream_ptr(stream))
    _check(rc, "bigint_mul")
    return out


def mul_kara_workspace_bytes(count: int, n: int, levels: int = -1) -> int:
    """Workspace bytes of bigint_mul_kara for one pass over the batch."""
    return int(load().bigint_mul_kara_workspace(count, n, levels))


def mul_kara(a, b, levels: int = -1, out=None, workspace=None, stream=None):
    """Full products of square operands by Karatsuba's method over the
    batched products (bit-identical to mul; levels -1: by size)."""
    a, b = _dev_tensor(a, "a"), _dev_tensor(b, "b")
    count, n = a.shape
    if b.shape != a.shape:
        raise BigIntError(EINVAL, "mul_kara: a and b must have the same shape")
    out = _empty_like_limbs(a, count, 2 * n) if out is None else _dev_tensor(out, "out")
    if workspace is None:
        workspace = _workspace(mul_kara_workspace_bytes(count, n, levels), a.device)
    rc = load().bigint_mul_kara(a.data_ptr(), b.data_ptr(), out.data_ptr(), count, n, levels,
                                workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                _stream_ptr(stream))
    _check(rc, "bigint_mul_kara")
    return out


def mul_split_workspace_bytes(count: int, na: int, nb: int) -> int:
    return int(load().bigint_mul_split_workspace(count, na, nb))


def mul_split(a, b, out=None, workspace=None, stream=None):
    """Full product as ``mul``, each product's output tiles on different CTAs
    (lower latency for few, large products)."""
    a, b = _dev_tensor(a, "a"), _dev_tensor(b, "b")
    count, na = a.shape
    nb = b.shape[1]
    if b.shape[0] != count:
        raise ValueError("batch sizes differ")
    out = _empty_like_limbs(a, count, na + nb) if out is None else _dev_tensor(out, "out")
    need = mul_split_workspace_bytes(count, na, nb)
    if workspace is None:
        workspace = _workspace(need, a.device)
    rc = load().bigint_mul_split(a.data_ptr(), b.data_ptr(), out.data_ptr(), count, na, nb,
                                 workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                                 _stream_ptr(stream))
    _check(rc, "bigint_mul_split")
    return out


def mul_lo(a, b, m: int, out=None, stream=None):
    """Low m limbs of the product (the product mod B^m)."""
    a, b = _dev_tensor(a, "a"), _dev_tensor(b, "b")
    count, na = a.shape
    nb = b.shape[1]
    out = _empty_like_limbs(a, count, m) if out is None else _dev_tensor(out, "out")
    rc = load().bigint_mul_lo(a.data_ptr(), b.data_ptr(), out.data_ptr(), count, na, nb, m,
                              _stream_ptr(stream))
    _check(rc, "bigint_mul_lo")
    return out


def divmod_workspace_bytes(count: int, nu: int, nv: int) -> int:
    return int(load().bigint_divmod_workspace(count, nu, nv))


def shinv_workspace_bytes(count: int, nv: int, h: int) -> int:
    return int(load().bigint_shinv_workspace(count, nv, h))


def _workspace(nbytes: int, device):
    torch = _torch()
    # torch's caching allocator returns blocks aligned to at least 512 bytes
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)


def divmod(u, v, q=None, r=None, status=None, workspace=None, stream=None):
    """q = floor(u / v) ((count, max(nu-nv+1, 1)) limbs), r = u mod v
    ((count, nv) limbs) and a per-instance int32 status."""
    torch = _torch()
    u, v = _dev_tensor(u, "u"), _dev_tensor(v, "v")
    count, nu = u.shape
    nv = v.shape[1]
    nq = max(nu - nv + 1, 1)
    q = _empty_like_limbs(u, count, nq) if q is None else _dev_tensor(q, "q")
    r = _empty_like_limbs(u, count, nv) if r is None else _dev_tensor(r, "r")
    if status is None:
        status = torch.empty(count, dtype=torch.int32, device=u.device)
    need = divmod_workspace_bytes(count, nu, nv)
    if workspace is None:
        workspace = _workspace(need, u.device)
    rc = load().bigint_divmod(u.data_ptr(), v.data_ptr(), q.data_ptr(), r.data_ptr(),
                              status.data_ptr(), count, nu, nv, workspace.data_ptr(),
                              workspace.numel() * workspace.element_size(),
                              _stream_ptr(stream))
    _check(rc, "bigint_divmod")
    return q, r, status


def divmod_noalloc(u, v, q=None, r=None, status=None, stream=None):
    """As divmod, with the library's own fixed scratch instead of a caller
    workspace (for callers that cannot allocate; see bigint.h)."""
    torch = _torch()
    u, v = _dev_tensor(u, "u"), _dev_tensor(v, "v")
    count, nu = u.shape
    nv = v.shape[1]
    nq = max(nu - nv + 1, 1)
    q = _empty_like_limbs(u, count, nq) if q is None else _dev_tensor(q, "q")
    r = _empty_like_limbs(u, count, nv) if r is None else _dev_tensor(r, "r")
    if status is None:
        status = torch.empty(count, dtype=torch.int32, device=u.device)
    rc = load().bigint_divmod_noalloc(u.data_ptr(), v.data_ptr(), q.data_ptr(), r.data_ptr(),
                                      status.data_ptr(), count, nu, nv, _stream_ptr(stream))
    _check(rc, "bigint_divmod_noalloc")
    return q, r, status


def divmod_inv(u, v, w, h: int, q=None, r=None, status=None, workspace=None, stream=None):
    """q, r and status as ``divmod``, from w = floor(B^h / v) (``shinv``),
    h >= nu.  v (nv limbs) and w (nw limbs) are (count, n) tensors, one per
    instance, or (1, n): one divisor and inverse for the whole batch."""
    torch = _torch()
    u, v, w = _dev_tensor(u, "u"), _dev_tensor(v, "v"), _dev_tensor(w, "w")
    count, nu = u.shape
    nv, nw = v.shape[1], w.shape[1]
    for t, name in ((v, "v"), (w, "w")):
        if t.shape[0] not in (1, count):
            raise ValueError(f"{name} must have 1 or {count} rows")
    vs = 0 if (v.shape[0] == 1 and count != 1) else nv
    ws_ = 0 if (w.shape[0] == 1 and count != 1) else nw
    nq = max(nu - nv + 1, 1)
    q = _empty_like_limbs(u, count, nq) if q is None else _dev_tensor(q, "q")
    r = _empty_like_limbs(u, count, nv) if r is None else _dev_tensor(r, "r")
    if status is None:
        status = torch.empty(count, dtype=torch.int32, device=u.device)
    need = divmod_workspace_bytes(count, nu, nv)
    if workspace is None:
        workspace = _workspace(need, u.device)
    rc = load().bigint_divmod_inv(u.data_ptr(), v.data_ptr(), w.data_ptr(), q.data_ptr(),
                                  r.data_ptr(), status.data_ptr(), count, nu, nv, nw, h, vs, ws_,
                                  workspace.data_ptr(),
                                  workspace.numel() * workspace.element_size(),
                                  _stream_ptr(stream))
    _check(rc, "bigint_divmod_inv")
    return q, r, status


def shinv(v, h: int, nw: int, w=None, status=None, workspace=None, stream=None):
    """w = floor(B^h / v), (count, nw) limbs, and a per-instance status."""
    torch = _torch()
    v = _dev_tensor(v, "v")
    count, nv = v.shape
    w = _empty_like_limbs(v, count, nw) if w is None else _dev_tensor(w, "w")
    if status is None:
        status = torch.empty(count, dtype=torch.int32, device=v.device)
    need = shinv_workspace_bytes(count, nv, h)
    if workspace is None:
        workspace = _workspace(need, v.device)
    rc = load().bigint_shinv(v.data_ptr(), w.data_ptr(), status.data_ptr(), count, nv, h, nw,
                             workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                             _stream_ptr(stream))
    _check(rc, "bigint_shinv")
    return w, status


# ---- fused programs (Sec. VI, Tables I and II) -------------------------------
def add_chain(a, b, k: int, out=None, carry=None, stream=None):
    """a + b + ... + b (k additions mod B^n, intermediates in registers);
    carry = floor((a + k b) / B^n) per instance (uint8) if given."""
    torch = _torch()
    a, b = _dev_tensor(a, "a"), _dev_tensor(b, "b")
    count, n = a.shape
    out = _empty_like_limbs(a, count, n) if out is None else _dev_tensor(out, "out")
    rc = load().bigint_add_chain(a.data_ptr(), b.data_ptr(), out.data_ptr(),
                                 carry.data_ptr() if carry is not None else None, count, n, k,
                                 _stream_ptr(stream))
    _check(rc, "bigint_add_chain")
    return out


def poly_workspace_bytes(count: int, n: int) -> int:
    return int(load().bigint_poly_workspace(count, n))


def poly(a, b, out=None, workspace=None, stream=None):
    """(a a + b)(b b + b) + a b mod B^n per instance, one fused launch."""
    a, b = _dev_tensor(a, "a"), _dev_tensor(b, "b")
    count, n = a.shape
    out = _empty_like_limbs(a, count, n) if out is None else _dev_tensor(out, "out")
    if workspace is None:
        workspace = _workspace(poly_workspace_bytes(count, n), a.device)
    rc = load().bigint_poly(a.data_ptr(), b.data_ptr(), out.data_ptr(), count, n,
                            workspace.data_ptr(), workspace.numel() * workspace.element_size(),
                            _stream_ptr(stream))
    _check(rc, "bigint_poly")
    return out


# ---- host-buffer entry points (copies overlapped with the kernels) ----------
def _host_tensor(x, name: str):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or x.device.type != "cpu" or x.dim() != 2:
        raise BigIntError(EINVAL, f"{name}: expected a 2-D CPU tensor of limbs (pinned for overlap)")
    if x.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)) or not x.is_contiguous():
        raise BigIntError(EINVAL, f"{name}: expected a contiguous int64/uint64 tensor")
    return x


def host_workspace_bytes(op: int, chunk: int, na: int, nb: int) -> int:
    return int(load().bigint_host_workspace(op, chunk, na, nb))


def _host_ws(op, count, na, nb, workspace, device):
    if workspace is not None:
        return workspace
    chunk = max(1, (count + 3) // 4)
    return _workspace(host_workspace_bytes(op, chunk, na, nb), device)


def _host_out(count, n, out):
    torch = _torch()
    return torch.empty((count, n), dtype=torch.int64).pin_memory() if out is None else out


def _host_call(op, a, b, out0, out1, aux, na, nb, ws, sync, name):
    count = a.shape[0]
    args = (a.data_ptr(), b.data_ptr(), out0.data_ptr(),
            out1.data_ptr() if out1 is not None else None,
            aux.data_ptr() if aux is not None else None, count, na, nb, ws.data_ptr(),
            ws.numel() * ws.element_size())
    if sync:
        L = load()
        if op in (OP_ADD, OP_SUB):
            fn = L.bigint_add_host if op == OP_ADD else L.bigint_sub_host
            rc = fn(args[0], args[1], args[2], args[4], count, na, args[8], args[9])
        elif op == OP_MUL:
            rc = L.bigint_mul_host(args[0], args[1], args[2], count, na, nb, args[8], args[9])
        else:
            rc = L.bigint_divmod_host(args[0], args[1], args[2], args[3], args[4], count, na, nb,
                                      args[8], args[9])
    else:
        rc = load().bigint_host_async(op, *args)
    _check(rc, name)


def add_host(a, b, out=None, carry=None, workspace=None, device="cuda", sync=True):
    """a + b for CPU (pinned) tensors: chunks copied in, added and copied
    back with the copies overlapping the kernels.  sync=False only enqueues
    (host_sync() waits)."""
    return _addsub_host(OP_ADD, a, b, out, carry, workspace, device, sync)


def sub_host(a, b, out=None, borrow=None, workspace=None, device="cuda", sync=True):
    return _addsub_host(OP_SUB, a, b, out, borrow, workspace, device, sync)


def _addsub_host(op, a, b, out, flag, workspace, device, sync):
    a, b = _host_tensor(a, "a"), _host_tensor(b, "b")
    count, n = a.shape
    out = _host_tensor(_host_out(count, n, out), "out")
    ws = _host_ws(op, count, n, n, workspace, device)
    _host_call(op, a, b, out, None, flag, n, n, ws, sync,
               "bigint_add_host" if op == OP_ADD else "bigint_sub_host")
    return out


def mul_host(a, b, out=None, workspace=None, device="cuda", sync=True):
    """Full products of CPU (pinned) tensors, copies overlapped with kernels."""
    a, b = _host_tensor(a, "a"), _host_tensor(b, "b")
    count, na = a.shape
    nb = b.shape[1]
    out = _host_tensor(_host_out(count, na + nb, out), "out")
    ws = _host_ws(OP_MUL, count, na, nb, workspace, device)
    _host_call(OP_MUL, a, b, out, None, None, na, nb, ws, sync, "bigint_mul_host")
    return out


def divmod_host(u, v, q=None, r=None, status=None, workspace=None, device="cuda", sync=True):
    """q, r (and per-instance status) of CPU (pinned) tensors, copies
    overlapped with the division kernels."""
    torch = _torch()
    u, v = _host_tensor(u, "u"), _host_tensor(v, "v")
    count, nu = u.shape
    nv = v.shape[1]
    q = _host_tensor(_host_out(count, max(nu - nv + 1, 1), q), "q")
    r = _host_tensor(_host_out(count, nv, r), "r")
    if status is None:
        status = torch.empty(count, dtype=torch.int32).pin_memory()
    ws = _host_ws(OP_DIVMOD, count, nu, nv, workspace, device)
    _host_call(OP_DIVMOD, u, v, q, r, status, nu, nv, ws, sync, "bigint_divmod_host")
    return q, r, status


def host_sync() -> None:
    """Waits for every host-buffer call enqueued with sync=False."""
    _check(load().bigint_host_sync(), "bigint_host_sync")


def set_variant(op: int, variant: int) -> None:
    """Select the kernel variant of an operation (op 0 = multiply, op 1 =
    division; see bigint_set_variant in include/bigint.h)."""
    _check(load().bigint_set_variant(op, variant), "bigint_set_variant")


def mul_variant_for(na: int, nb: int) -> int:
    """The multiply variant a full na x nb product runs with (1..12)."""
    return int(load().bigint_mul_variant_for(na, nb))


def check_timeout() -> None:
    """Raises BigIntError if a tensor-core product stopped at a device wait
    limit since the previous check (synchronises the device)."""
    _check(load().bigint_check_timeout(), "bigint_check_timeout")


def kernel_launches() -> int:
    """Kernels the library has launched in this process so far."""
    return int(load().bigint_kernel_launches())


def set_wait_limit(cycles: int) -> None:
    """Cycle limit of the tensor-core products' device waits (0: the
    default, about one second); a negative value makes every wait give up
    after -cycles cycles on a flag nothing sets (once the work it guards has
    finished), which tests the timeout path."""
    _check(load().bigint_set_wait_limit(int(cycles)), "bigint_set_wait_limit")


def probe_int_throughput(variant: int):
    """(thread operations per SM per cycle, SM MHz) of one integer form."""
    ops, mhz = ctypes.c_double(), ctypes.c_double()
    rc = load().bigint_probe_int_throughput(variant, ctypes.byref(ops), ctypes.byref(mhz))
    _check(rc, "bigint_probe_int_throughput")
    return ops.value, mhz.value


# ---- ragged batches -------------------------------------------------------
def op_dtype():
    """numpy dtype of one bigint_op descriptor (include/bigint.h)."""
    import numpy as np

    return np.dtype([("op", "<i4"), ("na", "<i4"), ("nb", "<i4"), ("flags", "<i4"),
                     ("a", "<i8"), ("b", "<i8"), ("o1", "<i8"), ("o2", "<i8")])


class Batch:
    """A ragged batch of mixed operations over an input and an output pool.

    ``ops`` is a numpy array of ``op_dtype()``; offsets are in limbs.  The
    plan (sort, size classes, launch shapes) is built on the host by the C
    library; ``launch`` only enqueues device work, so it can be captured in
    a CUDA graph."""

    def __init__(self, ops, device="cuda", stream=None, allocate=True):
        import numpy as np

        self.ops = np.ascontiguousarray(ops, dtype=op_dtype())
        h = ctypes.c_void_p()
        _check(load().bigint_batch_create(self.ops.ctypes.data, len(self.ops), ctypes.byref(h)),
               "bigint_batch_create")
        self._h = h
        self.workspace_bytes = int(load().bigint_batch_workspace(h))
        self.workspace = None
        if allocate:
            self.allocate(device, stream)

    def allocate(self, device="cuda", stream=None):
        """Allocates the device workspace (``workspace_bytes``, known from the
        host-side plan alone) and uploads the plan into it."""
        import torch

        self.workspace = torch.empty(max(self.workspace_bytes, 256), dtype=torch.uint8,
                                     device=device)
        _check(load().bigint_batch_upload(self._h, self.workspace.data_ptr(),
                                          self.workspace.numel(), _stream_ptr(stream)),
               "bigint_batch_upload")

    def launch(self, in_pool, out_pool, status=None, mode=BATCH_PERSISTENT, stream=None):
        rc = load().bigint_batch_launch(self._h, in_pool.data_ptr(), out_pool.data_ptr(),
                                        status.data_ptr() if status is not None else None,
                                        self.workspace.data_ptr(), mode, _stream_ptr(stream))
        _check(rc, "bigint_batch_launch")

    def tune(self, in_pool, out_pool, status=None, stream=None) -> int:
        best = ctypes.c_int()
        rc = load().bigint_batch_tune(self._h, in_pool.data_ptr(), out_pool.data_ptr(),
                                      status.data_ptr() if status is not None else None,
                                      self.workspace.data_ptr(), self.workspace.numel(),
                                      _stream_ptr(stream), ctypes.byref(best))
        _check(rc, "bigint_batch_tune")
        return best.value

    def close(self):
        if getattr(self, "_h", None):
            load().bigint_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tune(a, b, out=None, stream=None) -> int:
    """Times the multiply variants (tensor-core tiles, integer forms) on this
    batch; records the fastest for its size class and returns it."""
    a, b = _dev_tensor(a, "a"), _dev_tensor(b, "b")
    count, na = a.shape
    nb = b.shape[1]
    out = _empty_like_limbs(a, count, na + nb) if out is None else out
    best = ctypes.c_int()
    _check(load().bigint_tune(a.data_ptr(), b.data_ptr(), out.data_ptr(), count, na, nb,
                              _stream_ptr(stream), ctypes.byref(best)), "bigint_tune")
    return best.value


def save_tuning(path: str) -> None:
    _check(load().bigint_save_tuning(path.encode()), "bigint_save_tuning")


def load_tuning(path: str) -> None:
    _check(load().bigint_load_tuning(path.encode()), "bigint_load_tuning")


# ---- ragged views -----------------------------------------------------------
class _View(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("offset", ctypes.c_void_p),
                ("nlimbs", ctypes.c_void_p), ("count", ctypes.c_int64), ("n", ctypes.c_int32)]


ZEXT = 1


def view(data, offsets=None, nlimbs=None, count=None, n=0):
    """A ragged view (bigint_batch_cview / bigint_batch_view) over a 1-D or
    2-D CUDA limb tensor: instance i has nlimbs[i] limbs starting offsets[i]
    limbs into `data` (numpy int64 / int32 host arrays), or the uniform
    layout of a (count, n) tensor.  Returns the ctypes structure; it keeps
    the host arrays alive."""
    import numpy as np

    if not data.is_cuda:
        raise TypeError("view data must be a CUDA tensor")
    v = _View()
    v.data = data.data_ptr()
    if offsets is None:
        count, n = data.shape if data.dim() == 2 else (count, n)
        v.offset = v.nlimbs = None
    else:
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        nlimbs = np.ascontiguousarray(nlimbs, dtype=np.int32)
        count = offsets.size
        v.offset, v.nlimbs = offsets.ctypes.data, nlimbs.ctypes.data
        v._keep = (offsets, nlimbs)
    v.count, v.n = int(count), int(n)
    return v


def views_workspace_bytes(op: int, a, b) -> int:
    return int(load().bigint_batch_views_workspace(op, ctypes.byref(a), ctypes.byref(b)))


def _views_ws(op, a, b, workspace, device):
    torch = _torch()
    if workspace is None:
        workspace = torch.empty(max(views_workspace_bytes(op, a, b), 256), dtype=torch.uint8,
                                device=device)
    return workspace


def batch_add(a, b, out, carry=None, zext=False, workspace=None, stream=None, sub=False):
    """out = a + b (or a - b with sub=True) over ragged views; carry: a CUDA
    int32 tensor of count entries or None."""
    op = OP_SUB if sub else OP_ADD
    ws = _views_ws(op, a, b, workspace, "cuda")
    fn = load().bigint_batch_sub if sub else load().bigint_batch_add
    rc = fn(ctypes.byref(a), ctypes.byref(b), ctypes.byref(out),
            carry.data_ptr() if carry is not None else None, ZEXT if zext else 0,
            ws.data_ptr(), ws.numel(), _stream_ptr(stream))
    _check(rc, "bigint_batch_sub" if sub else "bigint_batch_add")


def batch_mul(a, b, out, workspace=None, stream=None):
    ws = _views_ws(OP_MUL, a, b, workspace, "cuda")
    _check(load().bigint_batch_mul(ctypes.byref(a), ctypes.byref(b), ctypes.byref(out),
                                   ws.data_ptr(), ws.numel(), _stream_ptr(stream)),
           "bigint_batch_mul")


def batch_divmod(u, v, q, r, status=None, workspace=None, stream=None):
    ws = _views_ws(OP_DIVMOD, u, v, workspace, "cuda")
    _check(load().bigint_batch_divmod(ctypes.byref(u), ctypes.byref(v), ctypes.byref(q),
                                      ctypes.byref(r),
                                      status.data_ptr() if status is not None else None,
                                      ws.data_ptr(), ws.numel(), _stream_ptr(stream)),
           "bigint_batch_divmod")


def batch_run(ops, in_pool, out_pool, status=None, mode=BATCH_PERSISTENT, workspace=None,
              stream=None):
    """Plans, uploads and launches a mixed batch of descriptors in one call."""
    import numpy as np

    torch = _torch()
    ops = np.ascontiguousarray(ops, dtype=op_dtype())
    L = load()
    need = int(L.bigint_batch_run_workspace(ops.ctypes.data, len(ops)))
    if workspace is None:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=in_pool.device)
    _check(L.bigint_batch_run(ops.ctypes.data, len(ops), in_pool.data_ptr(), out_pool.data_ptr(),
                              status.data_ptr() if status is not None else None,
                              workspace.data_ptr(), workspace.numel(), mode, _stream_ptr(stream)),
           "bigint_batch_run")
