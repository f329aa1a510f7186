"""Python marshalling for the plain CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY.  The test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` are the only callers.  The product path
(the CUDA library and ``paper_2607_28897_gb300``) never imports this module.

Every function takes and returns numpy ``uint64`` arrays of little-endian
64-bit limbs; batched functions take ``(count, n)`` arrays.  All arithmetic
happens in ``oracle.c``; this file only moves arrays across ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

OK, EINVAL, EDIVZERO = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` into ``liboracle.so`` (OpenMP when available)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", _LIB_PATH]
    try:
        subprocess.run(base[:5] + ["-fopenmp"] + base[5:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB points the pins at a deliberately broken build of this
        # oracle (tests/test_oracle_mutants.py); normal runs never set it.
        path = os.environ.get("ORACLE_LIB")
        if not path:
            build()
            path = _LIB_PATH
        L = ctypes.CDLL(path)
        p, i64, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        L.orc_add.argtypes = [p, p, p, i64]
        L.orc_sub.argtypes = [p, p, p, i64]
        L.orc_mul.argtypes = [p, i64, p, i64, p]
        L.orc_mul.restype = None
        L.orc_mul_lo.argtypes = [p, i64, p, i64, i64, p]
        L.orc_mul_lo.restype = None
        L.orc_divmod.argtypes = [p, i64, p, i64, p, p]
        L.orc_shinv.argtypes = [p, i64, i64, p, i64]
        L.orc_step.argtypes = [i64, i64, p, i64, p, i64, p, i64]
        L.orc_prec.argtypes = [p, i64]
        L.orc_prec.restype = i64
        L.orc_batch_add.argtypes = [p, p, p, p, i64, i64]
        L.orc_batch_sub.argtypes = [p, p, p, p, i64, i64]
        L.orc_batch_mul.argtypes = [p, p, p, i64, i64, i64]
        L.orc_batch_divmod.argtypes = [p, p, p, p, p, i64, i64, i64]
        L.orc_num_threads.argtypes = []
        L.orc_add_chain.argtypes = [p, p, p, i64, i32]
        L.orc_add_chain.restype = i32
        L.orc_poly.argtypes = [p, p, p, i64]
        L.orc_poly.restype = None
        for f in ("orc_add", "orc_sub", "orc_divmod", "orc_shinv", "orc_step",
                  "orc_batch_add", "orc_batch_sub", "orc_batch_mul",
                  "orc_batch_divmod", "orc_num_threads"):
            getattr(L, f).restype = i32
        _lib = L
    return _lib


def _u64(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.uint64)


def _ptr(x: np.ndarray):
    return x.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return lib().orc_num_threads()


# ---- single instances ------------------------------------------------------
def add(a, b):
    a, b = _u64(a), _u64(b)
    out = np.zeros_like(a)
    c = lib().orc_add(_ptr(a), _ptr(b), _ptr(out), a.size)
    return out, c


def sub(a, b):
    a, b = _u64(a), _u64(b)
    out = np.zeros_like(a)
    c = lib().orc_sub(_ptr(a), _ptr(b), _ptr(out), a.size)
    return out, c


def mul(a, b):
    a, b = _u64(a), _u64(b)
    out = np.zeros(a.size + b.size, dtype=np.uint64)
    lib().orc_mul(_ptr(a), a.size, _ptr(b), b.size, _ptr(out))
    return out


def mul_lo(a, b, m: int):
    a, b = _u64(a), _u64(b)
    out = np.zeros(m, dtype=np.uint64)
    lib().orc_mul_lo(_ptr(a), a.size, _ptr(b), b.size, m, _ptr(out))
    return out


def divmod_(u, v):
    u, v = _u64(u), _u64(v)
    nq = max(u.size - v.size + 1, 1)
    q = np.zeros(nq, dtype=np.uint64)
    r = np.zeros(v.size, dtype=np.uint64)
    s = lib().orc_divmod(_ptr(u), u.size, _ptr(v), v.size, _ptr(q), _ptr(r))
    return q, r, s


def shinv(v, h: int, nw: int):
    v = _u64(v)
    w = np.zeros(nw, dtype=np.uint64)
    s = lib().orc_shinv(_ptr(v), v.size, h, _ptr(w), nw)
    return w, s


def step(h: int, m: int, v, w, nout: int):
    v, w = _u64(v), _u64(w)
    out = np.zeros(nout, dtype=np.uint64)
    s = lib().orc_step(h, m, _ptr(v), v.size, _ptr(w), w.size, _ptr(out), nout)
    return out, s


def add_chain(a, b, k: int):
    a, b = _u64(a), _u64(b)
    out = np.zeros_like(a)
    c = lib().orc_add_chain(_ptr(a), _ptr(b), _ptr(out), a.size, k)
    return out, c


def poly(a, b):
    a, b = _u64(a), _u64(b)
    out = np.zeros_like(a)
    lib().orc_poly(_ptr(a), _ptr(b), _ptr(out), a.size)
    return out


def prec(x) -> int:
    x = _u64(x)
    return int(lib().orc_prec(_ptr(x), x.size))


# ---- uniform batches (count, n) --------------------------------------------
def batch_add(a, b):
    a, b = _u64(a), _u64(b)
    count, n = a.shape
    out = np.zeros_like(a)
    carry = np.zeros(count, dtype=np.uint8)
    lib().orc_batch_add(_ptr(a), _ptr(b), _ptr(out), _ptr(carry), count, n)
    return out, carry


def batch_sub(a, b):
    a, b = _u64(a), _u64(b)
    count, n = a.shape
    out = np.zeros_like(a)
    borrow = np.zeros(count, dtype=np.uint8)
    lib().orc_batch_sub(_ptr(a), _ptr(b), _ptr(out), _ptr(borrow), count, n)
    return out, borrow


def batch_mul(a, b):
    a, b = _u64(a), _u64(b)
    count, na = a.shape
    nb = b.shape[1]
    out = np.zeros((count, na + nb), dtype=np.uint64)
    lib().orc_batch_mul(_ptr(a), _ptr(b), _ptr(out), count, na, nb)
    return out


def batch_divmod(u, v):
    u, v = _u64(u), _u64(v)
    count, nu = u.shape
    nv = v.shape[1]
    nq = max(nu - nv + 1, 1)
    q = np.zeros((count, nq), dtype=np.uint64)
    r = np.zeros((count, nv), dtype=np.uint64)
    st = np.zeros(count, dtype=np.int32)
    lib().orc_batch_divmod(_ptr(u), _ptr(v), _ptr(q), _ptr(r), _ptr(st), count,
                           nu, nv)
    return q, r, st
