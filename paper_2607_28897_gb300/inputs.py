"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module only draws numbers: it holds none of the arithmetic of the
method (no carry, product or quotient is computed here).  The generator is
SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) used as a counter-based hash: element i of stream
``seed`` is ``mix(seed * 2^32 + stream_pos + (i + 1) * GAMMA)``, so any slice
can be drawn independently and the result does not depend on chunking.

Workload recipes (the paper's datasets are "random", Sec. VI; the shapes
follow its Bits x Insts = 2^32 rule):

* ``uniform``: limbs uniform over [0, 2^64).
* ``config_small``: 64 random pairs of 512 limbs plus 8 carry-stress pairs.
* ``config_sweep``: n in {512..8192} limbs, batch 2^26 / n, top limb nonzero.
* ``config_div``: dividend 2n limbs (top limb nonzero), divisor n limbs whose
  top limb has bit 63 set for even instances and lies in [1, 2^32) for odd.
* ``ragged_sizes``: bit lengths 2^U, U ~ Uniform[15, 19], rounded to limbs.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
ALL_ONES = np.uint64(0xFFFFFFFFFFFFFFFF)


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform(seed: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` uniform uint64 values: elements [start, start+count) of the
    stream ``seed``."""
    out = np.empty(count, dtype=np.uint64)
    chunk = 1 << 22
    base = np.uint64((seed * (1 << 32)) & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for s in range(0, count, chunk):
            e = min(count, s + chunk)
            idx = np.arange(start + s + 1, start + e + 1, dtype=np.uint64)
            out[s:e] = _mix(base + idx * GAMMA)
    return out


def limbs(seed: int, count: int, n: int, top_nonzero: bool = False) -> np.ndarray:
    """A (count, n) array of uniform limbs; optionally the top limb of each
    instance is redrawn (from a second stream) until nonzero."""
    x = uniform(seed, count * n).reshape(count, n)
    if top_nonzero and n > 0:
        k = 0
        while True:
            z = np.nonzero(x[:, -1] == 0)[0]
            if z.size == 0:
                break
            x[z, -1] = uniform(seed + 7919 + k, z.size)
            k += 1
    return x


def _lex_ge(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Row-wise a >= b for little-endian limb rows (a plain comparison from
    the top limb down, used only to order input pairs)."""
    ge = np.ones(a.shape[0], dtype=bool)
    decided = np.zeros(a.shape[0], dtype=bool)
    for j in range(a.shape[1] - 1, -1, -1):
        gt = (a[:, j] > b[:, j]) & ~decided
        lt = (a[:, j] < b[:, j]) & ~decided
        ge[lt] = False
        decided |= gt | lt
    return ge


def order_pairs(a: np.ndarray, b: np.ndarray):
    """Swap rows so that a >= b in every row (subtraction inputs)."""
    ge = _lex_ge(a, b)
    a2, b2 = a.copy(), b.copy()
    a2[~ge], b2[~ge] = b[~ge], a[~ge]
    return a2, b2


def stress_pairs(n: int):
    """Eight carry/borrow stress pairs of n limbs (n >= 2):
    (B^n-1, B^n-1), (B^n-1, 1), (1, B^n-1), (B^n-1, 0), (B^(n-1), 1),
    (all-ones with a zero limb at n/2, 1), (0x80..0 in every limb twice),
    (B^n-1, B^n-2)."""
    ones = np.full(n, ALL_ONES, dtype=np.uint64)
    one = np.zeros(n, dtype=np.uint64)
    one[0] = 1
    zero = np.zeros(n, dtype=np.uint64)
    top = np.zeros(n, dtype=np.uint64)
    top[n - 1] = 1
    holed = ones.copy()
    holed[n // 2] = 0
    half = np.full(n, np.uint64(1 << 63), dtype=np.uint64)
    ones_m1 = ones.copy()
    ones_m1[0] = np.uint64(0xFFFFFFFFFFFFFFFE)
    A = [ones, ones, one, ones, top, holed, half, ones]
    Bv = [ones, one, ones, zero, one, one, half, ones_m1]
    return np.stack(A), np.stack(Bv)


def config_small(seed: int = 1, n: int = 512, count: int = 64):
    """64 random pairs of 512 limbs followed by the 8 stress pairs."""
    a = limbs(seed, count, n)
    b = limbs(seed + 1000, count, n)
    sa, sb = stress_pairs(n)
    return np.concatenate([a, sa]), np.concatenate([b, sb])


SWEEP_LIMBS = (512, 1024, 2048, 4096, 8192)


def config_sweep(n: int, seed: int = 2, batch: int | None = None):
    """Operand arrays of 2^32 bits each (batch = 2^26 / n), top limb nonzero."""
    if batch is None:
        batch = (1 << 26) // n
    a = limbs(seed * 100 + n, batch, n, top_nonzero=True)
    b = limbs(seed * 100 + n + 50, batch, n, top_nonzero=True)
    return a, b


DIV_CONFIGS = ((512, 4096), (2048, 1024), (8192, 256))


def config_div(n: int, batch: int, seed: int = 3):
    """Dividend 2n limbs with nonzero top limb; divisor n limbs whose top limb
    has bit 63 set (even instances) or lies in [1, 2^32) (odd instances)."""
    u = limbs(seed * 100 + n, batch, 2 * n, top_nonzero=True)
    v = limbs(seed * 100 + n + 50, batch, n)
    t = uniform(seed * 100 + n + 77, batch)
    even = (np.arange(batch) % 2) == 0
    v[even, -1] = t[even] | np.uint64(1 << 63)
    v[~even, -1] = (t[~even] % np.uint64(0xFFFFFFFF)) + np.uint64(1)
    return u, v


def ragged_sizes(seed: int, count: int, lo_bits: int = 15, hi_bits: int = 19,
                 min_limbs: int = 512, max_limbs: int = 8192) -> np.ndarray:
    """Limb counts with bit length 2^U, U ~ Uniform[lo_bits, hi_bits]."""
    u01 = (uniform(seed, count) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    bits = np.power(2.0, lo_bits + (hi_bits - lo_bits) * u01)
    n = np.rint(bits / 64.0).astype(np.int64)
    return np.clip(n, min_limbs, max_limbs)


# ---------------------------------------------------------------------------
# The same generator evaluated with torch on a device (for the large bench
# arrays); bit-identical to the numpy version above.
# ---------------------------------------------------------------------------
def _s64(x: int) -> int:
    x &= 0xFFFFFFFFFFFFFFFF
    return x - (1 << 64) if x >= (1 << 63) else x


def uniform_torch(seed: int, count: int, device="cuda", start: int = 0):
    """Same values as uniform(seed, count, start), as an int64 tensor."""
    import torch

    def lsr(z, k):
        return (z >> k) & ((1 << (64 - k)) - 1)

    gamma = _s64(int(GAMMA))
    m1, m2 = _s64(int(_M1)), _s64(int(_M2))
    base = _s64(seed * (1 << 32))
    out = torch.empty(count, dtype=torch.int64, device=device)
    chunk = 1 << 24
    for s in range(0, count, chunk):
        e = min(count, s + chunk)
        z = torch.arange(start + s + 1, start + e + 1, dtype=torch.int64, device=device)
        z = base + z * gamma
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        out[s:e] = z ^ lsr(z, 31)
    return out


def limbs_torch(seed: int, count: int, n: int, top_nonzero: bool = False, device="cuda"):
    """Same values as limbs(...), as a (count, n) int64 tensor on `device`."""
    x = uniform_torch(seed, count * n, device).view(count, n)
    if top_nonzero and n > 0:
        k = 0
        while True:
            z = (x[:, -1] == 0).nonzero().flatten()
            if z.numel() == 0:
                break
            x[z, -1] = uniform_torch(seed + 7919 + k, z.numel(), device)
            k += 1
    return x


def config_sweep_torch(n: int, seed: int = 2, batch: int | None = None, device="cuda"):
    if batch is None:
        batch = (1 << 26) // n
    a = limbs_torch(seed * 100 + n, batch, n, True, device)
    b = limbs_torch(seed * 100 + n + 50, batch, n, True, device)
    return a, b


# ---------------------------------------------------------------------------
# Ragged mixed-op batches (the batched form): descriptors + pool layout.
# ---------------------------------------------------------------------------
OP_ADD, OP_SUB, OP_MUL, OP_DIVMOD = 1, 2, 3, 4


def ragged_ops(seed: int, count: int, min_limbs: int = 512, max_limbs: int = 8192,
               mix=(0.40, 0.15, 0.15, 0.30)):
    """Operation descriptors of a ragged batch: sizes 2^U bits, U ~
    Uniform[15, 19] rounded to limbs (clamped to [min_limbs, max_limbs]),
    ops drawn with probabilities mix = (mul, add, sub, divmod); a divmod
    draws n_v from the size law and n_u uniform in [n_v, 2 n_v].  Operands
    are laid out back to back in an input pool, results in an output pool.
    Returns (ops, in_limbs, out_limbs) with ops a numpy array of the
    bigint_op layout."""
    import numpy as np

    dt = np.dtype([("op", "<i4"), ("na", "<i4"), ("nb", "<i4"), ("flags", "<i4"),
                   ("a", "<i8"), ("b", "<i8"), ("o1", "<i8"), ("o2", "<i8")])
    n = ragged_sizes(seed, count, min_limbs=min_limbs, max_limbs=max_limbs)
    if min_limbs < 512 or max_limbs < 8192:  # small test batches: spread over the range
        u = (uniform(seed + 3, count) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
        n = np.clip(np.rint(min_limbs * (max_limbs / min_limbs) ** u), min_limbs, max_limbs)
        n = n.astype(np.int64)
    u01 = (uniform(seed + 1, count) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    c = np.cumsum(mix)
    op = np.where(u01 < c[0], OP_MUL, np.where(u01 < c[1], OP_ADD,
                  np.where(u01 < c[2], OP_SUB, OP_DIVMOD))).astype(np.int32)
    u2 = (uniform(seed + 2, count) >> np.uint64(11)).astype(np.float64) / float(1 << 53)
    na = n.copy()
    nb = n.copy()
    div = op == OP_DIVMOD
    na[div] = n[div] + np.floor(u2[div] * (n[div] + 1)).astype(np.int64)  # n_u in [n_v, 2 n_v]
    ops = np.zeros(count, dtype=dt)
    ops["op"], ops["na"], ops["nb"] = op, na, nb
    in_sizes = na + nb
    a_off = np.concatenate([[0], np.cumsum(in_sizes)[:-1]])
    ops["a"], ops["b"] = a_off, a_off + na
    nq = np.maximum(na - nb + 1, 1)
    out_sizes = np.where(op == OP_MUL, na + nb, np.where(div, nq + nb, na))
    o_off = np.concatenate([[0], np.cumsum(out_sizes)[:-1]])
    ops["o1"] = o_off
    ops["o2"] = np.where(div, o_off + nq, 0)
    return ops, int(in_sizes.sum()), int(out_sizes.sum())


def ragged_pool(seed: int, ops, in_limbs: int, device=None):
    """Input pool of uniform limbs with every operand's top limb nonzero
    (numpy when device is None, else a torch int64 tensor on device)."""
    import numpy as np

    tops = np.concatenate([ops["a"] + ops["na"] - 1, ops["b"] + ops["nb"] - 1])
    if device is None:
        pool = uniform(seed, in_limbs)
        pool[tops] |= np.uint64(1)
        return pool
    import torch

    pool = uniform_torch(seed, in_limbs, device)
    t = torch.from_numpy(tops.astype(np.int64)).to(device)
    pool[t] = pool[t] | 1
    return pool
