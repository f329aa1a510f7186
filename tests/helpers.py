"""Shared helpers of the GPU parity tests (no arithmetic of the method)."""
from __future__ import annotations

import numpy as np

# Primes below 2^31, so a Horner step r * 2^32 + digit stays below 2^63 in
# uint64 numpy arithmetic.
SMALL_PRIMES = (2147483647, 2147483629, 2147483587)


def to_dev(x, device="cuda:0"):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).to(device)


def to_host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def residues(x: np.ndarray, p: int) -> np.ndarray:
    """Row-wise value mod p of a (count, n) little-endian limb array, by
    Horner's rule over 32-bit half-limbs from the top down."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    P = np.uint64(p)
    sh = np.uint64(32)
    mask = np.uint64(0xFFFFFFFF)
    r = np.zeros(x.shape[0], dtype=np.uint64)
    for j in range(x.shape[1] - 1, -1, -1):
        limb = x[:, j]
        r = ((r << sh) + (limb >> sh)) % P
        r = ((r << sh) + (limb & mask)) % P
    return r


def mulmod(x: np.ndarray, y: np.ndarray, p: int) -> np.ndarray:
    """(x * y) mod p for arrays of residues below p < 2^31."""
    return (x.astype(np.uint64) * y.astype(np.uint64)) % np.uint64(p)
