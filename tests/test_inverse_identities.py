"""CPU checks, in exact integers, of the identities division by a reused
inverse (bigint_divmod_inv) rests on: the top limbs of floor(B^h / v) are
the inverse at a lower h, and with u < B^h the quotient estimate
floor(u w / B^h) is q or q - 1, so one correction round settles it."""
import numpy as np
import pytest

B = 1 << 64


@pytest.mark.parametrize("seed", range(6))
def test_top_limbs_are_the_lower_inverse(seed):
    rng = np.random.default_rng(seed)
    for _ in range(50):
        nv = int(rng.integers(1, 6))
        v = int.from_bytes(rng.bytes(8 * nv), "little") | 1
        h = nv + int(rng.integers(0, 8))
        s = int(rng.integers(0, h - nv + 1))
        w = B ** h // v
        assert w // B ** s == B ** (h - s) // v


@pytest.mark.parametrize("seed", range(6))
def test_estimate_within_one(seed):
    rng = np.random.default_rng(100 + seed)
    for _ in range(200):
        nv = int(rng.integers(1, 5))
        v = int.from_bytes(rng.bytes(8 * nv), "little") | (1 << (64 * nv - 64))
        h = nv + int(rng.integers(0, 6))
        ku = int(rng.integers(nv, h + 1))
        u = int.from_bytes(rng.bytes(8 * ku), "little")
        # the kernel takes the inverse at prec(u) = ku from the top limbs
        w = (B ** h // v) // B ** (h - ku)
        qhat = u * w // B ** ku
        q = u // v
        assert q - 1 <= qhat <= q
        r = u - qhat * v
        assert 0 <= r < 2 * v
