"""GPU parity of the full-product multiply (Sec. V-B) against the oracle."""
import numpy as np
import pytest

from helpers import SMALL_PRIMES, mulmod, residues, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bi():
    import paper_2607_28897_gb300 as m

    m.load()
    return m


def check_mul(bi, orc, a, b):
    p = bi.mul(to_dev(a), to_dev(b))
    assert np.array_equal(to_host(p), orc.batch_mul(a, b))


def test_config_small_mul(bi, orc):
    from paper_2607_28897_gb300 import inputs

    a, b = inputs.config_small(seed=1, n=512, count=64)
    check_mul(bi, orc, a, b)


@pytest.mark.parametrize("n", [1, 2, 3, 7, 8, 9, 31, 64, 100, 255, 256, 257, 700, 1023,
                               1025, 2048, 3001])
def test_square_lengths(bi, orc, n):
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(300 + n, 5, n)
    b = inputs.limbs(400 + n, 5, n)
    ones = np.full((1, n), np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    check_mul(bi, orc, np.concatenate([a, ones]), np.concatenate([b, ones]))


@pytest.mark.parametrize("na,nb", [(1, 5), (5, 1), (17, 300), (300, 17), (512, 1024),
                                   (2049, 2048), (10000, 10000), (10000, 3)])
def test_rectangular(bi, orc, na, nb):
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(500 + na, 4, na)
    b = inputs.limbs(600 + nb, 4, nb)
    check_mul(bi, orc, a, b)


def test_all_ones_closed_form(bi):
    """(B^n - 1)^2 = B^2n - 2 B^n + 1 at n = 8192 (2^19 bits)."""
    n = 8192
    ones = np.full((2, n), np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    p = to_host(bi.mul(to_dev(ones), to_dev(ones)))
    for row in p:
        assert row[0] == 1 and not row[1:n].any()
        assert row[n] == np.uint64(0xFFFFFFFFFFFFFFFE)
        assert np.all(row[n + 1:] == np.uint64(0xFFFFFFFFFFFFFFFF))


@pytest.mark.parametrize("m", [1, 7, 512, 1000, 1024])
def test_mul_lo(bi, orc, m):
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(7, 6, 512)
    b = inputs.limbs(8, 6, 512)
    lo = to_host(bi.mul_lo(to_dev(a), to_dev(b), m))
    for i in range(a.shape[0]):
        assert np.array_equal(lo[i], orc.mul_lo(a[i], b[i], m))


@pytest.mark.parametrize("n", [512, 1024, 2048, 4096, 8192])
def test_config_sweep_full_size(bi, orc, n):
    """Full 2^32-bit operand arrays in the launch configuration the bench
    times: residues mod three primes for every instance, and a full compare
    against the oracle on a seeded sample of instances."""
    from paper_2607_28897_gb300 import inputs

    a, b = inputs.config_sweep(n)
    p = to_host(bi.mul(to_dev(a), to_dev(b)))
    for pr in SMALL_PRIMES:
        assert np.array_equal(residues(p, pr), mulmod(residues(a, pr), residues(b, pr), pr))
    rng = np.random.default_rng(n)
    k = 8 if n >= 4096 else 16
    idx = np.unique(np.concatenate([[0, a.shape[0] - 1], rng.choice(a.shape[0], k)]))
    assert np.array_equal(p[idx], orc.batch_mul(a[idx], b[idx]))


@pytest.mark.parametrize("variant", [8, 9, 10, 11, 12, 13, 14, 15, 16, 17])
@pytest.mark.parametrize("n", [1, 63, 64, 65, 511, 1000, 2049])
def test_every_variant(bi, orc, variant, n):
    """Every multiply variant (integer digit size and chunk width, Karatsuba,
    the tensor-core product with each tile) gives the oracle's product;
    Karatsuba falls back to the schoolbook kernel below 64 limbs."""
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(700 + n, 3, n)
    b = inputs.limbs(800 + n, 3, n)
    ones = np.full((1, n), np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    a, b = np.concatenate([a, ones]), np.concatenate([b, ones])
    bi.set_variant(0, variant)
    try:
        p = to_host(bi.mul(to_dev(a), to_dev(b)))
    finally:
        bi.set_variant(0, 0)
    assert np.array_equal(p, orc.batch_mul(a, b))


@pytest.mark.parametrize("na,nb,m", [(1, 1, 2), (1, 64, 65), (64, 1, 3), (2, 3, 5), (17, 33, 50),
                                     (33, 17, 20), (64, 64, 128), (64, 64, 1), (31, 32, 40),
                                     (64, 63, 66), (5, 64, 69)])
def test_warp_per_instance_products(bi, orc, na, nb, m):
    """Variant 11 (one warp per instance, operands of at most 64 limbs): full
    and low products of ragged shapes, more instances than warps of one
    CTA, all-ones operands (every column sum at its largest)."""
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(60 + na, 21, na)
    b = inputs.limbs(61 + nb, 21, nb)
    a[::5] = np.uint64(0xFFFFFFFFFFFFFFFF)
    b[::5] = np.uint64(0xFFFFFFFFFFFFFFFF)
    bi.set_variant(0, 11)
    try:
        got = to_host(bi.mul_lo(to_dev(a), to_dev(b), m))
    finally:
        bi.set_variant(0, 0)
    want = np.stack([orc.mul_lo(a[i], b[i], m) for i in range(a.shape[0])])
    assert np.array_equal(got, want)
