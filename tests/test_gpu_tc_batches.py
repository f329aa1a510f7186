"""GPU parity of the tensor-core product in batches with several products
per persistent CTA (the launch shape of the 2^17-bit sweep products and of
the Karatsuba leaves: 256-column tiles, one CTA per SM): uneven products per
CTA, unequal operands, the digit patterns at the accumulator bound in the
first and last products a CTA computes, and Karatsuba products over such
batches, against the oracle."""
import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bi():
    import paper_2607_28897_gb300 as m

    m.load()
    m.set_variant(0, 0)
    yield m
    m.set_variant(0, 0)


@pytest.mark.parametrize("na,nb,count", [(2048, 2048, 304), (2048, 2048, 459),
                                         (2048, 1500, 320), (1500, 2048, 330),
                                         (2047, 2049, 305)])
def test_batches(bi, orc, na, nb, count):
    """Two to four products per CTA on 152 SMs (459: some CTAs take one
    more than others); every product equals the oracle's."""
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(1500 + na, count, na)
    b = inputs.limbs(1600 + nb, count, nb)
    got = to_host(bi.mul(to_dev(a), to_dev(b)))
    bi.check_timeout()
    assert np.array_equal(got, orc.batch_mul(a, b))


@pytest.mark.parametrize("pattern", [0xFFFFFFFFFFFFFFFF, 0x7F807F807F807F80,
                                     0x807F807F807F807F, 0x8080808080808080,
                                     0x7F7F7F7F7F7F7F7F, 0x0000000000000080])
def test_batch_extreme_digits(bi, orc, pattern):
    """Digit patterns that put every accumulator group at its bound 2^24,
    all-ones operands (carries through the whole product) and lone top
    bits, in the first and last products of a 310-product batch."""
    from paper_2607_28897_gb300 import inputs

    n, count = 2048, 310
    a = inputs.limbs(1700, count, n)
    b = inputs.limbs(1701, count, n)
    for r in (0, 1, 152, count - 1):
        a[r] = np.uint64(pattern)
        b[r] = np.uint64(pattern if r % 2 == 0 else 0xFFFFFFFFFFFFFFFF ^ pattern)
    got = to_host(bi.mul(to_dev(a), to_dev(b)))
    bi.check_timeout()
    rows = [0, 1, 2, 151, 152, 153, count - 1]
    assert np.array_equal(got[rows], orc.batch_mul(a[rows], b[rows]))


@pytest.mark.parametrize("n,count", [(4096, 320), (8192, 304)])
def test_kara_batches(bi, orc, n, count):
    """Karatsuba products whose 2048-limb leaves run in such batches (one
    level at 4096 limbs, two at 8192): sampled products against the oracle,
    all of them against the schoolbook product."""
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(1800 + n, count, n)
    b = inputs.limbs(1900 + n, count, n)
    da, db = to_dev(a), to_dev(b)
    k = to_host(bi.mul_kara(da, db))
    school = to_host(bi.mul(da, db))
    bi.check_timeout()
    assert np.array_equal(k, school)
    rows = [0, 151, count - 1]
    assert np.array_equal(k[rows], orc.batch_mul(a[rows], b[rows]))


@pytest.mark.parametrize("n,count", [(2048, 160), (4096, 160), (8192, 160), (1500, 200)])
def test_more_products_than_sms_against_fewer(bi, orc, n, count):
    """A batch with more products than SMs (persistent CTAs that compute
    several products in turn, reusing their shared memory and tensor memory)
    equals, product by product, the same products in a batch of at most one
    per SM, and sampled products equal the oracle's; multi-tile products
    (4096 and 8192 limbs) included."""
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(2000 + n, count, n)
    b = inputs.limbs(2100 + n, count, n)
    da, db = to_dev(a), to_dev(b)
    many = to_host(bi.mul(da, db))
    few = to_host(bi.mul(da[:150].contiguous(), db[:150].contiguous()))
    bi.check_timeout()
    assert np.array_equal(many[:150], few)
    rows = [0, 149, 151, count - 1]
    assert np.array_equal(many[rows], orc.batch_mul(a[rows], b[rows]))
