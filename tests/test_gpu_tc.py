"""GPU parity of the tensor-core product (multiply variant 12) against the
oracle: ragged and multi-tile shapes, low-part products, the digit patterns
that drive the fp32 accumulators to their bound, and the wait-limit record."""
import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu

TC = 12


@pytest.fixture(scope="module")
def bi():
    import paper_2607_28897_gb300 as m

    m.load()
    m.set_variant(0, TC)
    yield m
    m.set_variant(0, 0)


def check(bi, orc, a, b):
    assert bi.mul_variant_for(a.shape[1], b.shape[1]) == TC
    p = bi.mul(to_dev(a), to_dev(b))
    assert np.array_equal(to_host(p), orc.batch_mul(a, b))
    bi.check_timeout()


@pytest.mark.parametrize("na,nb", [(1, 1), (1, 2), (2, 3), (15, 16), (16, 16), (17, 17),
                                   (33, 40), (64, 64), (100, 37), (255, 257), (512, 512),
                                   (1000, 999), (1024, 1024), (1024, 1031), (1017, 1024),
                                   (2048, 2048), (3001, 17)])
def test_shapes(bi, orc, na, nb):
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(700 + na, 6, na)
    b = inputs.limbs(800 + nb, 6, nb)
    check(bi, orc, a, b)


@pytest.mark.parametrize("na,nb", [(1, 4200), (4150, 3), (4096, 4096), (8192, 8192),
                                   (10000, 10000)])
def test_multi_tile(bi, orc, na, nb):
    """More than 256 output columns of 128 digits: several tiles per product,
    carries handed from tile to tile."""
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(900 + na, 2, na)
    b = inputs.limbs(950 + nb, 2, nb)
    check(bi, orc, a, b)


@pytest.mark.parametrize("pattern", [0xFFFFFFFFFFFFFFFF, 0x7F807F807F807F80,
                                     0x807F807F807F807F, 0x8080808080808080,
                                     0x7F7F7F7F7F7F7F7F, 0x0000000000000080])
@pytest.mark.parametrize("n", [1024, 8192])
def test_extreme_digits(bi, orc, pattern, n):
    """Byte patterns whose signed digits are all +-128 (alternating 0x7F/0x80)
    put every accumulator group at its bound 2^24; all-ones and lone top
    bits exercise the carry digit above the top byte (1024 limbs: the shape
    whose x operand goes without it, corrected by t_x y B^nx)."""
    a = np.full((2, n), np.uint64(pattern), dtype=np.uint64)
    b = a.copy()
    b[1] = np.uint64(0xFFFFFFFFFFFFFFFF ^ pattern)
    check(bi, orc, a, b)


def test_batch_more_instances_than_sms(bi, orc):
    """A persistent CTA per SM loops over instances: 600 instances."""
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(31, 600, 96)
    b = inputs.limbs(32, 600, 96)
    check(bi, orc, a, b)


@pytest.mark.parametrize("na,nb,m", [(512, 512, 513), (512, 512, 1), (300, 4000, 2100),
                                     (4096, 4096, 4096)])
def test_low_part(bi, orc, na, nb, m):
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(1000 + m, 3, na)
    b = inputs.limbs(1100 + m, 3, nb)
    got = to_host(bi.mul_lo(to_dev(a), to_dev(b), m))
    want = np.stack([orc.mul_lo(a[i], b[i], m) for i in range(a.shape[0])])
    assert np.array_equal(got, want)
    bi.check_timeout()


def test_same_as_integer_variant(bi):
    """Variant 12 and the IMAD schoolbook give identical bytes at 2^19 bits."""
    from paper_2607_28897_gb300 import inputs

    a = to_dev(inputs.limbs(41, 8, 8192))
    b = to_dev(inputs.limbs(42, 8, 8192))
    p12 = to_host(bi.mul(a, b))
    bi.set_variant(0, 8)
    try:
        p8 = to_host(bi.mul(a, b))
    finally:
        bi.set_variant(0, TC)
    assert np.array_equal(p12, p8)


@pytest.mark.parametrize("na,nb,count", [(2048, 2049, 3), (4096, 4096, 2), (3000, 5000, 2),
                                         (1, 8000, 2), (8192, 8192, 2), (10000, 10000, 1),
                                         (9000, 10000, 1), (512, 512, 4), (300, 7000, 1),
                                         (8192, 8192, 16), (2100, 2100, 170),
                                         (4096, 4096, 17)])
def test_split(bi, orc, na, nb, count):
    """Products spread over CTAs -- up to 16 products cut into (tile, groups)
    units that add their column sums atomically (split-K), larger batches
    with each 4096-limb output tile on its own CTA, linked by a finishing
    kernel -- bit-identical to the oracle and to the one-CTA form (ragged
    last tiles, a one-limb operand, more units than SMs)."""
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(1200 + na, count, na)
    b = inputs.limbs(1300 + nb, count, nb)
    tiles = -(-(na + nb) // 4096)
    ws = bi.mul_split_workspace_bytes(count, na, nb)
    if count > 16 or min(na, nb) < 256:
        assert ws == 16 * count * tiles  # tile split
    else:
        assert ws >= count * tiles * 256 * 128 * 4  # column sums of every tile
    da, db = to_dev(a), to_dev(b)
    got = to_host(bi.mul_split(da, db))
    assert np.array_equal(got, orc.batch_mul(a, b))
    assert np.array_equal(got, to_host(bi.mul(da, db)))
    bi.check_timeout()


@pytest.mark.parametrize("pattern", [0xFFFFFFFFFFFFFFFF, 0x7F807F807F807F80,
                                     0x8080808080808080, 0x0000000000000080])
def test_split_extreme_digits(bi, orc, pattern):
    """Digit patterns at the accumulator bound and all-ones operands, whose
    products carry across the tile boundaries through long runs of ones."""
    n = 8192
    a = np.full((2, n), np.uint64(pattern), dtype=np.uint64)
    b = a.copy()
    b[1] = np.uint64(0xFFFFFFFFFFFFFFFF ^ pattern)
    got = to_host(bi.mul_split(to_dev(a), to_dev(b)))
    assert np.array_equal(got, orc.batch_mul(a, b))
    bi.check_timeout()


def test_split_small_shapes_run_unsplit(bi, orc):
    """Larger batches of products with a single tile need no workspace and
    run as the ordinary product."""
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(51, 40, 512)
    b = inputs.limbs(52, 40, 512)
    assert bi.mul_split_workspace_bytes(40, 512, 512) == 0
    got = to_host(bi.mul_split(to_dev(a), to_dev(b)))
    assert np.array_equal(got, orc.batch_mul(a, b))


def test_split_workspace_too_small(bi):
    import torch

    from paper_2607_28897_gb300 import inputs

    a = to_dev(inputs.limbs(53, 2, 4096))
    ws = torch.empty(16 * 2 * 2 - 8, dtype=torch.uint8, device="cuda")
    with pytest.raises(bi.BigIntError):
        bi.mul_split(a, a, workspace=ws)
