"""GPU parity of the tensor-core product with narrow x blocks (multiply
variants 16 and 17: 64- and 32-digit blocks, whose output columns' 128-row
windows overlap, so every coefficient is the sum of 2 or 4 accumulator
rows) against the oracle: ragged, multi-tile and low-part shapes, the digit
patterns that drive the accumulators to their bound, band products inside
step-batched divisions, and bit-identity with the 128-digit shapes."""
import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu

NARROW = (16, 17)


@pytest.fixture(scope="module")
def bi():
    import paper_2607_28897_gb300 as m

    m.load()
    yield m
    m.set_variant(0, 0)


def run(bi, variant, fn):
    bi.set_variant(0, variant)
    try:
        return fn()
    finally:
        bi.set_variant(0, 0)


@pytest.mark.parametrize("variant", NARROW)
@pytest.mark.parametrize("na,nb", [(1, 1), (2, 3), (15, 16), (64, 64), (100, 37), (255, 257),
                                   (256, 256), (511, 513), (512, 512), (700, 300), (1000, 999),
                                   (1024, 1024), (1025, 1000), (2048, 2048), (2049, 17),
                                   (3000, 5000), (4096, 4096), (8192, 8192),
                                   # y's top digits in the high rows of the last columns
                                   (1024, 1025), (1024, 1033), (512, 520), (256, 257),
                                   (768, 770), (2048, 2049), (1016, 1025)])
def test_shapes(bi, orc, variant, na, nb):
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(300 + na, 3, na)
    b = inputs.limbs(400 + nb, 3, nb)
    ones = np.full((1, na), np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    a = np.concatenate([a, ones])
    b = np.concatenate([b, np.full((1, nb), np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)])
    p = run(bi, variant, lambda: to_host(bi.mul(to_dev(a), to_dev(b))))
    assert np.array_equal(p, orc.batch_mul(a, b)), (variant, na, nb)
    bi.check_timeout()


@pytest.mark.parametrize("variant", NARROW)
@pytest.mark.parametrize("pattern", [0xFFFFFFFFFFFFFFFF, 0x7F807F807F807F80,
                                     0x807F807F807F807F, 0x8080808080808080,
                                     0x7F7F7F7F7F7F7F7F, 0x0000000000000080])
@pytest.mark.parametrize("n", [512, 1024, 2048])
def test_extreme_digits(bi, orc, variant, pattern, n):
    """Signed digits all +-128 give every product of a column the same sign:
    each accumulator row reaches G KB 2^14 (within 2^24), and a coefficient's
    rows sum to its full value in int32."""
    a = np.full((2, n), np.uint64(pattern), dtype=np.uint64)
    b = a.copy()
    b[1] = np.uint64(0xFFFFFFFFFFFFFFFF ^ pattern)
    p = run(bi, variant, lambda: to_host(bi.mul(to_dev(a), to_dev(b))))
    assert np.array_equal(p, orc.batch_mul(a, b))


@pytest.mark.parametrize("variant", NARROW)
@pytest.mark.parametrize("na,nb,m", [(512, 512, 513), (512, 512, 1), (512, 512, 9),
                                     (300, 4000, 2100), (1024, 1024, 1030), (2048, 2048, 2049)])
def test_low_part(bi, orc, variant, na, nb, m):
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(1000 + m, 3, na)
    b = inputs.limbs(1100 + m, 3, nb)
    got = run(bi, variant, lambda: to_host(bi.mul_lo(to_dev(a), to_dev(b), m)))
    want = np.stack([orc.mul_lo(a[i], b[i], m) for i in range(a.shape[0])])
    assert np.array_equal(got, want)


def test_model_choice_and_forced_shapes_agree(bi):
    """The shape the cost model picks and every forced shape give the same
    bytes (512 to 4096 limbs, a ragged pair and a low part)."""
    from paper_2607_28897_gb300 import inputs

    for na, nb in ((512, 512), (1024, 1024), (2048, 2048), (4096, 4096), (700, 2500)):
        a = to_dev(inputs.limbs(50 + na, 5, na))
        b = to_dev(inputs.limbs(51 + nb, 5, nb))
        ref = to_host(bi.mul(a, b))
        for v in (13, 14, 15, 16, 17):
            assert np.array_equal(run(bi, v, lambda: to_host(bi.mul(a, b))), ref), (na, nb, v)


@pytest.mark.parametrize("variant", NARROW)
@pytest.mark.parametrize("nu,nv,count", [(256, 128, 40), (1024, 512, 24), (1500, 700, 12),
                                         (4096, 2048, 6), (3000, 1100, 8)])
def test_division_products(bi, orc, variant, nu, nv, count):
    """The step-batched division with its tensor-core products forced to a
    narrow shape: low products and band products (tiles from S - 1 columns
    before limb lo's column, the limbs below it dropped) against the
    oracle, with adversarial divisors mixed in."""
    from paper_2607_28897_gb300 import inputs

    u = inputs.limbs(nu * 7 + variant, count, nu, top_nonzero=True)
    v = inputs.limbs(nv * 11 + variant, count, nv, top_nonzero=True)
    v[1, :] = np.uint64(0xFFFFFFFFFFFFFFFF)          # B^nv - 1
    v[2, :] = 0
    v[2, -1] = np.uint64(1)                           # B^(nv-1)
    v[3, -1] = np.uint64(1 << 63)
    u[4, :] = np.uint64(0xFFFFFFFFFFFFFFFF)
    q, r, st = run(bi, variant, lambda: bi.divmod(to_dev(u), to_dev(v)))
    oq, orr, ost = orc.batch_divmod(u, v)
    assert np.array_equal(st.cpu().numpy(), ost)
    assert np.array_equal(to_host(q), oq)
    assert np.array_equal(to_host(r), orr)
    bi.check_timeout()

