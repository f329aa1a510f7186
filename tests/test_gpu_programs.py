"""GPU parity of the fused programs (Sec. VI, Tables I and II): the add
chain (6-Add is k = 6) and Poly = (a a + b)(b b + b) + a b mod B^n, bit-exact
against the oracle."""
import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bi():
    import paper_2607_28897_gb300 as m

    m.load()
    return m


@pytest.mark.parametrize("n", [1, 7, 64, 511, 512, 1000, 8192, 9000])
@pytest.mark.parametrize("k", [1, 6, 13])
def test_add_chain(bi, orc, n, k):
    import torch
    from paper_2607_28897_gb300 import inputs

    count = 6
    a = inputs.limbs(500 + n, count, n)
    b = inputs.limbs(600 + n + k, count, n)
    a[0] = np.uint64(0xFFFFFFFFFFFFFFFF)  # all-ones chains: carries cross every limb
    b[0] = np.uint64(0xFFFFFFFFFFFFFFFF)
    b[1] = 0
    b[1, 0] = 1
    a[1] = np.uint64(0xFFFFFFFFFFFFFFFF)
    carry = torch.zeros(count, dtype=torch.uint8, device="cuda")
    out = to_host(bi.add_chain(to_dev(a), to_dev(b), k, carry=carry))
    for i in range(count):
        want, c = orc.add_chain(a[i], b[i], k)
        assert np.array_equal(out[i], want), i
        assert int(carry[i]) == c, i


@pytest.mark.parametrize("n", [1, 5, 100, 255, 256, 300, 512, 1024, 1025, 2048, 2049, 4096])
def test_poly(bi, orc, n):
    from paper_2607_28897_gb300 import inputs

    count = 5 if n <= 1024 else 3
    a = inputs.limbs(700 + n, count, n)
    b = inputs.limbs(800 + n, count, n)
    a[0] = np.uint64(0xFFFFFFFFFFFFFFFF)
    out = to_host(bi.poly(to_dev(a), to_dev(b)))
    for i in range(count):
        assert np.array_equal(out[i], orc.poly(a[i], b[i])), i
    bi.check_timeout()


def test_poly_many_instances(bi, orc):
    """More instances than resident CTAs (four per SM with the 64-column
    tile): the per-CTA scratch is reused."""
    from paper_2607_28897_gb300 import inputs

    n, count = 384, 1500
    a = inputs.limbs(901, count, n)
    b = inputs.limbs(902, count, n)
    out = to_host(bi.poly(to_dev(a), to_dev(b)))
    for i in (0, 1, 151, 152, 153, 607, 608, 609, 1216, 1499):
        assert np.array_equal(out[i], orc.poly(a[i], b[i])), i
