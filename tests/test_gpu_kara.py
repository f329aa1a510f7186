"""GPU parity of the Karatsuba full product (bigint_mul_kara) against the
oracle: one to three levels over the tensor-core and integer leaf
products, operands whose halves compare either way or are equal (the
middle term's sign and a zero difference), all-ones and zero operands, the
batch cut into chunks by a short workspace, and bit-identity with
bigint_mul."""
import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bi():
    import paper_2607_28897_gb300 as m

    m.load()
    return m


def operands(n, count, seed):
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(seed, count, n)
    b = inputs.limbs(seed + 1, count, n)
    k = n // 2
    if count > 5 and k > 0:
        a[1] = np.uint64(0xFFFFFFFFFFFFFFFF)           # all ones
        b[1] = np.uint64(0xFFFFFFFFFFFFFFFF)
        a[2, :k] = a[2, k:2 * k]                       # x0 = x1: zero difference
        b[3, k:2 * k] = b[3, :k]                       # y1 = y0
        a[4, :k] = 0                                   # x0 < x1
        b[4, :k] = np.uint64(0xFFFFFFFFFFFFFFFF)       # y1 < y0
        a[5] = 0                                       # a zero operand
    return a, b


@pytest.mark.parametrize("n,levels", [(2, 1), (8, 3), (64, 2), (512, 1), (1024, 1), (1024, 2),
                                      (1024, 3), (2048, 1), (4096, -1), (4096, 2), (8192, -1),
                                      (1000, 3), (1002, 2), (3000, -1)])
def test_against_oracle(bi, orc, n, levels):
    count = 7
    a, b = operands(n, count, 300 + n)
    got = to_host(bi.mul_kara(to_dev(a), to_dev(b), levels))
    assert np.array_equal(got, orc.batch_mul(a, b)), (n, levels)
    bi.check_timeout()


def test_chunked_workspace(bi, orc):
    """A workspace for 3 of 40 instances: the batch runs in chunks."""
    import torch

    n, count = 2048, 40
    a, b = operands(n, count, 71)
    full = bi.mul_kara_workspace_bytes(count, n, 1)
    part = bi.mul_kara_workspace_bytes(3, n, 1)
    assert 0 < part < full
    ws = torch.empty(part, dtype=torch.uint8, device="cuda")
    got = to_host(bi.mul_kara(to_dev(a), to_dev(b), 1, workspace=ws))
    assert np.array_equal(got, orc.batch_mul(a, b))


def test_workspace_too_small(bi):
    import torch

    n = 2048
    a, b = operands(n, 4, 9)
    ws = torch.empty(bi.mul_kara_workspace_bytes(1, n, 1) - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(bi.BigIntError):
        bi.mul_kara(to_dev(a), to_dev(b), 1, workspace=ws)


@pytest.mark.parametrize("n", [4096, 8192])
def test_same_as_mul(bi, n):
    """Many instances (more than the resident CTAs of every launch): the
    Karatsuba form and bigint_mul give the same bytes."""
    from paper_2607_28897_gb300 import inputs

    count = 400 if n == 4096 else 200
    a = to_dev(inputs.limbs(5 + n, count, n))
    b = to_dev(inputs.limbs(6 + n, count, n))
    assert np.array_equal(to_host(bi.mul_kara(a, b)), to_host(bi.mul(a, b)))
