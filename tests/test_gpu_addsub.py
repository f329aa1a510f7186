"""GPU parity of add/sub (Sec. V-A) against the CPU oracle: bit-exact."""
import numpy as np
import pytest

from helpers import SMALL_PRIMES, residues, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bi():
    import paper_2607_28897_gb300 as m

    m.load()
    return m


def check_add(bi, orc, a, b):
    s, c = bi.add(to_dev(a), to_dev(b))
    ro, rc = orc.batch_add(a, b)
    assert np.array_equal(to_host(s), ro)
    assert np.array_equal(c.cpu().numpy(), rc)


def check_sub(bi, orc, a, b):
    d, br = bi.sub(to_dev(a), to_dev(b))
    ro, rb = orc.batch_sub(a, b)
    assert np.array_equal(to_host(d), ro)
    assert np.array_equal(br.cpu().numpy(), rb)


def test_config_small_add_sub(bi, orc):
    from paper_2607_28897_gb300 import inputs

    a, b = inputs.config_small(seed=1, n=512, count=64)
    check_add(bi, orc, a, b)
    sa, sb = inputs.order_pairs(a, b)
    check_sub(bi, orc, sa, sb)
    check_sub(bi, orc, a, b)  # unordered pairs: borrow out and wrap-around


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 63, 64, 65, 127, 129, 511, 513, 1000,
                               2047, 4097, 8191, 8192, 12289, 16384])
def test_ragged_lengths(bi, orc, n):
    from paper_2607_28897_gb300 import inputs

    count = 9
    a = inputs.limbs(100 + n, count, n)
    b = inputs.limbs(200 + n, count, n)
    sa, sb = inputs.stress_pairs(max(n, 2))
    a = np.concatenate([a, sa[:, :n]])
    b = np.concatenate([b, sb[:, :n]])
    check_add(bi, orc, a, b)
    check_sub(bi, orc, a, b)


def test_unaligned_buffers(bi, orc):
    """Instances that start on an 8-byte (not 16-byte) boundary take the
    one-limb-per-lane path."""
    import torch
    from paper_2607_28897_gb300 import inputs

    n, count = 515, 7
    a = inputs.limbs(5, count, n)
    b = inputs.limbs(6, count, n)
    buf_a = torch.zeros(count * n + 1, dtype=torch.int64, device="cuda:0")
    buf_b = torch.zeros_like(buf_a)
    buf_o = torch.zeros_like(buf_a)
    buf_a[1:].copy_(to_dev(a).view(-1))
    buf_b[1:].copy_(to_dev(b).view(-1))
    da, db, do = (x[1:].view(count, n) for x in (buf_a, buf_b, buf_o))
    s, c = bi.add(da, db, out=do)
    ro, rc = orc.batch_add(a, b)
    assert np.array_equal(to_host(s), ro) and np.array_equal(c.cpu().numpy(), rc)


def test_empty_batch(bi):
    import torch

    a = torch.zeros((0, 8), dtype=torch.int64, device="cuda:0")
    s, c = bi.add(a, a)
    assert s.shape == (0, 8)


def test_errors(bi):
    import torch

    a = torch.zeros((2, bi.MAX_LIMBS + 1), dtype=torch.int64, device="cuda:0")
    with pytest.raises(bi.BigIntError):
        bi.add(a, a)


@pytest.mark.parametrize("n", [512, 8192])
def test_config_sweep_full_size(bi, orc, n):
    """The full 2^32-bit operand arrays: every instance vs the oracle."""
    from paper_2607_28897_gb300 import inputs

    a, b = inputs.config_sweep(n)
    check_add(bi, orc, a, b)
    sa, sb = inputs.order_pairs(a, b)
    d, br = bi.sub(to_dev(sa), to_dev(sb))
    ro, rb = orc.batch_sub(sa, sb)
    assert np.array_equal(to_host(d), ro) and not br.cpu().numpy().any()
    # residues: (a - b) + b == a mod p for every instance
    for p in SMALL_PRIMES[:1]:
        assert np.array_equal((residues(to_host(d), p) + residues(sb, p)) % p, residues(sa, p))
