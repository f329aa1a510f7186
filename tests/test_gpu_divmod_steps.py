"""Division in the step-batched form (divstep.cu: every Newton step batched
across the instances, products on the batched multiply kernels, irregular
instances left to the one-CTA-per-division kernel) against the oracle's long
division, and against the one-CTA-per-division form, bit for bit."""
import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu

B = 1 << 64


@pytest.fixture(scope="module")
def bi():
    import paper_2607_28897_gb300 as m

    m.load()
    yield m
    m.set_variant(1, 0)


def from_int(x, n):
    out = np.zeros(n, dtype=np.uint64)
    for i in range(n):
        out[i] = x & (B - 1)
        x >>= 64
    return out


def run(bi, u, v, variant):
    bi.set_variant(1, variant)
    try:
        q, r, st = bi.divmod(to_dev(u), to_dev(v))
        return to_host(q), to_host(r), st.cpu().numpy()
    finally:
        bi.set_variant(1, 0)


def expect(bi, orc, u, v):
    oq, orr, ost = orc.batch_divmod(u, v)
    est = np.where(ost == orc.EDIVZERO, bi.EDIVZERO, np.where(ost == orc.EINVAL, bi.ERANGE, 0))
    return oq, orr, est


@pytest.mark.parametrize("nu,nv", [(16, 8), (17, 8), (40, 9), (64, 64), (65, 64), (300, 150),
                                   (513, 256), (700, 300), (1024, 512), (1500, 1499),
                                   (3000, 1100), (2048, 1024)])
def test_step_form_shapes(bi, orc, nu, nv):
    """Forced step-batched form (variant 3) on ragged shapes, small to 2^17
    bits, both divisor families of the division workload."""
    from paper_2607_28897_gb300 import inputs

    count = 24
    u = inputs.limbs(nu * 13 + nv, count, nu, top_nonzero=True)
    v = inputs.limbs(nu * 17 + nv, count, nv, top_nonzero=True)
    v[1::2, -1] = (v[1::2, -1] % np.uint64(1 << 32)) | np.uint64(1)
    v[::4, -1] |= np.uint64(1 << 63)
    u[3::6, nu - nu // 3:] = 0  # dividends with leading zero limbs stay on the step path
    q, r, st = run(bi, u, v, 3)
    oq, orr, est = expect(bi, orc, u, v)
    assert np.array_equal(st, est)
    assert np.array_equal(q, oq) and np.array_equal(r, orr)


def test_step_form_adversarial_and_irregular(bi, orc):
    """One batch mixing regular instances with adversarial divisors (B^k,
    B^k + 1, B^(k+1) - 1, top limb 1, all limbs 0x80..0) and irregular ones
    (divisor or dividend with zero top limbs, zero divisor, quotient
    overflow): the step form and the one-CTA form agree with the oracle."""
    nu, nv = 600, 300
    k = nv - 1
    rng = np.random.default_rng(11)

    def rnd(n):
        return int.from_bytes(rng.bytes(8 * n), "little")

    divisors = [1 << (64 * k), (1 << (64 * k)) + 1, (1 << (64 * nv)) - 1,
                (1 << (64 * k)) | rnd(k), int.from_bytes(b"\x00" * 7 + b"\x80", "little") *
                sum(1 << (64 * i) for i in range(nv)),
                rnd(nv) | (1 << (64 * nv - 1))]
    rows_u, rows_v = [], []
    for d in divisors:
        for x in (rnd(nu) | (1 << (64 * nu - 1)), (1 << (64 * nu)) - 1, d * (rnd(nu - nv) |
                  (1 << (64 * (nu - nv) - 1))) + (d - 1), (1 << (64 * (nu - 1)))):
            rows_u.append(from_int(x % (1 << (64 * nu)), nu))
            rows_v.append(from_int(d, nv))
    # irregular: zero top limb of the divisor (a quotient that may not fit),
    # zero top limb of the dividend, a zero divisor, a divisor of one limb
    rows_u += [from_int(rnd(nu) | 1 << (64 * nu - 1), nu), from_int(rnd(nu - 3), nu),
               from_int(rnd(nu), nu), from_int(rnd(nu), nu)]
    rows_v += [from_int(rnd(nv - 1) | 1, nv), from_int(rnd(nv) | 1 << (64 * nv - 1), nv),
               np.zeros(nv, dtype=np.uint64), from_int(12345, nv)]
    u, v = np.stack(rows_u), np.stack(rows_v)
    oq, orr, est = expect(bi, orc, u, v)
    for variant in (3, 1):
        q, r, st = run(bi, u, v, variant)
        assert np.array_equal(st, est), (variant, st, est)
        assert np.array_equal(q, oq), variant
        assert np.array_equal(r, orr), variant


@pytest.mark.parametrize("n,count", [(512, 96), (2048, 20), (8192, 3)])
def test_default_form_equals_one_cta_form(bi, n, count):
    """The default (step-batched at these sizes) and the one-CTA-per-division
    forms give the same bits on the division workload's operands."""
    from paper_2607_28897_gb300 import inputs

    u, v = inputs.config_div(n, count, seed=77)
    a = run(bi, u, v, 0)
    b = run(bi, u, v, 1)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert not a[2].any()


def test_single_division_2_20_bits(bi, orc):
    """One 2^20 / 2^19-bit division alone (the latency case): every product
    of its steps is one launch over the whole GPU."""
    from paper_2607_28897_gb300 import inputs

    u, v = inputs.config_div(8192, 2, seed=78)
    u, v = u[1:], v[1:]  # the divisor with a small top limb
    q, r, st = run(bi, u, v, 0)
    oq, orr, est = expect(bi, orc, u, v)
    assert np.array_equal(st, est) and np.array_equal(q, oq) and np.array_equal(r, orr)
