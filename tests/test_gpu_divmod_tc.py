"""GPU parity of division whose large products run on the tensor cores
(operands of 2048 limbs and more, division variant 0/1): q, r and status
bit-exact against the oracle, the same results as the integer-product
kernel (variant 2), shifted inverses, and the wait-limit record."""
import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu

B = 1 << 64


@pytest.fixture(scope="module")
def bi():
    import paper_2607_28897_gb300 as m

    m.load()
    m.set_variant(1, 0)
    yield m
    m.set_variant(1, 0)


def from_int(v, n):
    out = np.zeros(n, dtype=np.uint64)
    for i in range(n):
        out[i] = v & (B - 1)
        v >>= 64
    return out


def check(bi, orc, u, v):
    q, r, st = bi.divmod(to_dev(u), to_dev(v))
    oq, orr, ost = orc.batch_divmod(u, v)
    st = st.cpu().numpy()
    exp_st = np.where(ost == orc.EDIVZERO, bi.EDIVZERO, np.where(ost == orc.EINVAL, bi.ERANGE, 0))
    assert np.array_equal(st, exp_st), (st, exp_st)
    assert np.array_equal(to_host(q), oq)
    assert np.array_equal(to_host(r), orr)
    bi.check_timeout()


@pytest.mark.parametrize("nu,nv", [(2048, 1024), (2048, 256), (2048, 300), (2048, 1800),
                                   (2048, 2048), (3000, 1500), (4096, 2), (4096, 700),
                                   (5000, 4999), (2100, 7), (6000, 2500), (1536, 768),
                                   (1536, 1), (1600, 800), (1535, 700)])
def test_shapes(bi, orc, nu, nv):
    from paper_2607_28897_gb300 import inputs

    count = 6
    u = inputs.limbs(nu * 13 + nv, count, nu, top_nonzero=True)
    v = inputs.limbs(nu * 17 + nv, count, nv, top_nonzero=True)
    v[1::3, -1] = (v[1::3, -1] % np.uint64(1 << 32)) | np.uint64(1)  # small top limb
    v[2::3, -1] |= np.uint64(1 << 63)
    check(bi, orc, u, v)


def test_special_divisors(bi, orc):
    """B^k, B^k + 1, B^(k+1) - 1, B^k plus noise, divisors with leading zero
    limbs (quotient overflow), a zero divisor, zero and small dividends, at
    2304 / 1100 limbs."""
    nu, nv = 2304, 1100
    rows_u, rows_v = [], []
    rng = np.random.default_rng(11)

    def rnd(n):
        return int.from_bytes(rng.bytes(8 * n), "little")

    for k in (300, 700, 1099):
        for v in ((1 << (64 * k)), (1 << (64 * k)) + 1, (1 << (64 * (k + 1))) - 1,
                  (1 << (64 * k)) | rnd(k)):
            for u in (rnd(nu), (1 << (64 * nu)) - 1, v * rnd(3) + 99, 0, 7):
                rows_u.append(from_int(u % (1 << (64 * nu)), nu))
                rows_v.append(from_int(v, nv))
    rows_u.append(from_int(rnd(nu), nu))
    rows_v.append(np.zeros(nv, dtype=np.uint64))
    check(bi, orc, np.stack(rows_u), np.stack(rows_v))


def test_quotient_near_power(bi, orc):
    """u = q v + r with q = B^j - 1 or B^j and r = 0, 1 or v - 1: the
    quotient estimate's band error crosses a limb boundary."""
    nu, nv = 4096, 2048
    rng = np.random.default_rng(5)
    rows_u, rows_v = [], []
    for j in (1, 1000, 2047):
        v = int.from_bytes(rng.bytes(8 * nv), "little") | (1 << (64 * nv - 1))
        for q in ((1 << (64 * j)) - 1, 1 << (64 * j)):
            for r in (0, 1, v - 1):
                u = q * v + r
                if u < (1 << (64 * nu)):
                    rows_u.append(from_int(u, nu))
                    rows_v.append(from_int(v, nv))
    check(bi, orc, np.stack(rows_u), np.stack(rows_v))


@pytest.mark.parametrize("n,count", [(768, 64), (2048, 48), (8192, 6)])
def test_same_as_integer_products(bi, n, count):
    from paper_2607_28897_gb300 import inputs

    u, v = inputs.config_div(n, count)
    du, dv = to_dev(u), to_dev(v)
    q0, r0, s0 = bi.divmod(du, dv)
    bi.set_variant(1, 2)
    try:
        q2, r2, s2 = bi.divmod(du, dv)
    finally:
        bi.set_variant(1, 0)
    assert np.array_equal(to_host(q0), to_host(q2))
    assert np.array_equal(to_host(r0), to_host(r2))
    assert np.array_equal(s0.cpu().numpy(), s2.cpu().numpy())


@pytest.mark.parametrize("nv,h", [(2048, 4096), (1500, 2100), (300, 5000), (4096, 4096),
                                  (768, 1536)])
def test_shinv(bi, orc, nv, h):
    from paper_2607_28897_gb300 import inputs

    v = inputs.limbs(nv + h, 4, nv, top_nonzero=True)
    v[1, -1] = np.uint64(1)
    nw = h - nv + 2
    w, st = bi.shinv(to_dev(v), h, nw)
    w = to_host(w)
    assert not st.cpu().numpy().any()
    for i in range(v.shape[0]):
        ow, ost = orc.shinv(v[i], h, nw)
        assert ost == 0 and np.array_equal(w[i], ow)
    bi.check_timeout()
