"""GPU parity of division by the shifted inverse (Sec. V-C, Fig. 6): q and r
bit-exact against the oracle's long division, status codes included."""
import numpy as np
import pytest

from helpers import SMALL_PRIMES, mulmod, residues, to_dev, to_host

pytestmark = pytest.mark.gpu

B = 1 << 64


@pytest.fixture(scope="module")
def bi():
    import paper_2607_28897_gb300 as m

    m.load()
    return m


def from_int(v, n):
    out = np.zeros(n, dtype=np.uint64)
    for i in range(n):
        out[i] = v & (B - 1)
        v >>= 64
    return out


def check_divmod(bi, orc, u, v):
    q, r, st = bi.divmod(to_dev(u), to_dev(v))
    oq, orr, ost = orc.batch_divmod(u, v)
    st = st.cpu().numpy()
    # the oracle reports a quotient that does not fit with its own code
    exp_st = np.where(ost == orc.EDIVZERO, bi.EDIVZERO, np.where(ost == orc.EINVAL, bi.ERANGE, 0))
    assert np.array_equal(st, exp_st), (st, exp_st)
    assert np.array_equal(to_host(q), oq)
    assert np.array_equal(to_host(r), orr)


@pytest.mark.parametrize("nu,nv", [(1, 1), (2, 1), (1, 2), (3, 2), (8, 3), (17, 16), (64, 32),
                                   (100, 7), (300, 299), (5, 7), (40, 1), (129, 64), (513, 256)])
def test_shapes(bi, orc, nu, nv):
    from paper_2607_28897_gb300 import inputs

    count = 12
    u = inputs.limbs(nu * 31 + nv, count, nu, top_nonzero=True)
    v = inputs.limbs(nu * 37 + nv, count, nv, top_nonzero=True)
    v[1::3, -1] = (v[1::3, -1] % np.uint64(1 << 32)) | np.uint64(1)  # small top limb
    v[2::3, -1] |= np.uint64(1 << 63)
    check_divmod(bi, orc, u, v)


def test_special_divisors(bi, orc):
    """B^k, B^k + 1, B^(k+1) - 1, a top limb of 1, divisors with leading zero
    limbs (quotient overflow), zero divisors, zero and small dividends."""
    nu, nv = 24, 10
    rows_u, rows_v = [], []
    rng = np.random.default_rng(3)

    def rnd(n):
        return int.from_bytes(rng.bytes(8 * n), "little")

    for k in (0, 1, 4, 9):
        for v in ((1 << (64 * k)), (1 << (64 * k)) + 1, (1 << (64 * (k + 1))) - 1,
                  (1 << (64 * k)) | rnd(k)):
            for u in (rnd(nu), (1 << (64 * nu)) - 1, v * rnd(2) + 12345 % max(v, 1), 0, 7):
                rows_u.append(from_int(u % (1 << (64 * nu)), nu))
                rows_v.append(from_int(v, nv))
    rows_u.append(from_int(rnd(nu), nu))
    rows_v.append(np.zeros(nv, dtype=np.uint64))  # division by zero
    check_divmod(bi, orc, np.stack(rows_u), np.stack(rows_v))


@pytest.mark.parametrize("n,batch", [(512, 4096), (2048, 1024)])
def test_config_div_full(bi, orc, n, batch):
    from paper_2607_28897_gb300 import inputs

    u, v = inputs.config_div(n, batch)
    check_divmod(bi, orc, u, v)


def test_config_div_8192(bi, orc):
    """n = 8192 (2^20-bit dividends), batch 256, in the bench's launch
    configuration: q v + r = u modulo three primes and r < v for every
    instance, and a full compare on a seeded sample."""
    from paper_2607_28897_gb300 import inputs

    u, v = inputs.config_div(8192, 256)
    q, r, st = bi.divmod(to_dev(u), to_dev(v))
    q, r, st = to_host(q), to_host(r), st.cpu().numpy()
    assert not st.any()
    for p in SMALL_PRIMES:
        lhs = (mulmod(residues(q, p), residues(v, p), p) + residues(r, p)) % np.uint64(p)
        assert np.array_equal(lhs, residues(u, p))
    # r < v: compare from the top limb down
    for i in range(u.shape[0]):
        diff = np.nonzero(r[i] != v[i])[0]
        assert diff.size and r[i][diff[-1]] < v[i][diff[-1]]
    idx = np.array([0, 1, 77, 200, 255])
    oq, orr, _ = orc.batch_divmod(u[idx], v[idx])
    assert np.array_equal(q[idx], oq) and np.array_equal(r[idx], orr)


@pytest.mark.parametrize("nv,h", [(1, 1), (1, 5), (2, 3), (3, 9), (16, 40), (64, 64), (100, 257),
                                  (512, 1024)])
def test_shinv(bi, orc, nv, h):
    from paper_2607_28897_gb300 import inputs

    count = 8
    v = inputs.limbs(nv * 101 + h, count, nv, top_nonzero=True)
    v[1::2, -1] = (v[1::2, -1] >> np.uint64(40)) | np.uint64(1)
    nw = h - nv + 2
    w, st = bi.shinv(to_dev(v), h, nw)
    w = to_host(w)
    assert not st.cpu().numpy().any()
    for i in range(count):
        ow, s = orc.shinv(v[i], h, nw)
        assert s == 0 and np.array_equal(w[i], ow), i


def test_shinv_power_of_base(bi):
    """shinv_h(B^k) = B^(h-k)."""
    k, h = 5, 23
    v = np.zeros((2, k + 1), dtype=np.uint64)
    v[:, k] = 1
    w, st = bi.shinv(to_dev(v), h, h - k + 1)
    w = to_host(w)
    assert not st.cpu().numpy().any()
    assert w[0][h - k] == 1 and not w[0][: h - k].any()
