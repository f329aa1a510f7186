"""GPU parity of division by a reused shifted inverse (bigint_divmod_inv):
w = floor(B^h / v) from bigint_shinv, then q, r for many dividends without
the Newton loop; q, r and status bit-exact against the oracle's division,
for one divisor shared by the batch and one per instance, h above the
dividends' precision, short dividends, and an inverse that is not one."""
import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bi():
    import paper_2607_28897_gb300 as m

    m.load()
    return m


def expect(bi, orc, u, v_rows):
    oq, orr, ost = orc.batch_divmod(u, v_rows)
    exp_st = np.where(ost == orc.EDIVZERO, bi.EDIVZERO, np.where(ost == orc.EINVAL, bi.ERANGE, 0))
    return oq, orr, exp_st


def run_case(bi, orc, u, v, h, shared):
    """v: (1, nv) shared or (count, nv); the inverse from shinv at h."""
    nv = v.shape[1]
    nw = h - nv + 2
    w, st = bi.shinv(to_dev(v), h, nw)
    assert not st.cpu().numpy().any()
    q, r, st = bi.divmod_inv(to_dev(u), to_dev(v), w, h)
    v_rows = np.repeat(v, u.shape[0], axis=0) if shared else v
    oq, orr, exp_st = expect(bi, orc, u, v_rows)
    assert np.array_equal(st.cpu().numpy(), exp_st)
    assert np.array_equal(to_host(q), oq)
    assert np.array_equal(to_host(r), orr)
    bi.check_timeout()


@pytest.mark.parametrize("nu,nv,h,count", [(600, 300, 600, 64), (500, 200, 900, 32),
                                           (2048, 1024, 2048, 8), (4096, 2048, 4096, 4),
                                           (1536, 9, 1600, 8), (40, 40, 40, 16)])
def test_shared_divisor(bi, orc, nu, nv, h, count):
    """One divisor and its inverse for the whole batch (strides 0)."""
    from paper_2607_28897_gb300 import inputs

    u = inputs.limbs(2000 + nu, count, nu)
    v = inputs.limbs(2100 + nv, 1, nv)
    v[0, -1] |= np.uint64(1 << 63)
    run_case(bi, orc, u, v, h, shared=True)


@pytest.mark.parametrize("nu,nv,h,count", [(700, 350, 700, 24), (2100, 1000, 2500, 6)])
def test_per_instance_divisors(bi, orc, nu, nv, h, count):
    from paper_2607_28897_gb300 import inputs

    u = inputs.limbs(2200 + nu, count, nu)
    v = inputs.limbs(2300 + nv, count, nv)
    v[:, -1] |= np.uint64(1)
    run_case(bi, orc, u, v, h, shared=False)


def test_short_dividends(bi, orc):
    """Dividends of every precision under h (the inverse's low limbs are
    dropped per instance), zero, below and equal to the divisor."""
    from paper_2607_28897_gb300 import inputs

    nu, nv, h, count = 512, 100, 640, 12
    u = inputs.limbs(2400, count, nu)
    v = inputs.limbs(2401, 1, nv)
    v[0, -1] |= np.uint64(1 << 40)
    for i, top in enumerate([512, 400, 300, 200, 150, 101, 100, 99, 50, 1, 0]):
        u[i, top:] = 0
    u[count - 1, :] = 0
    u[count - 1, :nv] = v[0]  # u = v: q = 1, r = 0
    run_case(bi, orc, u, v, h, shared=True)


def test_not_an_inverse(bi, orc):
    """An all-ones w overshoots the quotient by far more than the correction
    rounds: status EINTERNAL, no hang or fault."""
    from paper_2607_28897_gb300 import inputs

    nu, nv, h, count = 400, 100, 400, 4
    u = inputs.limbs(2500, count, nu)
    v = inputs.limbs(2501, 1, nv)
    v[0, -1] |= np.uint64(1 << 63)
    w = np.full((1, h - nv + 2), np.uint64(0xFFFFFFFFFFFFFFFF), dtype=np.uint64)
    q, r, st = bi.divmod_inv(to_dev(u), to_dev(v), to_dev(w), h)
    assert (st.cpu().numpy() == bi.EINTERNAL).all()
    bi.check_timeout()
