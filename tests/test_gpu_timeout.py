"""The tensor-core products' device waits give up cleanly.  With an
injected timeout (a negative wait limit: each wait, once the MMAs it guards
have finished, runs out on a flag that nothing sets) a multiply and a
division report BIGINT_ETIMEOUT (bigint_check_timeout, the division's
per-instance status), the CTAs release their tensor memory, and after the
default limit is restored the next calls on the same device are bit-exact
against the oracle.  No fault is involved."""
import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


def test_wait_limit_timeout_then_recovery(orc):
    import torch

    import paper_2607_28897_gb300 as bi
    from paper_2607_28897_gb300 import inputs

    a, b = inputs.config_small(seed=9, n=512, count=4)  # 2^15-bit tensor-core products
    u, v = inputs.config_div(1024, 4, seed=10)  # division with tensor-core products
    assert bi.mul_variant_for(512, 512) == 12
    bi.check_timeout()  # nothing recorded before
    bi.set_wait_limit(-2000)
    try:
        bi.mul(to_dev(a), to_dev(b))
        with pytest.raises(bi.BigIntError) as e:
            bi.check_timeout()
        assert e.value.code == bi.ETIMEOUT
        q, r, st = bi.divmod(to_dev(u), to_dev(v))
        torch.cuda.synchronize()
        st = st.cpu().numpy()
        assert (st == bi.ETIMEOUT).all(), st
        assert set(np.unique(st)) <= {0, bi.ETIMEOUT}, st
        with pytest.raises(bi.BigIntError) as e:
            bi.check_timeout()
        assert e.value.code == bi.ETIMEOUT
        # an instance that finished before any wait gave up is still exact
        oq, orr, _ = orc.batch_divmod(u, v)
        ok = st == 0
        assert np.array_equal(to_host(q)[ok], oq[ok]) and np.array_equal(to_host(r)[ok], orr[ok])
    finally:
        bi.set_wait_limit(0)
    bi.check_timeout()  # the record was cleared by the reads above
    p = bi.mul(to_dev(a), to_dev(b))
    assert np.array_equal(to_host(p), orc.batch_mul(a, b))
    q, r, st = bi.divmod(to_dev(u), to_dev(v))
    oq, orr, ost = orc.batch_divmod(u, v)
    assert np.array_equal(to_host(q), oq) and np.array_equal(to_host(r), orr)
    assert not st.cpu().numpy().any()
    bi.check_timeout()
