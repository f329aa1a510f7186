"""GPU parity of the host-buffer entry points (bigint_*_host): the same
results as the device entry points and the oracle, with pinned and pageable
host buffers, many chunks, and a workspace too small for one instance."""
import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bi():
    import paper_2607_28897_gb300 as m

    m.load()
    return m


def host(x, pinned=True):
    import torch

    t = torch.from_numpy(np.ascontiguousarray(x).view(np.int64)).clone()
    return t.pin_memory() if pinned else t


def ws_for(bi, op, chunk, na, nb):
    import torch

    return torch.empty(bi.host_workspace_bytes(op, chunk, na, nb), dtype=torch.uint8,
                       device="cuda")


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("chunk", [1, 3, 64])
def test_mul_host(bi, orc, pinned, chunk):
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(71, 20, 300)
    b = inputs.limbs(72, 20, 257)
    ws = ws_for(bi, bi.OP_MUL, chunk, 300, 257)
    out = bi.mul_host(host(a, pinned), host(b, pinned), workspace=ws)
    assert np.array_equal(out.numpy().view(np.uint64), orc.batch_mul(a, b))


def test_mul_host_tensor_cores(bi):
    """Large products (tensor-core kernel) through the host path equal the
    device entry point's."""
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(73, 24, 2048)
    b = inputs.limbs(74, 24, 2048)
    ws = ws_for(bi, bi.OP_MUL, 5, 2048, 2048)
    out = bi.mul_host(host(a), host(b), workspace=ws).numpy().view(np.uint64)
    assert np.array_equal(out, to_host(bi.mul(to_dev(a), to_dev(b))))


def test_mul_host_karatsuba(bi, orc):
    """Square products of 4096 and 8192 limbs take the Karatsuba form in the
    host path (its workspace inside each staging slot): the oracle's
    products, over several chunks."""
    from paper_2607_28897_gb300 import inputs

    for n, count in ((4096, 7), (8192, 5)):
        a = inputs.limbs(75 + n, count, n)
        b = inputs.limbs(76 + n, count, n)
        a[0] = np.uint64(0xFFFFFFFFFFFFFFFF)
        ws = ws_for(bi, bi.OP_MUL, 2, n, n)
        out = bi.mul_host(host(a), host(b), workspace=ws).numpy().view(np.uint64)
        assert np.array_equal(out, orc.batch_mul(a, b)), n


@pytest.mark.parametrize("sub", [False, True])
def test_addsub_host(bi, orc, sub):
    import torch
    from paper_2607_28897_gb300 import inputs

    a = inputs.limbs(75, 33, 1024)
    b = inputs.limbs(76, 33, 1024)
    a[::4] = np.uint64(0xFFFFFFFFFFFFFFFF)
    flag = torch.zeros(33, dtype=torch.uint8).pin_memory()
    ws = ws_for(bi, bi.OP_ADD, 4, 1024, 1024)
    fn = bi.sub_host if sub else bi.add_host
    out = fn(host(a), host(b), workspace=ws, **({"borrow": flag} if sub else {"carry": flag}))
    want, wflag = (orc.batch_sub if sub else orc.batch_add)(a, b)
    assert np.array_equal(out.numpy().view(np.uint64), want)
    assert np.array_equal(flag.numpy(), wflag)


@pytest.mark.parametrize("nu,nv,chunk", [(64, 30, 2), (4096, 2048, 3)])
def test_divmod_host(bi, orc, nu, nv, chunk):
    from paper_2607_28897_gb300 import inputs

    u = inputs.limbs(77 + nu, 10, nu, top_nonzero=True)
    v = inputs.limbs(78 + nv, 10, nv, top_nonzero=True)
    v[3] = 0  # a zero divisor: status EDIVZERO, q = r = 0
    ws = ws_for(bi, bi.OP_DIVMOD, chunk, nu, nv)
    q, r, st = bi.divmod_host(host(u), host(v), workspace=ws)
    oq, orr, ost = orc.batch_divmod(u, v)
    assert np.array_equal(q.numpy().view(np.uint64), oq)
    assert np.array_equal(r.numpy().view(np.uint64), orr)
    exp = np.where(ost == orc.EDIVZERO, bi.EDIVZERO, 0)
    assert np.array_equal(st.numpy(), exp)


def test_workspace_too_small(bi):
    import torch

    a = host(np.ones((4, 512), dtype=np.uint64))
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(bi.BigIntError):
        bi.mul_host(a, a, workspace=ws)


def test_async_calls_share_a_workspace(bi, orc):
    """Enqueued calls of different operations and shapes on ONE workspace
    (each carves it differently), then one host_sync: every result equals
    the oracle's, so a call never overwrites a region an earlier call still
    copies out of."""
    import torch
    from paper_2607_28897_gb300 import inputs

    n = 256
    a = inputs.limbs(81, 24, n)
    b = inputs.limbs(82, 24, n)
    u = inputs.limbs(83, 24, 2 * n, top_nonzero=True)
    v = inputs.limbs(84, 24, n, top_nonzero=True)
    big = max(bi.host_workspace_bytes(op, 3, 2 * n if op == bi.OP_DIVMOD else n, n)
              for op in (bi.OP_ADD, bi.OP_SUB, bi.OP_MUL, bi.OP_DIVMOD))
    ws = torch.empty(big, dtype=torch.uint8, device="cuda")
    ha, hb, hu, hv = host(a), host(b), host(u), host(v)
    carry = torch.zeros(24, dtype=torch.uint8).pin_memory()
    borrow = torch.zeros(24, dtype=torch.uint8).pin_memory()
    outs = []
    for rep in range(3):
        s = bi.add_host(ha, hb, carry=carry, workspace=ws, sync=False)
        d = bi.sub_host(ha, hb, borrow=borrow, workspace=ws, sync=False)
        p = bi.mul_host(ha, hb, workspace=ws, sync=False)
        q, r, st = bi.divmod_host(hu, hv, workspace=ws, sync=False)
        outs.append((s, d, p, q, r, st))
    bi.host_sync()
    ws_add = orc.batch_add(a, b)
    ws_sub = orc.batch_sub(a, b)
    prod = orc.batch_mul(a, b)
    oq, orr, _ = orc.batch_divmod(u, v)
    for s, d, p, q, r, st in outs:
        assert np.array_equal(s.numpy().view(np.uint64), ws_add[0])
        assert np.array_equal(d.numpy().view(np.uint64), ws_sub[0])
        assert np.array_equal(p.numpy().view(np.uint64), prod)
        assert np.array_equal(q.numpy().view(np.uint64), oq)
        assert np.array_equal(r.numpy().view(np.uint64), orr)
        assert not st.numpy().any()
    assert np.array_equal(carry.numpy(), ws_add[1])
    assert np.array_equal(borrow.numpy(), ws_sub[1])
