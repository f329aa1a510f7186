"""Ragged mixed-op batches: persistent (work queue) and per-class launches
give bit-exactly the oracle's results, and every result is the same alone
and in the mix."""
import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


def oracle_results(orc, ops, pool, threads=16):
    """Expected output pool and statuses from the oracle, op by op (each
    operation computed alone; the oracle's C calls release the GIL, so a
    thread pool runs them side by side)."""
    from concurrent.futures import ThreadPoolExecutor

    def one(i):
        o = ops[i]
        a = pool[o["a"]:o["a"] + o["na"]]
        b = pool[o["b"]:o["b"] + o["nb"]]
        if o["op"] == 1:
            r, c = orc.add(a, b)
            return (r,), c
        if o["op"] == 2:
            r, c = orc.sub(a, b)
            return (r,), c
        if o["op"] == 3:
            return (orc.mul(a, b),), 0
        q, r, s = orc.divmod_(a, b)
        return (q, r), {0: 0, 2: -2, 1: -7}[s]

    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(one, range(len(ops))))
    out = {i: r for i, (r, _) in enumerate(res)}
    st = np.array([s for _, s in res], dtype=np.int32)
    return out, st


def check(ops, got_pool, got_st, exp, exp_st):
    assert np.array_equal(got_st, exp_st)
    for i, o in enumerate(ops):
        if o["op"] == 4:
            q, r = exp[i]
            assert np.array_equal(got_pool[o["o1"]:o["o1"] + q.size], q), i
            assert np.array_equal(got_pool[o["o2"]:o["o2"] + r.size], r), i
        else:
            (r,) = exp[i]
            assert np.array_equal(got_pool[o["o1"]:o["o1"] + r.size], r), i


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_small_ragged(orc, mode):
    import torch

    import paper_2607_28897_gb300 as bi
    from paper_2607_28897_gb300 import inputs

    ops, nin, nout = inputs.ragged_ops(7, 300, min_limbs=1, max_limbs=700)
    pool = inputs.ragged_pool(8, ops, nin)
    exp, exp_st = oracle_results(orc, ops, pool)
    dpool = to_dev(pool)[None, :].view(-1)
    dout = torch.zeros(nout, dtype=torch.int64, device="cuda")
    st = torch.zeros(len(ops), dtype=torch.int32, device="cuda")
    B = bi.Batch(ops)
    B.launch(dpool, dout, st, mode=mode)
    torch.cuda.synchronize()
    check(ops, to_host(dout), st.cpu().numpy(), exp, exp_st)


def test_batch_alone_equals_mix(orc):
    """Each operation run alone (a batch of one) gives the same bits as in
    the mixed batch (persistent form)."""
    import torch

    import paper_2607_28897_gb300 as bi
    from paper_2607_28897_gb300 import inputs

    ops, nin, nout = inputs.ragged_ops(11, 60, min_limbs=8, max_limbs=2000)
    pool = to_dev(inputs.ragged_pool(12, ops, nin)).view(-1)
    mix_out = torch.zeros(nout, dtype=torch.int64, device="cuda")
    mix_st = torch.zeros(len(ops), dtype=torch.int32, device="cuda")
    bi.Batch(ops).launch(pool, mix_out, mix_st)
    for i in range(len(ops)):
        one = ops[i:i + 1].copy()
        alone_out = torch.zeros(nout, dtype=torch.int64, device="cuda")
        alone_st = torch.zeros(1, dtype=torch.int32, device="cuda")
        bi.Batch(one).launch(pool, alone_out, alone_st)
        o = ops[i]
        n_out = {1: o["na"], 2: o["na"], 3: o["na"] + o["nb"]}.get(int(o["op"]), 0)
        if o["op"] == 4:
            nq = max(o["na"] - o["nb"] + 1, 1)
            n_out = nq + o["nb"]
        s = slice(int(o["o1"]), int(o["o1"]) + int(n_out))
        assert torch.equal(alone_out[s], mix_out[s]), i
        assert int(alone_st[0]) == int(mix_st[i]), i


def test_batch_tune_and_graph(orc):
    """The autotuner picks a CTA size; a CUDA-graph replay of the persistent
    launch gives the oracle's results."""
    import torch

    import paper_2607_28897_gb300 as bi
    from paper_2607_28897_gb300 import inputs

    ops, nin, nout = inputs.ragged_ops(21, 120, min_limbs=16, max_limbs=1500)
    pool = inputs.ragged_pool(22, ops, nin)
    exp, exp_st = oracle_results(orc, ops, pool)
    dpool = to_dev(pool).view(-1)
    dout = torch.zeros(nout, dtype=torch.int64, device="cuda")
    st = torch.zeros(len(ops), dtype=torch.int32, device="cuda")
    B = bi.Batch(ops)
    best = B.tune(dpool, dout, st)
    assert best in (256, 384, 512, 544)  # 544: the tensor-core form
    dout.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        B.launch(dpool, dout, st, stream=s)  # warm-up on the capture stream
        torch.cuda.synchronize()
        dout.zero_()
        with torch.cuda.graph(g, stream=s):
            B.launch(dpool, dout, st, stream=s)
    g.replay()
    torch.cuda.synchronize()
    check(ops, to_host(dout), st.cpu().numpy(), exp, exp_st)
    bi.set_variant(0, 0)


@pytest.mark.parametrize("mode", [0, 1])
def test_batch_tensor_cores_equal_integer(orc, mode):
    """Large ragged operations (up to 6000 limbs): the tensor-core launches
    (batch variant 0) and integer-only launches (variant 2) give the same
    bits, and the oracle's."""
    import torch

    import paper_2607_28897_gb300 as bi
    from paper_2607_28897_gb300 import inputs

    ops, nin, nout = inputs.ragged_ops(31, 60, min_limbs=200, max_limbs=6000)
    pool = inputs.ragged_pool(32, ops, nin)
    exp, exp_st = oracle_results(orc, ops, pool)
    dpool = to_dev(pool).view(-1)
    results = []
    for variant in (0, 2):
        bi.set_variant(2, variant)
        try:
            dout = torch.zeros(nout, dtype=torch.int64, device="cuda")
            st = torch.zeros(len(ops), dtype=torch.int32, device="cuda")
            bi.Batch(ops).launch(dpool, dout, st, mode=mode)
            torch.cuda.synchronize()
            results.append((to_host(dout), st.cpu().numpy()))
        finally:
            bi.set_variant(2, 0)
    bi.check_timeout()
    (p0, s0), (p2, s2) = results
    check(ops, p0, s0, exp, exp_st)
    assert np.array_equal(s0, s2)
    check(ops, p2, s2, exp, exp_st)


def config4_slice(count, seed_ops=4, seed_pool=5):
    """The first `count` operations of the batched workload (200k ragged
    instances, 2^15..2^19 bits, 40 % mul / 15 % add / 15 % sub / 30 %
    divmod; the same seeds as the bench) followed by four operations at the
    largest sizes: 8192 x 8192-limb products, 16384 / 8192-limb divisions
    (one with a divisor of top limb 1) and an 8192-limb addition."""
    from paper_2607_28897_gb300 import inputs

    ops_all, _, _ = inputs.ragged_ops(seed_ops, 200000)
    ops = ops_all[:count].copy()
    nin = int(ops["b"][-1] + ops["nb"][-1])
    nout = int(max(o["o2"] + o["nb"] if o["op"] == 4 else o["o1"] + (
        o["na"] + o["nb"] if o["op"] == 3 else o["na"]) for o in ops))
    pool = inputs.ragged_pool(seed_pool, ops, nin)
    extra = np.zeros(4, dtype=ops.dtype)
    shapes = [(3, 8192, 8192), (4, 16384, 8192), (4, 16384, 8192), (1, 8192, 8192)]
    parts = [pool]
    pos, opos = nin, nout
    for k, (op, na, nb) in enumerate(shapes):
        a = inputs.limbs(900 + k, 1, na, top_nonzero=True)[0]
        b = inputs.limbs(950 + k, 1, nb, top_nonzero=True)[0]
        if k == 2:
            b[-1] = np.uint64(1)  # divisor just above B^(nb-1)
        nq = na - nb + 1
        extra[k] = (op, na, nb, 0, pos, pos + na, opos, opos + nq if op == 4 else 0)
        parts += [a, b]
        pos += na + nb
        opos += (na + nb) if op == 3 else (nq + nb if op == 4 else na)
    return np.concatenate([ops, extra]), np.concatenate(parts), opos


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_batch_config4_slice_against_oracle(orc, mode):
    """A slice of the batched workload at its own sizes (up to 8192-limb
    products and 16384 / 8192-limb divisions on the tensor cores), in the
    persistent, the per-class and the steps form (division classes padded to
    one shape and divided step-batched), against the oracle op by op."""
    import torch

    import paper_2607_28897_gb300 as bi

    ops, pool, nout = config4_slice(1500)
    assert ops["na"].max() == 16384 and (ops["op"] == 4).sum() > 100
    exp, exp_st = oracle_results(orc, ops, pool)
    dpool = to_dev(pool).view(-1)
    dout = torch.zeros(nout, dtype=torch.int64, device="cuda")
    st = torch.zeros(len(ops), dtype=torch.int32, device="cuda")
    B = bi.Batch(ops)
    B.launch(dpool, dout, st, mode=mode)
    torch.cuda.synchronize()
    bi.check_timeout()
    check(ops, to_host(dout), st.cpu().numpy(), exp, exp_st)


def test_division_classes_with_irregular_members(orc):
    """One class of divisions of nearby shapes (the steps form pads them to
    one shape) whose members include a zero divisor, divisors with zero top
    limbs (a quotient that may not fit), dividends with leading zero limbs
    and a dividend below the divisor: the steps form equals the persistent
    form and the oracle, statuses included."""
    import torch

    import paper_2607_28897_gb300 as bi
    from paper_2607_28897_gb300 import inputs

    rng = np.random.default_rng(81)
    count = 40
    nv = rng.integers(300, 330, count)
    nu = nv + rng.integers(180, 220, count)
    ops = np.zeros(count, dtype=bi.op_dtype())
    ops["op"], ops["na"], ops["nb"] = bi.OP_DIVMOD, nu, nv
    pos, opos, parts = 0, 0, []
    for i in range(count):
        a = inputs.limbs(500 + i, 1, int(nu[i]), top_nonzero=True)[0]
        b = inputs.limbs(600 + i, 1, int(nv[i]), top_nonzero=True)[0]
        if i == 0:
            b[:] = 0                        # division by zero
        elif i in (1, 2):
            b[-3:] = 0                      # divisor with zero top limbs
        elif i in (3, 4):
            a[-50:] = 0                     # dividend with leading zero limbs
        elif i == 5:
            a[:] = 0
            a[:10] = 7                      # dividend below the divisor
        nq = int(nu[i] - nv[i] + 1)
        ops[i]["a"], ops[i]["b"], ops[i]["o1"], ops[i]["o2"] = pos, pos + nu[i], opos, opos + nq
        parts += [a, b]
        pos += int(nu[i] + nv[i])
        opos += nq + int(nv[i])
    pool = np.concatenate(parts)
    exp, exp_st = oracle_results(orc, ops, pool)
    dpool = to_dev(pool).view(-1)
    got = []
    for mode in (0, 2):
        dout = torch.zeros(opos, dtype=torch.int64, device="cuda")
        st = torch.zeros(count, dtype=torch.int32, device="cuda")
        bi.Batch(ops).launch(dpool, dout, st, mode=mode)
        torch.cuda.synchronize()
        check(ops, to_host(dout), st.cpu().numpy(), exp, exp_st)
        got.append(to_host(dout))
    assert np.array_equal(got[0], got[1])
