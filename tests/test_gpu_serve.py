"""Continuous batching: requests that arrive while others run are admitted
into new batches on other streams; every result equals the oracle's result
for that request computed alone."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_serving_results_equal_alone(orc):
    from paper_2607_28897_gb300 import serve

    w = serve.make_workload(31, 400, rate=20000.0, min_limbs=8, max_limbs=900)
    res = serve.run_continuous(w, streams=3, max_batch=64, keep_results=True)
    assert res["requests"] == 400 and not res["status"].any()
    pool = w.pool.numpy().view(np.uint64)
    for i, o in enumerate(w.ops):
        a = pool[o["a"]:o["a"] + o["na"]]
        b = pool[o["b"]:o["b"] + o["nb"]]
        if o["op"] == 3:
            exp = orc.mul(a, b)
        else:
            q, r, s = orc.divmod_(a, b)
            assert s == 0
            exp = np.concatenate([q, r])
        assert np.array_equal(res["results"][i], exp), i
    assert res["p99_ms"] >= res["p50_ms"] > 0


def test_serving_budget_admission():
    """A budget smaller than one batch still serves (one batch at a time)."""
    from paper_2607_28897_gb300 import serve

    w = serve.make_workload(32, 100, rate=50000.0, min_limbs=8, max_limbs=300)
    res = serve.run_continuous(w, budget_bytes=1, streams=2, max_batch=16)
    assert res["requests"] == 100 and not res["status"].any()


def test_server_submit_poll_wait(orc):
    """The request-level API: mixed requests submitted one by one, results
    (device tensors) equal the oracle's; a tight HBM budget forces several
    batches; poll reports completion."""
    import numpy as np
    import torch

    import paper_2607_28897_gb300 as bi
    from paper_2607_28897_gb300 import inputs
    from paper_2607_28897_gb300.serve import Server

    rng = np.random.default_rng(5)
    srv = Server(budget_bytes=4 << 20, streams=2, max_batch=16)
    reqs = []
    for i in range(40):
        op = (bi.OP_ADD, bi.OP_SUB, bi.OP_MUL, bi.OP_DIVMOD)[i % 4]
        nb = int(rng.integers(1, 600))
        na = nb if op in (bi.OP_ADD, bi.OP_SUB) else int(rng.integers(nb, 2 * nb + 1))
        a = inputs.limbs(1000 + i, 1, na)[0]
        b = inputs.limbs(2000 + i, 1, nb, top_nonzero=True)[0]
        ta = torch.from_numpy(a.view(np.int64)).cuda() if i % 2 else torch.from_numpy(a.view(np.int64))
        tb = torch.from_numpy(b.view(np.int64)).cuda()
        reqs.append((srv.submit(op, ta, tb), op, a, b))
    for t, op, a, b in reqs:
        res = [x.cpu().numpy().view(np.uint64) for x in srv.wait(t)]
        if op == bi.OP_ADD:
            assert np.array_equal(res[0], orc.add(a, b)[0])
        elif op == bi.OP_SUB:
            assert np.array_equal(res[0], orc.sub(a, b)[0])
        elif op == bi.OP_MUL:
            assert np.array_equal(res[0], orc.mul(a, b))
        else:
            q, r, _ = orc.divmod_(a, b)
            assert np.array_equal(res[0], q) and np.array_equal(res[1], r)
    t = srv.submit(bi.OP_MUL, torch.ones(8, dtype=torch.int64), torch.ones(8, dtype=torch.int64))
    srv.wait(t)
    assert not srv.poll(t)  # consumed
    with pytest.raises(bi.BigIntError):
        srv.submit(bi.OP_MUL, torch.ones(1 << 20, dtype=torch.int64),
                   torch.ones(1 << 20, dtype=torch.int64))


def test_admission_counts_batch_workspace(orc):
    """The HBM budget covers operands, results AND the batch workspace (the
    division scratch that holds the Newton iterates): with a budget that all
    requests' operands and results fit but not their divisions' scratch, the
    requests are split into several batches and the bytes in flight never
    exceed the budget."""
    import numpy as np

    from paper_2607_28897_gb300 import Batch, serve

    w = serve.make_workload(33, 24, rate=1e9, mix_mul=0.0, min_limbs=1024, max_limbs=2048)
    io = int(8 * (w.ops["na"] + w.ops["nb"] + w.out_limbs).sum())
    sub, _, _, _ = serve._sub_batch(w, 0, 1)
    ws1 = Batch(sub, allocate=False).workspace_bytes
    assert ws1 > 0
    budget = io + 3 * ws1
    res = serve.run_continuous(w, budget_bytes=budget, streams=3, max_batch=64,
                               keep_results=True)
    assert res["batches"] >= 2
    assert res["peak_bytes_in_flight"] <= budget
    assert not res["status"].any()
    pool = w.pool.numpy().view(np.uint64)
    for i, o in enumerate(w.ops):
        q, r, s = orc.divmod_(pool[o["a"]:o["a"] + o["na"]], pool[o["b"]:o["b"] + o["nb"]])
        assert s == 0
        assert np.array_equal(res["results"][i], np.concatenate([q, r])), i


def test_serving_full_sizes_equal_alone(orc):
    """Continuous batching at the serving workload's own sizes (2^15..2^19
    bits, half products half divisions, so products and divisions run on the
    tensor cores inside the batches): every request's result equals the
    oracle's result for that request computed alone."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor

    from paper_2607_28897_gb300 import serve

    w = serve.make_workload(34, 160, rate=20000.0)
    assert w.ops["nb"].max() > 4096 and w.ops["na"].max() > 8192
    res = serve.run_continuous(w, streams=3, max_batch=32, keep_results=True)
    assert res["requests"] == 160 and not res["status"].any()
    assert res["batches"] >= 2
    pool = w.pool.numpy().view(np.uint64)

    def expected(i):
        o = w.ops[i]
        a = pool[o["a"]:o["a"] + o["na"]]
        b = pool[o["b"]:o["b"] + o["nb"]]
        if o["op"] == 3:
            return orc.mul(a, b)
        q, r, s = orc.divmod_(a, b)
        assert s == 0
        return np.concatenate([q, r])

    with ThreadPoolExecutor(16) as ex:  # the oracle's C calls release the GIL
        exp = list(ex.map(expected, range(len(w.ops))))
    for i in range(len(w.ops)):
        assert np.array_equal(res["results"][i], exp[i]), i
