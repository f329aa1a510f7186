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
