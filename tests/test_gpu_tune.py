"""The multiply autotuner (bigint_tune): it times the tensor-core tiles and
the integer forms on the caller's batch, records the fastest per size class
(saved and loaded as a JSON table), and whatever it picks gives the oracle's
product bit for bit."""
import json

import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


def size_class(n):
    c = 0
    while (2 << c) <= n:
        c += 1
    return c


def test_tuner_choice_is_exact_and_saved(orc, tmp_path):
    import paper_2607_28897_gb300 as bi
    from paper_2607_28897_gb300 import inputs

    path = tmp_path / "tuning.json"
    picks = {}
    try:
        for n, count in ((512, 512), (2048, 64), (300, 256)):
            a = inputs.limbs(60 + n, count, n)
            b = inputs.limbs(61 + n, count, n)
            da, db = to_dev(a), to_dev(b)
            best = bi.tune(da, db)
            assert best in (8, 9, 10, 12, 13, 14, 15, 16, 17)
            assert bi.mul_variant_for(n, n) == best  # the size class now uses it
            picks[n] = best
            p = to_host(bi.mul(da, db))
            assert np.array_equal(p, orc.batch_mul(a, b)), (n, best)
            # every tensor-core tile the tuner weighed gives the same bits
            for v in (13, 14, 15, 16, 17):
                bi.set_variant(0, v)
                try:
                    assert np.array_equal(to_host(bi.mul(da, db)), p), (n, v)
                finally:
                    bi.set_variant(0, 0)
        bi.save_tuning(str(path))
        table = json.loads(path.read_text())
        for n, best in picks.items():
            assert table["mul_variant_by_class"][size_class(n)] == best
        assert any(v >= 12 for v in table["mul_variant_by_class"])  # tensor-core entries
        # a saved table loads back; a table of zeros restores the built-in choice
        bi.load_tuning(str(path))
        assert bi.mul_variant_for(512, 512) == picks[512]
    finally:  # leave the built-in choice for the tests that follow
        bi.save_tuning(str(path))
        table = json.loads(path.read_text())
        table["mul_variant_by_class"] = [0] * 32
        path.write_text(json.dumps(table))
        bi.load_tuning(str(path))
    assert bi.mul_variant_for(512, 512) == 12
