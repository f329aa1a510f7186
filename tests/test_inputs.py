"""The seeded generators: numpy and torch versions agree bit for bit, and
the workload recipes have the stated structure."""
import numpy as np

from paper_2607_28897_gb300 import inputs


def test_torch_generator_matches_numpy():
    import torch

    for seed, count, start in ((1, 1000, 0), (7, 333, 12345), (2 ** 20 + 3, 5000, 99)):
        a = inputs.uniform(seed, count, start)
        b = inputs.uniform_torch(seed, count, device="cpu", start=start).numpy().view(np.uint64)
        assert np.array_equal(a, b)
    x = inputs.limbs(5, 40, 7, top_nonzero=True)
    y = inputs.limbs_torch(5, 40, 7, True, device="cpu").numpy().view(np.uint64)
    assert np.array_equal(x, y)


def test_generator_is_chunk_independent():
    a = inputs.uniform(3, 5000)
    b = np.concatenate([inputs.uniform(3, 1234), inputs.uniform(3, 5000 - 1234, start=1234)])
    assert np.array_equal(a, b)


def test_recipes():
    a, b = inputs.config_sweep(512, batch=64)
    assert a.shape == (64, 512) and (a[:, -1] != 0).all() and (b[:, -1] != 0).all()
    u, v = inputs.config_div(16, 10)
    assert u.shape == (10, 32) and v.shape == (10, 16)
    assert (v[0::2, -1] >> np.uint64(63) == 1).all()
    assert ((v[1::2, -1] >= 1) & (v[1::2, -1] < (1 << 32))).all()
    s = inputs.ragged_sizes(1, 10000)
    assert s.min() >= 512 and s.max() <= 8192
    sa, sb = inputs.stress_pairs(8)
    assert sa.shape == (8, 8)
