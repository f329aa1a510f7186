"""Host-side argument checks of the C ABI (they run before any CUDA call,
so they are exercised here without a GPU)."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def L():
    import paper_2607_28897_gb300 as bi

    return bi.load()


def test_addsub_mul_argument_checks(L):
    import paper_2607_28897_gb300 as bi

    p = ctypes.c_void_p(16)
    assert L.bigint_add(p, p, p, None, -1, 4, None) == bi.EINVAL
    assert L.bigint_sub(p, p, p, None, 1, bi.MAX_LIMBS + 1, None) == bi.EINVAL
    assert L.bigint_mul(p, p, p, 1, bi.MUL_MAX_LIMBS + 1, 1, None) == bi.EINVAL
    assert L.bigint_mul_lo(p, p, p, 1, 4, 4, 9, None) == bi.EINVAL  # m > na + nb
    assert L.bigint_mul_lo(p, p, p, 1, 4, 4, 0, None) == bi.EINVAL
    assert L.bigint_mul(None, None, None, 0, 4, 4, None) == bi.OK  # empty batch


def test_divmod_workspace_checks(L):
    import paper_2607_28897_gb300 as bi

    p = ctypes.c_void_p(256)
    need = L.bigint_divmod_workspace(8, 64, 32)
    assert need > 0 and need % 256 == 0
    assert L.bigint_divmod_workspace(16, 64, 32) == 2 * need
    # too small a workspace, or a misaligned one, is refused before any launch
    assert L.bigint_divmod(p, p, p, p, None, 8, 64, 32, p, need - 1, None) == bi.ENOMEM
    assert L.bigint_divmod(p, p, p, p, None, 8, 64, 32, ctypes.c_void_p(264), need,
                           None) == bi.EINVAL
    assert L.bigint_shinv(p, p, None, 1, 8, 4, 6, p, 1 << 20, None) == bi.EINVAL  # h < nv


def test_batch_descriptor_validation(L):
    import paper_2607_28897_gb300 as bi

    dt = bi.op_dtype()
    bad = [
        dict(op=9, na=4, nb=4),                          # unknown op
        dict(op=bi.OP_ADD, na=4, nb=5),                  # add with unequal widths
        dict(op=bi.OP_MUL, na=bi.MUL_MAX_LIMBS + 1, nb=4),
        dict(op=bi.OP_DIVMOD, na=0, nb=4),
    ]
    for d in bad:
        ops = np.zeros(1, dtype=dt)
        for k, v in d.items():
            ops[k] = v
        h = ctypes.c_void_p()
        assert L.bigint_batch_create(ops.ctypes.data, 1, ctypes.byref(h)) == bi.EINVAL
    ops = np.zeros(1, dtype=dt)
    ops["op"], ops["na"], ops["nb"], ops["a"] = bi.OP_MUL, 4, 4, -1
    h = ctypes.c_void_p()
    assert L.bigint_batch_create(ops.ctypes.data, 1, ctypes.byref(h)) == bi.EINVAL


def test_tuning_table_rejects_other_gpu(L, tmp_path):
    import paper_2607_28897_gb300 as bi

    f = tmp_path / "t.json"
    f.write_text('{"gpu": "some other GPU", "batch_threads": 256, '
                 '"mul_variant_by_class": [' + ", ".join(["0"] * 32) + "]}")
    assert L.bigint_tuning_load(str(f).encode()) == bi.EINVAL
    assert L.bigint_tuning_load(b"/nonexistent/tuning.json") == bi.EINVAL
    assert L.bigint_set_variant(0, 99) == bi.EINVAL
    assert L.bigint_set_variant(7, 0) == bi.EINVAL
