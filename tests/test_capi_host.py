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


def test_mul_split_checks(L):
    """Workspace: up to 16 products, the column sums of each 256-column tile
    (256 x 128 int32) of the split-K form; larger batches, 16 bytes per
    4096-limb tile of each tile-split product; none for products that do not
    split; short or misaligned workspaces are refused."""
    import paper_2607_28897_gb300 as bi

    tile_sums = 256 * 128 * 4
    assert L.bigint_mul_split_workspace(2, 4096, 4096) == 2 * 2 * tile_sums
    assert L.bigint_mul_split_workspace(3, 8192, 8192) == 3 * 4 * tile_sums
    assert L.bigint_mul_split_workspace(1, 2048, 2049) == 2 * tile_sums
    assert L.bigint_mul_split_workspace(4, 512, 512) == 4 * tile_sums
    assert L.bigint_mul_split_workspace(17, 4096, 4096) == 16 * 17 * 2  # tile split
    assert L.bigint_mul_split_workspace(17, 512, 512) == 0
    assert L.bigint_mul_split_workspace(4, 100, 512) == 0  # shorter operand too small
    assert L.bigint_mul_split_workspace(1, 12000, 12000) == 0  # x beyond shared memory
    assert L.bigint_mul_split_workspace(-1, 4096, 4096) == 0
    p = ctypes.c_void_p(256)
    assert L.bigint_mul_split(p, p, p, -1, 4, 4, p, 0, None) == bi.EINVAL
    assert L.bigint_mul_split(p, p, p, 1, bi.MUL_MAX_LIMBS + 1, 4, p, 0, None) == bi.EINVAL
    assert L.bigint_mul_split(None, None, None, 0, 4, 4, None, 0, None) == bi.OK
    assert L.bigint_mul_split(p, p, p, 2, 4096, 4096, p, 63, None) == bi.ENOMEM
    assert L.bigint_mul_split(p, p, p, 2, 4096, 4096, ctypes.c_void_p(260), 1 << 20,
                              None) == bi.EINVAL


def test_divmod_inv_checks(L):
    """Division by a given inverse: h must cover both operands, w at most
    h + 1 limbs, strides nv / nw or 0, and the divmod workspace."""
    import paper_2607_28897_gb300 as bi

    p = ctypes.c_void_p(256)
    need = L.bigint_divmod_workspace(8, 64, 32)
    args = dict(u=p, v=p, w=p, q=p, r=p, st=None, count=8, nu=64, nv=32, nw=34, h=64, vs=32,
                wst=34, ws=p, nb=need)

    def call(**kw):
        a = dict(args, **kw)
        return L.bigint_divmod_inv(a["u"], a["v"], a["w"], a["q"], a["r"], a["st"], a["count"],
                                   a["nu"], a["nv"], a["nw"], a["h"], a["vs"], a["wst"], a["ws"],
                                   a["nb"], None)

    assert call(h=63) == bi.EINVAL            # h < nu
    assert call(nw=66) == bi.EINVAL           # nw > h + 1
    assert call(vs=5) == bi.EINVAL            # stride neither nv nor 0
    assert call(wst=7) == bi.EINVAL
    assert call(count=-1) == bi.EINVAL
    assert call(nb=need - 1) == bi.ENOMEM
    assert call(ws=ctypes.c_void_p(264)) == bi.EINVAL
    assert call(count=0, u=None, v=None, w=None, q=None, r=None) == bi.OK


def test_divmod_workspace_checks(L):
    import paper_2607_28897_gb300 as bi

    p = ctypes.c_void_p(256)
    need = L.bigint_divmod_workspace(8, 64, 32)
    assert need > 0 and need % 256 == 0
    # per-instance regions plus a list of instances and two counters
    need16 = L.bigint_divmod_workspace(16, 64, 32)
    assert need16 % 256 == 0 and 2 * need - 512 <= need16 <= 2 * need
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
    assert L.bigint_load_tuning(str(f).encode()) == bi.EINVAL
    assert L.bigint_load_tuning(b"/nonexistent/tuning.json") == bi.EINVAL
    assert L.bigint_set_variant(0, 99) == bi.EINVAL
    assert L.bigint_set_variant(7, 0) == bi.EINVAL
    for v in (1, 3, 7, 18):  # forms the library does not carry
        assert L.bigint_set_variant(0, v) == bi.EINVAL
    for v in (8, 9, 10, 11, 12, 13, 14, 15, 16, 17, 0):
        assert L.bigint_set_variant(0, v) == bi.OK
    assert L.bigint_set_variant(3, 0) == bi.EINVAL


# ---- host-buffer entry points: argument checks that need no GPU -------------
def test_host_workspace_rejects_bad_shapes():
    import paper_2607_28897_gb300 as bi

    lib = bi.load()
    assert lib.bigint_host_workspace(bi.OP_MUL, 0, 8, 8) == 0
    assert lib.bigint_host_workspace(bi.OP_ADD, 4, 8, 9) == 0  # add needs na == nb
    assert lib.bigint_host_workspace(99, 4, 8, 8) == 0
    assert lib.bigint_host_workspace(bi.OP_MUL, 4, 0, 8) == 0
    assert lib.bigint_host_workspace(bi.OP_MUL, 4, bi.MUL_MAX_LIMBS + 1, 8) == 0
    # two staging slots of 4 instances: operands, product, 256-byte aligned
    assert lib.bigint_host_workspace(bi.OP_MUL, 4, 8, 8) == 2 * (256 + 256 + 512)


def test_host_calls_check_arguments():
    import ctypes

    import paper_2607_28897_gb300 as bi

    lib = bi.load()
    buf = (ctypes.c_uint64 * 64)()
    p = ctypes.addressof(buf)
    # count 0: nothing to do
    assert lib.bigint_mul_host(None, None, None, 0, 4, 4, None, 0) == bi.OK
    # null operands, null workspace, misaligned workspace
    assert lib.bigint_mul_host(None, p, p, 2, 4, 4, p, 1 << 20) == bi.EINVAL
    assert lib.bigint_mul_host(p, p, p, 2, 4, 4, None, 1 << 20) == bi.EINVAL
    assert lib.bigint_mul_host(p, p, p, 2, 4, 4, p + 8, 1 << 20) == bi.EINVAL
    # add/sub need equal lengths; divmod needs the remainder buffer
    assert lib.bigint_add_host(p, p, p, None, 2, 0, p, 1 << 20) == bi.EINVAL
    assert lib.bigint_divmod_host(p, p, p, None, None, 2, 4, 2, p, 1 << 20) == bi.EINVAL
    assert lib.bigint_divmod_host(p, p, p, p, None, -1, 4, 2, p, 1 << 20) == bi.EINVAL


def test_views_rejected_on_the_host(L):
    """Malformed views and mismatched lengths are refused before any device
    work (no GPU needed)."""
    import numpy as np

    import paper_2607_28897_gb300 as bi

    class V(ctypes.Structure):
        _fields_ = [("data", ctypes.c_void_p), ("offset", ctypes.c_void_p),
                    ("nlimbs", ctypes.c_void_p), ("count", ctypes.c_int64), ("n", ctypes.c_int32)]

    def v(count, n, data=256, lengths=None):
        x = V()
        x.data, x.count, x.n = data, count, n
        if lengths is not None:
            arr = np.asarray(lengths, dtype=np.int32)
            off = np.arange(len(arr), dtype=np.int64) * 100
            x.offset, x.nlimbs = off.ctypes.data, arr.ctypes.data
            x._keep = (arr, off)
        return x

    a, b = v(4, 8), v(4, 8)
    ws = ctypes.c_void_p(256)
    for out, flags, why in ((v(4, 9), 0, "wrong result length"),
                            (v(3, 8), 0, "count mismatch"),
                            (v(4, 8, data=260), 0, "misaligned data"),
                            (v(4, 8), 2, "unknown flag")):
        assert L.bigint_batch_add(ctypes.byref(a), ctypes.byref(b), ctypes.byref(out), None, flags,
                                  ws, 1 << 20, None) == bi.EINVAL, why
    ragged = v(2, 0, lengths=[5, 7])
    same = v(2, 0, lengths=[5, 5])
    out7 = v(2, 0, lengths=[5, 7])
    assert L.bigint_batch_sub(ctypes.byref(ragged), ctypes.byref(same), ctypes.byref(out7), None,
                              0, ws, 1 << 20, None) == bi.EINVAL  # unequal without ZEXT
    assert L.bigint_batch_mul(ctypes.byref(a), ctypes.byref(b), ctypes.byref(v(4, 15)), ws,
                              1 << 20, None) == bi.EINVAL  # product needs 16 limbs
    q, r = v(4, 1), v(4, 7)
    assert L.bigint_batch_divmod(ctypes.byref(a), ctypes.byref(b), ctypes.byref(q),
                                 ctypes.byref(r), None, ws, 1 << 20, None) == bi.EINVAL
    assert L.bigint_batch_run(None, 3, None, None, None, ws, 0, 0, None) == bi.EINVAL
    assert L.bigint_batch_run(None, 0, None, None, None, None, 0, 9, None) == bi.EINVAL


def test_mul_kara_checks(L):
    """Argument checks of the Karatsuba product that need no GPU."""
    import paper_2607_28897_gb300 as bi

    P = ctypes.c_void_p(8)
    assert L.bigint_mul_kara(P, P, P, -1, 8, 1, None, 0, None) == bi.EINVAL
    assert L.bigint_mul_kara(P, P, P, 4, 0, 1, None, 0, None) == bi.EINVAL
    assert L.bigint_mul_kara(P, P, P, 4, 20000, 1, None, 0, None) == bi.EINVAL
    assert L.bigint_mul_kara(None, P, P, 4, 8, 1, None, 0, None) == bi.EINVAL
    assert L.bigint_mul_kara(P, P, P, 0, 8, 1, None, 0, None) == bi.OK
