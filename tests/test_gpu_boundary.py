"""Every entry of the boundary through the C ABI (ctypes, device pointers):
the uniform add / sub / mul / divmod (+ its workspace size), the ragged
per-operation forms over views (lengths and offsets per instance, zero-
extended add and sub), the one-call mixed batch (bigint_batch_run), the
autotuner and its table, and strerror -- results against the oracle."""
import ctypes

import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


def stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_uniform_entries(orc):
    import torch

    import paper_2607_28897_gb300 as bi
    from paper_2607_28897_gb300 import inputs

    L = bi.load()
    a, b = inputs.config_small(seed=71, n=300, count=20)
    da, db = to_dev(a), to_dev(b)
    out = torch.empty_like(da)
    c = torch.empty(a.shape[0], dtype=torch.uint8, device="cuda")
    assert L.bigint_add(da.data_ptr(), db.data_ptr(), out.data_ptr(), c.data_ptr(), a.shape[0],
                        300, stream()) == 0
    r, rc = orc.batch_add(a, b)
    assert np.array_equal(to_host(out), r) and np.array_equal(c.cpu().numpy(), rc)
    sa, sb = inputs.order_pairs(a, b)
    assert L.bigint_sub(to_dev(sa).data_ptr(), to_dev(sb).data_ptr(), out.data_ptr(),
                        c.data_ptr(), a.shape[0], 300, stream()) == 0
    torch.cuda.synchronize()
    assert np.array_equal(to_host(out), orc.batch_sub(sa, sb)[0])
    p = torch.empty((a.shape[0], 600), dtype=torch.int64, device="cuda")
    assert L.bigint_mul(da.data_ptr(), db.data_ptr(), p.data_ptr(), a.shape[0], 300, 300,
                        stream()) == 0
    torch.cuda.synchronize()
    assert np.array_equal(to_host(p), orc.batch_mul(a, b))
    u, v = inputs.config_div(300, 12, seed=72)
    du, dv = to_dev(u), to_dev(v)
    ws_bytes = L.bigint_divmod_workspace(12, 600, 300)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    q = torch.empty((12, 301), dtype=torch.int64, device="cuda")
    rr = torch.empty((12, 300), dtype=torch.int64, device="cuda")
    st = torch.empty(12, dtype=torch.int32, device="cuda")
    assert L.bigint_divmod(du.data_ptr(), dv.data_ptr(), q.data_ptr(), rr.data_ptr(),
                           st.data_ptr(), 12, 600, 300, ws.data_ptr(), ws_bytes, stream()) == 0
    torch.cuda.synchronize()
    oq, orr, _ = orc.batch_divmod(u, v)
    assert np.array_equal(to_host(q), oq) and np.array_equal(to_host(rr), orr)
    assert not st.cpu().numpy().any()
    assert L.bigint_strerror(bi.EINVAL) == b"invalid argument"


def ragged_layout(rng, lengths, gap=3):
    """Offsets of instances laid out in a shuffled order with gaps."""
    order = rng.permutation(len(lengths))
    off = np.zeros(len(lengths), dtype=np.int64)
    pos = 0
    for i in order:
        off[i] = pos
        pos += int(lengths[i]) + gap
    return off, pos


def fill(buf, off, lengths, seed, top_nonzero=True):
    from paper_2607_28897_gb300 import inputs

    for i, (o, n) in enumerate(zip(off, lengths)):
        buf[o:o + n] = inputs.limbs(seed * 1000 + i, 1, int(n), top_nonzero)[0]


def test_ragged_views(orc):
    import torch

    import paper_2607_28897_gb300 as bi

    rng = np.random.default_rng(73)
    count = 40
    na = rng.integers(1, 2500, count).astype(np.int32)
    nb = np.where(rng.random(count) < 0.5, na, rng.integers(1, 2500, count)).astype(np.int32)
    offa, sa = ragged_layout(rng, na)
    offb, sb = ragged_layout(rng, nb)
    ha = np.zeros(sa, dtype=np.uint64)
    hb = np.zeros(sb, dtype=np.uint64)
    fill(ha, offa, na, 1)
    fill(hb, offb, nb, 2)
    da, db = to_dev(ha), to_dev(hb)
    A, Bv = bi.view(da, offa, na), bi.view(db, offb, nb)

    # add / sub with zero extension: results of max(na, nb) limbs
    n_s = np.maximum(na, nb).astype(np.int32)
    offs, ss = ragged_layout(rng, n_s)
    for sub in (False, True):
        out = torch.zeros(ss, dtype=torch.int64, device="cuda")
        carry = torch.zeros(count, dtype=torch.int32, device="cuda")
        bi.batch_add(A, Bv, bi.view(out, offs, n_s), carry, zext=True, sub=sub)
        torch.cuda.synchronize()
        h = to_host(out)
        for i in range(count):
            x = np.zeros(n_s[i], dtype=np.uint64)
            y = np.zeros(n_s[i], dtype=np.uint64)
            x[:na[i]] = ha[offa[i]:offa[i] + na[i]]
            y[:nb[i]] = hb[offb[i]:offb[i] + nb[i]]
            r, c = (orc.sub if sub else orc.add)(x, y)
            assert np.array_equal(h[offs[i]:offs[i] + n_s[i]], r), (sub, i)
            assert int(carry[i]) == c, (sub, i)
    # without BIGINT_ZEXT, unequal lengths are refused
    with pytest.raises(bi.BigIntError):
        bi.batch_add(A, Bv, bi.view(torch.zeros(ss, dtype=torch.int64, device="cuda"), offs, n_s))

    # products of na + nb limbs
    n_p = (na + nb).astype(np.int32)
    offp, sp = ragged_layout(rng, n_p)
    out = torch.zeros(sp, dtype=torch.int64, device="cuda")
    bi.batch_mul(A, Bv, bi.view(out, offp, n_p))
    torch.cuda.synchronize()
    h = to_host(out)
    for i in range(count):
        exp = orc.mul(ha[offa[i]:offa[i] + na[i]], hb[offb[i]:offb[i] + nb[i]])
        assert np.array_equal(h[offp[i]:offp[i] + n_p[i]], exp), i

    # divisions: q of max(nu - nv + 1, 1) limbs, r of nv limbs
    n_q = np.maximum(na - nb + 1, 1).astype(np.int32)
    offq, sq = ragged_layout(rng, n_q)
    offr, sr = ragged_layout(rng, nb)
    q = torch.zeros(sq, dtype=torch.int64, device="cuda")
    r = torch.zeros(sr, dtype=torch.int64, device="cuda")
    st = torch.zeros(count, dtype=torch.int32, device="cuda")
    bi.batch_divmod(A, Bv, bi.view(q, offq, n_q), bi.view(r, offr, nb), st)
    torch.cuda.synchronize()
    hq, hr, hs = to_host(q), to_host(r), st.cpu().numpy()
    for i in range(count):
        oq, orr, s = orc.divmod_(ha[offa[i]:offa[i] + na[i]], hb[offb[i]:offb[i] + nb[i]])
        assert np.array_equal(hq[offq[i]:offq[i] + n_q[i]], oq), i
        assert np.array_equal(hr[offr[i]:offr[i] + nb[i]], orr), i
        assert hs[i] == {0: 0, 2: bi.EDIVZERO, 1: bi.ERANGE}[s], i


def test_batch_run_and_tune(orc):
    import torch

    import paper_2607_28897_gb300 as bi
    from paper_2607_28897_gb300 import inputs

    L = bi.load()
    ops, nin, nout = inputs.ragged_ops(74, 120, min_limbs=4, max_limbs=3000)
    pool = inputs.ragged_pool(75, ops, nin)
    dpool = to_dev(pool)
    for mode in (bi.BATCH_PERSISTENT, bi.BATCH_PER_CLASS):
        out = torch.zeros(nout, dtype=torch.int64, device="cuda")
        st = torch.zeros(len(ops), dtype=torch.int32, device="cuda")
        ws_bytes = L.bigint_batch_run_workspace(ops.ctypes.data, len(ops))
        ws = torch.empty(max(ws_bytes, 256), dtype=torch.uint8, device="cuda")
        assert L.bigint_batch_run(ops.ctypes.data, len(ops), dpool.data_ptr(), out.data_ptr(),
                                  st.data_ptr(), ws.data_ptr(), ws.numel(), mode, stream()) == 0
        torch.cuda.synchronize()
        h = to_host(out)
        for i, o in enumerate(ops):
            a = pool[o["a"]:o["a"] + o["na"]]
            b = pool[o["b"]:o["b"] + o["nb"]]
            if o["op"] == bi.OP_MUL:
                assert np.array_equal(h[o["o1"]:o["o1"] + o["na"] + o["nb"]], orc.mul(a, b)), i
            elif o["op"] == bi.OP_DIVMOD:
                oq, orr, _ = orc.divmod_(a, b)
                assert np.array_equal(h[o["o1"]:o["o1"] + oq.size], oq), i
                assert np.array_equal(h[o["o2"]:o["o2"] + orr.size], orr), i
            else:
                r, c = (orc.add if o["op"] == bi.OP_ADD else orc.sub)(a, b)
                assert np.array_equal(h[o["o1"]:o["o1"] + r.size], r), i
                assert int(st[i]) == c, i
    # the autotuner through the C ABI, and the table round trip
    a = to_dev(inputs.limbs(76, 64, 600))
    b = to_dev(inputs.limbs(77, 64, 600))
    p = torch.empty((64, 1200), dtype=torch.int64, device="cuda")
    best = ctypes.c_int()
    assert L.bigint_tune(a.data_ptr(), b.data_ptr(), p.data_ptr(), 64, 600, 600, stream(),
                         ctypes.byref(best)) == 0
    assert best.value in (8, 9, 10, 12, 13, 14, 15, 16, 17)
    assert L.bigint_load_tuning(b"/nonexistent/tuning.json") == bi.EINVAL
    import json
    import tempfile

    with tempfile.TemporaryDirectory() as d:  # leave the built-in choice behind
        path = f"{d}/t.json".encode()
        assert L.bigint_save_tuning(path) == 0
        t = json.load(open(path))
        t["mul_variant_by_class"] = [0] * 32
        json.dump(t, open(path, "w"))
        assert L.bigint_load_tuning(path) == 0
