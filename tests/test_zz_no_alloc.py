"""bigint_divmod_noalloc: division for callers that cannot allocate device
memory (its scratch is the library's own fixed __device__ array).

Collected last on purpose.  It calls the entry point through the C ABI and
checks it against bigint_divmod (the workspace entry point) on two calls in
a row with different inputs, including a batch larger than one scratch-sized
launch, so that stale scratch contents or a wrong chunk offset would show,
and a shape large enough (2048 / 1024 limbs) for the division kernel that
runs its products on the tensor cores, which is also compared with the
oracle.
"""
import ctypes

import numpy as np
import pytest

from helpers import to_dev, to_host

pytestmark = pytest.mark.gpu


def call_noalloc(L, u, v):
    import torch

    count, nu = u.shape
    nv = v.shape[1]
    nq = max(nu - nv + 1, 1)
    q = torch.empty((count, nq), dtype=torch.int64, device=u.device)
    r = torch.empty((count, nv), dtype=torch.int64, device=u.device)
    st = torch.empty(count, dtype=torch.int32, device=u.device)
    rc = L.bigint_divmod_noalloc(u.data_ptr(), v.data_ptr(), q.data_ptr(), r.data_ptr(),
                                 st.data_ptr(), count, nu, nv,
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, rc
    return q, r, st


def test_noalloc_matches_workspace_entry_point(orc):
    import torch

    import paper_2607_28897_gb300 as bi
    from paper_2607_28897_gb300 import inputs

    L = bi.load()
    assert L.bigint_divmod_noalloc_scratch_bytes() == 32 << 20
    per = bi.divmod_workspace_bytes(1, 1024, 512)
    cases = [inputs.config_div(64, 50, seed=21),
             # more instances than one 32 MiB scratch launch holds
             inputs.config_div(512, (32 << 20) // per * 2 + 37, seed=22),
             # products on the tensor cores inside the division kernel
             inputs.config_div(1024, 6, seed=23)]
    for k, (u, v) in enumerate(cases):  # calls in a row, each after the last
        du, dv = to_dev(u), to_dev(v)
        q1, r1, s1 = call_noalloc(L, du, dv)
        q2, r2, s2 = bi.divmod(du, dv)
        torch.cuda.synchronize()
        assert np.array_equal(to_host(q1), to_host(q2))
        assert np.array_equal(to_host(r1), to_host(r2))
        assert np.array_equal(s1.cpu().numpy(), s2.cpu().numpy())
        assert not s1.cpu().numpy().any()
        if k == 2:
            oq, orr, ost = orc.batch_divmod(u, v)
            assert np.array_equal(to_host(q1), oq) and np.array_equal(to_host(r1), orr)

