"""The CUDA path on the stored carry-stress fixture (tests/golden/): every
add, sub, mul and divmod result equals the stored one."""
import os

import numpy as np
import pytest

from helpers import to_dev, to_host
from test_golden import HERE, parse

pytestmark = pytest.mark.gpu


def test_cuda_path_on_golden_fixture():
    import paper_2607_28897_gb300 as bi

    rows = [parse(l) for l in open(os.path.join(HERE, "carry_stress_n4.txt"))
            if not l.startswith("#")]
    for op, i, L, tail in rows:
        if op in ("add", "sub"):
            a, b, exp = to_dev(L[0][None]), to_dev(L[1][None]), L[2]
            r, c = (bi.add if op == "add" else bi.sub)(a, b)
            assert np.array_equal(to_host(r)[0], exp) and int(c[0]) == tail, (op, i)
        elif op == "mul":
            p = bi.mul(to_dev(L[0][None]), to_dev(L[1][None]))
            assert np.array_equal(to_host(p)[0], L[2]), (op, i)
        else:
            q, r, st = bi.divmod(to_dev(L[0][None]), to_dev(L[1][None]))
            assert np.array_equal(to_host(q)[0], L[2]), (op, i)
            assert np.array_equal(to_host(r)[0], L[3]), (op, i)
            assert int(st[0]) == 0, (op, i)
