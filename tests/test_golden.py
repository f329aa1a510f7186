"""The stored fixtures of tests/golden/, pinned to what fixes them:

* scan_operator.txt, the (generate, propagate) operator of Sec. V-A, Fig. 3:
  every row agrees with the carry a two-digit block actually produces, by
  brute force over all digit pairs in a small base;
* carry_stress_n4.txt, the oracle's results on the carry-stress pairs: the
  oracle still writes exactly these values (a regression pin of the oracle),
  and they are the exact results by CPython integers."""
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def test_scan_operator_table_matches_carry_chains():
    rows = [list(map(int, l.split())) for l in open(os.path.join(HERE, "scan_operator.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 9  # every pair of the states (0,0), (0,1), (1,0)
    base = 5

    def state(x, y):  # one digit position of x + y: (generate, propagate)
        s = x + y
        return int(s >= base), int(s == base - 1)

    table = {(g1, p1, g2, p2): (g, p) for g1, p1, g2, p2, g, p in rows}
    seen = set()
    for x1 in range(base):
        for y1 in range(base):
            for x2 in range(base):
                for y2 in range(base):
                    lo, hi = state(x1, y1), state(x2, y2)
                    # the block of both positions: carry out with carry-in 0
                    # (generate) and whether a carry-in passes through both
                    v0 = x1 + y1 + base * (x2 + y2)
                    v1 = v0 + 1
                    g = int(v0 >= base * base)
                    p = int(v0 == base * base - 1)
                    assert int(v1 >= base * base) == (g | p)
                    assert table[lo + hi] == (g, p), (lo, hi)
                    seen.add(lo + hi)
    assert seen == set(table)


def parse(line):
    """(op, index, limb arrays, flag): every |-separated field of limbs as a
    uint64 array; the trailing carry / borrow / status field (all ops but
    mul) as an int."""
    op, idx, rest = line.split(" ", 2)
    parts = [p.strip() for p in rest.split("|")]
    flag = None
    if op != "mul":
        flag = int(parts.pop())
    limbs = [np.array([int(h, 16) for h in p.split()], dtype=np.uint64) for p in parts]
    return op, int(idx), limbs, flag


def as_int(x):
    return sum(int(v) << (64 * i) for i, v in enumerate(x))


def test_carry_stress_fixture_is_exact_and_reproduced(orc):
    import sys

    sys.path.insert(0, HERE)
    import make_golden

    lines = [l.rstrip("\n") for l in open(os.path.join(HERE, "carry_stress_n4.txt"))
             if not l.startswith("#")]
    assert lines == make_golden.rows()  # the oracle still writes exactly these values
    B4 = 1 << 256
    for line in lines:
        op, _, L, tail = parse(line)
        if op == "add":
            a, b, s = map(as_int, L)
            assert s == (a + b) % B4 and tail == (a + b) // B4
        elif op == "sub":
            a, b, d = map(as_int, L)
            assert a >= b and d == a - b and tail == 0
        elif op == "mul":
            a, b, p = map(as_int, L)
            assert p == a * b
        else:
            u, v, q, r = map(as_int, L)
            assert q == u // v and r == u % v and tail == 0
