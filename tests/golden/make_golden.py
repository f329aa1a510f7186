"""Writes carry_stress_n4.txt: the eight carry/borrow stress pairs of the
small configuration at n = 4 limbs and their sum, difference (a >= b
ordered), full product and quotient/remainder, computed by the CPU oracle
only (the stored values are regression pins of the oracle and expected
values of the GPU tests).

    python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def hexs(x):
    return " ".join("%016x" % int(v) for v in x)


def rows():
    import numpy as np

    import oracle
    from paper_2607_28897_gb300 import inputs

    a, b = inputs.stress_pairs(4)
    out = []
    for i in range(a.shape[0]):
        x, y = a[i], b[i]
        s, c = oracle.add(x, y)
        out.append(f"add {i} {hexs(x)} | {hexs(y)} | {hexs(s)} | {c}")
        hi, lo = (x, y) if inputs._lex_ge(x[None], y[None])[0] else (y, x)
        d, br = oracle.sub(hi, lo)
        out.append(f"sub {i} {hexs(hi)} | {hexs(lo)} | {hexs(d)} | {br}")
        out.append(f"mul {i} {hexs(x)} | {hexs(y)} | {hexs(oracle.mul(x, y))}")
        u = np.concatenate([y, x])  # an 8-limb dividend
        q, r, st = oracle.divmod_(u, x)
        out.append(f"divmod {i} {hexs(u)} | {hexs(x)} | {hexs(q)} | {hexs(r)} | {st}")
    return out


if __name__ == "__main__":
    with open(os.path.join(HERE, "carry_stress_n4.txt"), "w") as f:
        f.write("# Carry/borrow stress pairs of the small configuration (n = 4 limbs) and their\n")
        f.write("# results by the CPU oracle (tests/golden/make_golden.py): op index a | b | result\n")
        f.write("# [| remainder] | carry, borrow or oracle status; limbs hex, least significant first.\n")
        f.write("# The pairs make the carry scan of Sec. V-A (Fig. 3) run across every limb:\n")
        f.write("# (B^4-1)+(B^4-1), (B^4-1)+1, 1+(B^4-1), (B^4-1)+0, B^3 - 1, a run of ones\n")
        f.write("# broken at limb 2, 0x80.. in every limb, (B^4-1) - (B^4-2).\n")
        for line in rows():
            f.write(line + "\n")
