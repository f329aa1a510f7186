"""The oracle pins catch planted mistakes.

Each case copies oracle/oracle.c, plants one plausible bug (a dropped carry,
a wrong shift, a skipped add-back step, floor instead of ceiling, a wrong
sign), builds the copy, and runs the pin suite against it in a subprocess:
the suite must fail.  Mistakes are planted only in the oracle, on the CPU.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "add_drops_carry": ("uint64_t hi = (a[i] >> 32) + (b[i] >> 32) + (lo >> 32);",
                        "uint64_t hi = (a[i] >> 32) + (b[i] >> 32);"),
    "sub_never_borrows": ("        borrow = hi >> 63;\n", "        borrow = 0;\n"),
    "mul_wrong_carry_shift": ("            carry = t >> 32;\n        }\n        out->d[i + b->len]",
                              "            carry = t >> 31;\n        }\n        out->d[i + b->len]"),
    "divmod_skips_add_back": ("        if (t < 0) {\n            /* the estimate was one too large",
                              "        if (0) {\n            /* the estimate was one too large"),
    "divmod_remainder_unshifted": ("        r->d[i] = (un[i] >> s) | (s ? un[i + 1] << (32 - s) : 0);",
                                   "        r->d[i] = un[i];"),
    "step_floor_not_ceiling": ("        if (neg && dropped) {", "        if (0 && neg && dropped) {"),
    "step_wrong_sign": ("    if (!neg) {\n        nat_add(&WS, &Y, &R);",
                        "    if (neg) {\n        nat_add(&WS, &Y, &R);"),
    "shinv_wrong_power": ("    x.d[2 * h] = 1;\n    x.len = 2 * h + 1;\n    nat_divmod",
                          "    x.d[2 * h - 1] = 1;\n    x.len = 2 * h;\n    nat_divmod"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor not found once: {name}"
    src = tmp_path / "oracle_mut.c"
    src.write_text(text.replace(old, new))
    so = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-I",
                    os.path.join(ROOT, "oracle"), str(src), "-o", str(so)], check=True)
    env = dict(os.environ, ORACLE_LIB=str(so))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch {name}:\n{r.stdout[-2000:]}"
