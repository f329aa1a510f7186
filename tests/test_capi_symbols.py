"""The C-ABI library builds and exports every symbol include/bigint.h declares
(no compute calls: this runs without a GPU)."""
import os
import re
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bigint.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bigint_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_entry_points():
    syms = declared_symbols()
    for s in ("bigint_add", "bigint_sub", "bigint_mul", "bigint_mul_lo", "bigint_divmod",
              "bigint_divmod_workspace", "bigint_shinv", "bigint_strerror"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_2607_28897_gb300 import build

    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\b(bigint_[a-z0-9_]+)\b", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_binding_signatures_cover_header():
    import paper_2607_28897_gb300 as bi

    assert set(declared_symbols()) == set(bi.SIGNATURES)


def test_library_loads_and_reports_errors_without_gpu():
    import paper_2607_28897_gb300 as bi

    L = bi.load()
    assert L.bigint_version() >= 100
    assert L.bigint_strerror(bi.EDIVZERO) == b"division by zero"
    # host-side argument checks run before any device call
    assert L.bigint_add(None, None, None, None, 4, 0, None) == bi.EINVAL
    assert L.bigint_mul(None, None, None, 1, 1, 0, None) == bi.EINVAL
    assert L.bigint_add(None, None, None, None, 0, 8, None) == bi.OK  # empty batch
