"""CPU checks of the boundary: the library builds, loads and exports every entry point that
include/p2mpp.h declares (no compute calls: no GPU here)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "p2mpp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(p2m_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2605_00429_gb300 import build as b
    try:
        b.build()
    except RuntimeError as e:  # pragma: no cover - nvcc missing
        pytest.skip(str(e))
    import paper_2605_00429_gb300 as p
    return p.lib()


def test_header_parses():
    names = _declared()
    assert "p2m_build" in names and "p2m_query" in names and "p2m_backward" in names
    assert len(names) >= 18


def test_every_declared_symbol_is_exported(lib):
    import paper_2605_00429_gb300 as p
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in p.SIGNATURES, f"binding lacks a signature for {name}"


def test_defaults_and_errors_without_gpu(lib):
    import ctypes
    import paper_2605_00429_gb300 as p
    prm = p.default_params()
    assert abs(prm.domain_scale - 1.5) < 1e-7 and prm.enable_aux == 1 and prm.ring_sites == 12
    assert lib.p2m_default_params(None) == -1
    assert b"NULL" in lib.p2m_last_error()
    assert lib.p2m_version().startswith(b"p2mpp")
    lib.p2m_destroy(None)  # no-op


def test_no_oracle_in_product():
    """The product package never imports or loads the oracle."""
    pkg = os.path.join(ROOT, "paper_2605_00429_gb300")
    for dp, _, fs in os.walk(pkg):
        for f in fs:
            if f.endswith((".py", ".cu", ".cuh", ".cpp", ".h")):
                txt = open(os.path.join(dp, f), errors="replace").read()
                assert "import oracle" not in txt and "from oracle" not in txt and "_oracle.so" not in txt, f


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs (build parameters, statistics, counters)
    have the C layout: every field at the same offset with the same size, and the same total
    size.  A plain C program compiled against include/p2mpp.h prints the C side."""
    import ctypes
    import shutil
    import subprocess
    import paper_2605_00429_gb300 as p
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:  # pragma: no cover
        pytest.skip("no C compiler")
    structs = {"p2m_build_params": p.BuildParams, "p2m_stats": p.Stats, "p2m_counters": p.Counters}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "p2mpp.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'printf("{cname}.{fname} %zu %zu\\n", offsetof({cname}, {fname}), '
                         f'sizeof((({cname}*)0)->{fname}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    c = {}
    for line in out:
        if line:
            key, *vals = line.split()
            c[key] = [int(v) for v in vals if v.isdigit()]
    for cname, cls in structs.items():
        assert c[cname][-1] == ctypes.sizeof(cls), cname
        for fname, ftype in cls._fields_:
            off = getattr(cls, fname).offset
            assert c[f"{cname}.{fname}"] == [off, ctypes.sizeof(ftype)], f"{cname}.{fname}"
