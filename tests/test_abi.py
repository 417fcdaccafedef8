"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/mf.h (no GPU needed: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "mf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2406_04795_gb300 import build, mf
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(mf.EXPORTS) == names


def test_build_targets_sm_103a_only():
    from paper_2406_04795_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_2406_04795_gb300 import mf
    monkeypatch.setattr(mf, "_lib", None)
    monkeypatch.setattr(mf, "lib_path", lambda: str(tmp_path / "libmf.so"))
    with pytest.raises(RuntimeError):
        mf.load(build_if_missing=False)


def test_binding_structs_match_header_layout(tmp_path):
    """Every ctypes struct has the C compiler's size and field offsets."""
    from paper_2406_04795_gb300 import mf
    structs = [mf.mf_rbf, mf.mf_domain, mf.mf_trace_opts, mf.mf_trace_out, mf.mf_robot,
               mf.mf_scene, mf.mf_stats, mf.mf_tune, mf.mf_rates, mf.mf_certify_out]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mf.h"', "int main(void){"]
    expect = []
    for s in structs:
        lines.append('printf("%%zu\\n", sizeof(%s));' % s.__name__)
        expect.append(ctypes.sizeof(s))
        for name, _ in s._fields_:
            cname = "lambda" if name == "lambda_" else name
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (s.__name__, cname))
            expect.append(getattr(s, name).offset)
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == expect
