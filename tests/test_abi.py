"""The C-ABI library loads without a GPU and exports every entry point that
include/sabr.h declares (no compute calls: this runs on CPU-only hosts)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sabr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sabr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2407_20713_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_entry_points():
    names = declared_functions()
    for required in ("sabr_implied_vol", "sabr_mc_price", "sabr_calibrate", "sabr_shard_level",
                     "sabr_mc_shard_partials"):
        assert required in names


def test_library_exports_every_declared_function(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_layouts_match_the_header(lib, tmp_path):
    """Every field offset and struct size of the ctypes mirror equals what the
    C compiler lays out for include/sabr.h."""
    import shutil
    import subprocess
    from paper_2407_20713_gb300 import capi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"sabr_problem": capi.Problem, "sabr_bounds": capi.Bounds, "sabr_cooling": capi.Cooling,
               "sabr_result": capi.Result, "sabr_chain_point": capi.ChainPoint,
               "sabr_server_config": capi.ServerConfig, "sabr_server_stats": capi.ServerStats}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sabr.h"', "int main(void){"]
    expect = []
    for cname, py in structs.items():
        lines.append('printf("%%zu\\n", sizeof(%s));' % cname)
        expect.append(ctypes.sizeof(py))
        for fname, _ in py._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, fname))
            expect.append(getattr(py, fname).offset)
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == expect


def test_binding_declares_every_exported_entry_point():
    from paper_2407_20713_gb300 import capi
    missing = [n for n in declared_functions() if n not in capi.SIGNATURES]
    assert not missing, missing


def test_binding_refuses_to_run_without_the_library(tmp_path, monkeypatch):
    from paper_2407_20713_gb300 import capi
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(ImportError):
        capi.load()
