"""The C-ABI library builds, loads and exports every entry point of include/nks.h,
and the binding's struct layouts match the header (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nks.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nks_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    import paper_2209_08001_gb300 as nks
    return nks.load()


def test_every_declared_entry_point_is_exported(lib):
    import paper_2209_08001_gb300 as nks
    names = _declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(nks.exported_symbols()) == names


def test_struct_layouts_match_header(tmp_path, lib):
    import paper_2209_08001_gb300 as nks
    prog = tmp_path / "sizes.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "nks.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", '
                    'sizeof(nks_grid), sizeof(nks_coeffs), sizeof(nks_opts), sizeof(nks_step_info), '
                    'sizeof(nks_stats), sizeof(nks_allocator), offsetof(nks_opts, timing), offsetof(nks_coeffs, S), '
                    'offsetof(nks_opts, graphs), sizeof(nks_server_opts), sizeof(nks_request_result), '
                    'sizeof(nks_server_state), offsetof(nks_request_result, t_submit));return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(nks.nks_grid), ctypes.sizeof(nks.nks_coeffs), ctypes.sizeof(nks.nks_opts),
            ctypes.sizeof(nks.nks_step_info), ctypes.sizeof(nks.nks_stats), ctypes.sizeof(nks.nks_allocator),
            nks.nks_opts.timing.offset, nks.nks_coeffs.S.offset, nks.nks_opts.graphs.offset,
            ctypes.sizeof(nks.nks_server_opts), ctypes.sizeof(nks.nks_request_result),
            ctypes.sizeof(nks.nks_server_state), nks.nks_request_result.t_submit.offset]
    assert got == want


def test_default_options_are_the_papers(lib):
    import paper_2209_08001_gb300 as nks
    o = nks.nks_opts()
    lib.nks_default_opts(ctypes.byref(o))
    assert o.dt_init == 0.01 and o.dt_min == 0.01 and o.dt_max == 2.0 and o.zeta == 100.0
    assert o.gmres_restart == 30 and o.ilu_reuse == 1


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2209_08001_gb300 as nks
    monkeypatch.setattr(nks, "_lib", None)
    monkeypatch.setattr(nks, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        nks.load()
