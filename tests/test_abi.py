"""The C-ABI library loads and exports every symbol include/ws.h declares
(no GPU needed: nothing is called)."""
import ctypes
import os

import pytest

from paper_2410_08946_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    import __graft_entry__
    __graft_entry__.build()
    return binding.LIB_PATH


def test_header_declares_entry_points():
    names = binding.declared_symbols()
    for must in ("ws_context_create", "ws_context_destroy", "ws_context_check", "ws_last_error",
                 "ws_gradient", "ws_watershed", "ws_waterfall", "ws_segment", "ws_segment_host"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in binding.declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads(lib_path):
    lib = binding.load()
    for n in binding.declared_symbols():
        assert getattr(lib, n) is not None


def test_shape_marshalling():
    s = binding._shape_of((5, 7))
    assert (s.ndim, s.dims[0], s.dims[1], s.dims[2]) == (2, 7, 5, 1)
    s = binding._shape_of((3, 5, 7))
    assert (s.ndim, s.dims[0], s.dims[1], s.dims[2]) == (3, 7, 5, 3)
    assert ctypes.sizeof(binding.ws_shape) == 32
    assert ctypes.sizeof(binding.ws_tuning) == 40   # 4 x int32, int64, 4 x int32 (include/ws.h)


def test_no_oracle_import_in_product():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2410_08946_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "ws_oracle" not in txt, f


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the public structs have the sizes and field
    offsets the C compiler gives include/ws.h."""
    import subprocess
    from paper_2410_08946_gb300 import binding
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "layout.c"
    structs = {"ws_tuning": binding.ws_tuning, "ws_shape": binding.ws_shape, "ws_item": binding.ws_item,
               "ws_request": binding.ws_request}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ws.h"', 'int main(void) {']
    for name, cls in structs.items():
        lines.append(f'printf("{name} %zu\\n", sizeof({name}));')
        for f in cls._fields_:
            lines.append(f'printf("{name}.{f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines.append("return 0; }")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f in cls._fields_:
            assert int(got[f"{name}.{f[0]}"]) == getattr(cls, f[0]).offset, f"{name}.{f[0]}"
