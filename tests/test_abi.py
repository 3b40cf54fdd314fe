"""The C-ABI library builds, loads and exports every symbol include/fsgp.h declares
(CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(fsgp_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2603_14895_gb300 import build
    path = build.build()
    try:
        return ctypes.CDLL(path)
    except OSError as e:   # libcudart missing on a CPU-only host
        pytest.skip(f"cannot dlopen: {e}")


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert {"fsgp_graph_create", "fsgp_simulate", "fsgp_last_error"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), f"missing export {n}"


def test_host_only_entry_points(lib):
    lib.fsgp_model_planes.restype = ctypes.c_int
    assert lib.fsgp_model_planes(0) == 2
    assert lib.fsgp_model_planes(1) == 1
    assert lib.fsgp_model_planes(9) < 0
    lib.fsgp_last_error.restype = ctypes.c_char_p
    assert b"model" in lib.fsgp_last_error()
    lib.fsgp_version.restype = ctypes.c_int
    assert lib.fsgp_version() >= 10000
    # argument validation happens before any device work
    out = ctypes.c_void_p()
    assert lib.fsgp_graph_create(None, None, 0, 0, 0, None, ctypes.byref(out)) < 0


def test_product_path_does_not_touch_the_oracle():
    """The package must never import or load the oracle (test infrastructure)."""
    pkg = os.path.join(ROOT, "paper_2603_14895_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets gcc gives the
    C structure of include/fsgp.h (a mismatch would pass garbage through the ABI)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no gcc")
    from paper_2603_14895_gb300 import fsgp
    structs = ["fsgp_params", "fsgp_profile", "fsgp_options", "fsgp_result", "fsgp_request",
               "fsgp_batch_options"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fsgp.h"', "int main(void) {"]
    expect = []
    for sname in structs:
        cls = getattr(fsgp, sname)
        lines.append(f'    printf("%zu\\n", sizeof({sname}));')
        expect.append(ctypes.sizeof(cls))
        for fname, _ in cls._fields_:
            lines.append(f'    printf("%zu\\n", offsetof({sname}, {fname}));')
            expect.append(getattr(cls, fname).offset)
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(x) for x in subprocess.check_output([str(exe)]).decode().split()]
    assert got == expect


def test_binding_rejects_bad_arguments_before_any_call():
    """Argument errors in the binding raise TypeError/ValueError (not assertions, which
    `python -O` strips) before the library is called."""
    import types

    import numpy as np
    torch = pytest.importorskip("torch")
    from paper_2603_14895_gb300 import fsgp
    g = types.SimpleNamespace(n=5, handle=None)
    with pytest.raises(ValueError):
        fsgp.hk(g, np.zeros((2, 4), np.float32), 3, 0.1)
    with pytest.raises(TypeError):
        fsgp.hk(g, torch.zeros((2, 5), dtype=torch.float64), 3, 0.1)
    with pytest.raises(TypeError):
        fsgp.fsgp_graph_set_arc_weights(None, torch.zeros(4, dtype=torch.float64))
    with pytest.raises(TypeError):
        fsgp.Graph(torch.zeros(3, dtype=torch.int64), torch.zeros(2, dtype=torch.int32))
