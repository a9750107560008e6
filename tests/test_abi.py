"""The C-ABI library builds for sm_103a and exports every declared entry point (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "mqo.h")).read()
    return sorted(set(re.findall(r"MQO_API\s+[\w\s\*]+?\b(mqo_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ("mqo_graph_create_csr", "mqo_graph_create_packed", "mqo_solver_create", "mqo_init", "mqo_step",
              "mqo_run", "mqo_reset", "mqo_round", "mqo_evaluate", "mqo_local_search", "mqo_best", "mqo_get_x",
              "mqo_set_x", "mqo_objective_f64", "mqo_spmm_grad", "mqo_last_error"):
        assert s in syms


def test_library_exports_every_declared_symbol():
    from paper_2605_06921_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)  # loading needs only the CUDA runtime, not a GPU
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    lib.mqo_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.mqo_version()


def test_python_binding_names_match_header():
    import paper_2605_06921_gb300 as mq
    assert set(mq._SIGS) | {"mqo_last_error", "mqo_version"} == set(declared_symbols())


def test_invalid_graph_is_rejected_without_gpu_work():
    """Validation runs on the host before any device call."""
    import numpy as np
    import paper_2605_06921_gb300 as mq
    lib = mq.lib()
    h = ctypes.c_void_p()
    rp = np.array([0, 1, 1], dtype=np.int64)      # edge 0->1 without 1->0
    col = np.array([1], dtype=np.int32)
    st = lib.mqo_graph_create_csr(2, 1, rp.ctypes.data_as(ctypes.c_void_p), col.ctypes.data_as(ctypes.c_void_p),
                                  None, 0, None, ctypes.byref(h))
    assert st == -2 and b"reverse" in lib.mqo_last_error()
    rp = np.array([0, 1, 2], dtype=np.int64)
    col = np.array([0, 0], dtype=np.int32)        # self loop
    st = lib.mqo_graph_create_csr(2, 2, rp.ctypes.data_as(ctypes.c_void_p), col.ctypes.data_as(ctypes.c_void_p),
                                  None, 0, None, ctypes.byref(h))
    assert st == -2 and b"self loop" in lib.mqo_last_error()


def test_struct_layouts_match_header(tmp_path):
    """The binding's ctypes structures have the sizes and field offsets of the
    C structures in include/mqo.h (compiled here with the host compiler)."""
    import shutil
    import subprocess
    import paper_2605_06921_gb300 as mq
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        import pytest
        pytest.skip("no host C compiler")
    fields = {"mqo_params": [f for f, _ in mq.Params._fields_],
              "mqo_traj_info": [f for f, _ in mq.TrajInfo._fields_]}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "mqo.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'  printf("{st} size %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'  printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines.append("  return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            st, name, val = ln.split()
            got[(st, name)] = int(val)
    for st, cls in (("mqo_params", mq.Params), ("mqo_traj_info", mq.TrajInfo)):
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for f, _ in cls._fields_:
            assert got[(st, f)] == getattr(cls, f).offset, (st, f)
