"""The C library loads and exports every entry point include/gf.h declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gf.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(gf_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    import torch  # noqa: F401  (loads the CUDA runtime the library links against)
    from paper_1603_09596_gb300 import _build
    return _build.build()


def test_header_declares_the_path():
    names = declared_functions()
    for must in ("gf_build", "gf_query", "gf_query_ex", "gf_descend", "gf_candidates", "gf_score_topk",
                 "gf_forest_free", "gf_forest_import", "gf_forest_export", "gf_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(declared_functions()) <= exported


def test_binding_reports_errors_without_a_gpu(libpath):
    import paper_1603_09596_gb300 as gf
    lib = gf.lib()
    assert lib.gf_version() >= 100
    # argument validation happens before any device work
    assert lib.gf_query(None, None, 1, 1, None, None) == gf.GF_EINVAL
    assert b"null" in lib.gf_last_error()
    assert lib.gf_build(None, 10, 4, 2, 4, None, 0, None) == gf.GF_EINVAL


def test_oracle_is_not_imported_by_the_package():
    pkg = os.path.join(ROOT, "paper_1603_09596_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "gf_oracle" not in txt, f


def test_every_entry_point_rejects_null_arguments_without_a_gpu(libpath):
    """Argument checks come before any device work: a null forest, server or output is GF_EINVAL
    (and freeing a null forest is a no-op), with no GPU in the process."""
    import paper_1603_09596_gb300 as gf
    L = gf.lib()
    calls = {
        "gf_query_ex": lambda: L.gf_query_ex(None, None, 1, 1, None, None, None),
        "gf_query_workspace_size": lambda: L.gf_query_workspace_size(None, 1, None, None),
        "gf_descend": lambda: L.gf_descend(None, None, 1, None, None),
        "gf_candidates": lambda: L.gf_candidates(None, None, 1, None, None, None),
        "gf_score_topk": lambda: L.gf_score_topk(None, None, 1, None, None, 1, 1, None, None, None),
        "gf_score_screened": lambda: L.gf_score_screened(None, None, 1, None, None, 1, 1, None, None),
        "gf_prio_leaves": lambda: L.gf_prio_leaves(None, None, 1, 1, 0.0, None, None, 1, None),
        "gf_forest_import": lambda: L.gf_forest_import(None, 1, 1, 1, 1, None, None, None, None),
        "gf_forest_export": lambda: L.gf_forest_export(None, None, None, None),
        "gf_forest_get_info": lambda: L.gf_forest_get_info(None, None),
        "gf_forest_add_screen": lambda: L.gf_forest_add_screen(None, 1, None),
        "gf_forest_set_tuning": lambda: L.gf_forest_set_tuning(None, 0, 8, 0, 0, 0),
        "gf_forest_set_reflections": lambda: L.gf_forest_set_reflections(None, None),
        "gf_forest_save": lambda: L.gf_forest_save(None, b"f.gff"),
        "gf_forest_load": lambda: L.gf_forest_load(None, None),
        "gf_kernel_status": lambda: L.gf_kernel_status(None),
        "gf_server_create": lambda: L.gf_server_create(None, 0, None, None),
        "gf_server_submit": lambda: L.gf_server_submit(None, 0, None, 1, None),
        "gf_server_poll": lambda: L.gf_server_poll(None, 0, None, None, 0),
        "gf_server_get_stats": lambda: L.gf_server_get_stats(None, None),
        "gf_build_ex": lambda: L.gf_build_ex(None, 10, 4, 2, 4, None, 0, 0, None, None),
        "gf_build_reflected": lambda: L.gf_build_reflected(None, 10, 4, 2, 4, None, 0, None, 0, None, None),
    }
    bad = {name: code for name, code in ((n, f()) for n, f in calls.items()) if code != gf.GF_EINVAL}
    assert not bad, bad
    assert L.gf_forest_free(None) == gf.GF_OK


def test_binding_rejects_host_tensors_without_a_gpu(libpath):
    """The binding passes device pointers only: a host tensor is refused before any CUDA call."""
    import torch
    import paper_1603_09596_gb300 as gf
    with pytest.raises(ValueError, match="CUDA tensor"):
        gf.gf_build(torch.zeros(10, 4), 2, 4)
    with pytest.raises(ValueError, match="CUDA tensor"):
        gf.gf_query(gf.Forest(None), torch.zeros(2, 4), 1)
    with pytest.raises(ValueError, match="CUDA tensor"):
        gf.gf_forest_import(torch.zeros(10, 4), 2, 4, [[0]], [[0.0]], [[0]])
    with pytest.raises(gf.GFError) as e:
        gf.gf_forest_load(os.path.join(ROOT, "no_such_dir", "f.gff"))
    assert e.value.code == gf.GF_EIO


def test_too_deep_forest_is_rejected_before_any_device_work(libpath):
    # n > 2^30 points in leaves of one point would need depth 31: refused from the shape alone
    import numpy as np
    import paper_1603_09596_gb300 as gf
    L = gf.lib()
    one = np.zeros(1, np.int32)
    code = L.gf_forest_import(16, (1 << 30) + 1, 1, 1, 1, one.ctypes.data, one.ctypes.data, one.ctypes.data,
                              ctypes.byref(ctypes.c_void_p()))
    assert code == gf.GF_EINVAL
    assert b"tree depth 31 too large" in L.gf_last_error()
