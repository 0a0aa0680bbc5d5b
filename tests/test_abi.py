"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h (no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(mg(?:enkf|k)_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("mgenkf_create", "mgenkf_forecast", "mgenkf_analyse", "mgenkf_prolong_correct",
                     "mgenkf_destroy", "mgenkf_cycle", "mgenkf_rmse", "mgk_forecast"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2012_10091_gb300 import build as B
    lib_path = B.build()
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_imports_and_config_layout_matches_header():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2012_10091_gb300 import mgenkf as M
    # 8 int32 + 6 double + 1 uint64 with natural alignment
    assert ctypes.sizeof(M.mgenkf_config) == 8 * 4 + 6 * 8 + 8
    assert M.mgenkf_config.seed.offset == 8 * 4 + 6 * 8
