"""The C ABI library loads and exports every entry point include/ng.h declares (CPU only:
no compute calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ng.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ng_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_1911_01211_gb300 as ng
    if not os.path.exists(ng.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return ng.load_library()


def test_header_declares_the_expected_calls():
    names = _declared()
    for required in ("ng_create", "ng_destroy", "ng_dyson_mat", "ng_dyson_start", "ng_dyson_timestep",
                     "ng_kreduce_timestep", "ng_sigma2b_timestep", "ng_extrapolate_timestep", "ng_run_2b"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    import paper_1911_01211_gb300 as ng
    for name in _declared():
        assert hasattr(lib, name), name
        assert name in ng.SIGNATURES, name


def test_binding_has_no_cpu_fallback(tmp_path):
    import paper_1911_01211_gb300 as ng
    with pytest.raises(ImportError):
        ng._lib = None
        try:
            ng.load_library(str(tmp_path / "missing.so"))
        finally:
            ng._lib = None
            ng.load_library()
