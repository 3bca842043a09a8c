"""Host-side checks of the C ABI (no GPU compute): the library builds and loads,
exports every symbol declared in include/gsn.h, and rejects bad arguments."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gsn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gsn_[a-z_]+)\s*\(", src)) - {"gsn_ctx"})


@pytest.fixture(scope="module")
def lib():
    from paper_1812_05686_gb300 import build, gsn
    if not os.path.exists(gsn.LIB_PATH):
        build.build()
    return gsn.load_library()


def test_header_declares_the_api():
    syms = declared_symbols()
    for name in ("gsn_create", "gsn_set_data", "gsn_set_species", "gsn_set_params", "gsn_eval",
                 "gsn_eval_grad", "gsn_eval_grad_batch", "gsn_expected", "gsn_destroy"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    from paper_1812_05686_gb300 import gsn
    for name in declared_symbols():
        assert hasattr(lib, name), f"libgsn.so does not export {name}"
    assert set(declared_symbols()) == set(gsn.exported_symbols())


def test_host_only_calls(lib):
    from paper_1812_05686_gb300 import gsn
    assert lib.gsn_n_slots(16) == 54
    o = gsn.gsn_options()
    assert lib.gsn_default_options(C.byref(o)) == 0
    assert o.precision == gsn.GSN_FP64 and o.max_toys_per_launch == 4096
    assert lib.gsn_default_options(None) == gsn.GSN_ERR_ARG
    assert lib.gsn_last_error(None) == b"no context"
    assert lib.gsn_create(None, None) == gsn.GSN_ERR_ARG
    bad = gsn.gsn_options(); lib.gsn_default_options(C.byref(bad)); bad.precision = 7
    h = C.c_void_p()
    assert lib.gsn_create(C.byref(h), C.byref(bad)) == gsn.GSN_ERR_ARG
    lib.gsn_destroy(None)  # no-op


def test_missing_library_fails_loudly(tmp_path):
    from paper_1812_05686_gb300 import gsn
    saved = gsn._lib
    try:
        gsn._lib = None
        with pytest.raises(RuntimeError, match="not found"):
            gsn.load_library(str(tmp_path / "libgsn.so"))
    finally:
        gsn._lib = saved
