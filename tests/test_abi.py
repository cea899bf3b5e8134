"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/oca.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w \*]*?\b(oca_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libpath():
    from paper_2406_07048_gb300 import _build
    return _build.build()


def test_header_declares_entry_points():
    names = _declared()
    for n in ["oca_create", "oca_destroy", "oca_scene_create", "oca_scale_detect_batch", "oca_pair_qp_batch",
              "oca_admm_solve"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2406_07048_gb300 import binding
    assert sorted(binding.EXPORTED) == sorted(n for n in _declared() if n in binding.EXPORTED)
    assert set(binding.EXPORTED) >= set(_declared()) - set()


def test_status_string_without_gpu(libpath):
    L = ctypes.CDLL(libpath)
    L.oca_status_string.restype = ctypes.c_char_p
    assert L.oca_status_string(0) == b"OCA_OK"
    assert L.oca_status_string(5) == b"OCA_ERR_CAPACITY"


def test_null_arguments_rejected_before_any_launch(libpath):
    L = ctypes.CDLL(libpath)
    assert L.oca_create(None, 0) == 1                      # OCA_ERR_INVALID_ARGUMENT
    assert L.oca_scene_create(None, None, None) == 1
    assert L.oca_scale_detect_batch(*([None] * 11)) == 1
    assert L.oca_pair_qp_batch(*([None] * 6), ctypes.c_double(0.0), *([None] * 6)) == 1
    assert L.oca_admm_solve(*([None] * 12)) == 1
