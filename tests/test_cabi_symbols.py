"""The C-ABI library builds for sm_103a, loads, and exports every function
include/keig.h declares (no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "keig.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(?:int|const char \*)\s*\*?\s*((?:tt|keig)_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("tt_build_operator", "tt_matvec", "tt_round", "tt_solve_local", "keig_fixed_point",
                     "tt_dot_noalloc", "keig_sensitivities", "keig_batch", "keig_alpha"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2309_03347_gb300 import build as kb
    path = kb.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert lib.tt_version  # callable without a device
    lib.tt_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.tt_version()


def test_binding_refuses_without_cuda():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2309_03347_gb300 as K
    with pytest.raises(K.KeigError):
        K.tt_ctx_create()
