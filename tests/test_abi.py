"""Host-side checks of the C ABI (no GPU needed): the library builds for sm_103a, loads, exports
every function include/lbm.h declares, and fails loudly instead of falling back when no GPU is
present."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["lbm_create", "lbm_set_geometry", "lbm_step", "lbm_moments", "lbm_adjoint_step", "lbm_destroy",
                 "lbm_reduce", "lbm_objective_forward", "lbm_objective_backward", "lbm_save", "lbm_load"]:
        assert must in names


def test_library_builds_and_exports_every_symbol():
    from paper_2506_21804_gb300 import build
    path = build.build()
    L = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing
    from paper_2506_21804_gb300 import lbm
    assert set(declared_functions()) == set(lbm.SIGNATURES), "binding and header disagree"


def test_no_silent_fallback_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2506_21804_gb300 import lbm
    with pytest.raises(lbm.LBMError):
        lbm.Lattice(19, 8, 8, 8, 0.6)
