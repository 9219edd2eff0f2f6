"""The C-ABI library builds, loads without a GPU, and exports every entry point
include/condipm.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "condipm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(opf_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_11875_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("opf_create", "opf_eval_derivatives", "opf_condense", "opf_kkt_factor",
                     "opf_kkt_solve", "opf_kkt_solve_adjoint", "opf_powerflow", "opf_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol(lib):
    from paper_2203_11875_gb300 import binding
    assert sorted(binding.exported_symbols()) == _declared()
    binding.load_library()
    assert binding.load_library().opf_strerror(-3) == b"condensed matrix not positive definite"


def test_create_rejects_invalid_network_before_touching_the_gpu(lib):
    # generator 0 not on the slack bus: refused by the host-side checks
    import numpy as np
    import gridgen
    from paper_2203_11875_gb300 import binding
    net = gridgen.tiny3()
    net.slack = 2
    with pytest.raises(binding.OPFError) as e:
        binding.Handle(net)
    assert e.value.code == -1


def test_queries_reject_a_null_handle(lib):
    """The inspection calls check their handle before touching anything."""
    import ctypes as C
    from paper_2203_11875_gb300 import binding
    L = binding.load_library()
    f, nb = C.c_int(), C.c_int()
    ms = (C.c_float * 11)()
    assert L.opf_chol_choice(None, C.byref(f), C.byref(nb), ms) == -1
    assert L.opf_chol_solve_choice(None, C.byref(f), ms) == -1
    wk = (C.c_double * 2)()
    assert L.opf_forward_reach(None, C.byref(f), wk) == -1
    k, k1 = C.c_int(), C.c_int()
    ms6 = (C.c_float * 6)()
    assert L.opf_trsm_choice(None, C.byref(k), ms6, C.byref(k1)) == -1
