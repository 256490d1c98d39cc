"""The C-ABI library loads on a machine without a GPU and exports every entry
point that include/pcr.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LIB = os.path.join(ROOT, "paper_2609_04573_b300", "libpcr.so")


def declared():
    src = open(os.path.join(ROOT, "include", "pcr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pcr_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    """The calls of the boundary: refactor (single, batched), plan, the
    one-call retrieve(target) with its info, batched retrieve by target,
    every stream's tables, the container, free, last error, and the test
    entry that encodes given coefficients."""
    names = declared()
    for n in ["pcr_refactor", "pcr_refactor_batch", "pcr_plan", "pcr_retrieve",
              "pcr_retrieve_plan", "pcr_retrieve_batch", "pcr_retrieve_batch_plan", "pcr_get_tables",
              "pcr_serialize", "pcr_deserialize", "pcr_free", "pcr_last_error", "pcr_debug_encode"]:
        assert n in names
    src = open(os.path.join(ROOT, "include", "pcr.h")).read()
    for token in ["PCR_MODE_EXPLICIT", "has_box", "pcr_retrieval_info", "pcr_tables",
                  "PCR_ERR_UNSATISFIABLE", "PCR_ERR_TIMEOUT", "PCR_ERR_CORRUPT"]:
        assert token in src, token
    assert re.search(r"pcr_status pcr_retrieve\(const pcr_handle\* h, const pcr_target\* target, void\* d_out, "
                     r"void\* cuda_stream,\s*pcr_retrieval_info\* info\)", src)


def test_library_exports_every_declared_symbol():
    if not os.path.exists(LIB):
        from paper_2609_04573_b300 import build as b  # noqa
    lib = ctypes.CDLL(LIB)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_marshals_all_exports():
    import paper_2609_04573_b300 as pcr
    assert sorted(declared()) == pcr.EXPORTS


def test_last_error_without_gpu():
    lib = ctypes.CDLL(LIB)
    lib.pcr_last_error.restype = ctypes.c_char_p
    lib.pcr_plan.restype = ctypes.c_int
    st = lib.pcr_plan(None, None, None)
    assert st == 1 and b"null" in lib.pcr_last_error()
