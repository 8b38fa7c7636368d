"""The C-ABI library builds, loads, and exports every entry point that
include/sem.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(sem_[a-z0-9_]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    b = __graft_entry__._build_module()
    if not os.path.exists(b.LIB):
        b.build()
    return ctypes.CDLL(b.LIB)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sem_setup", "sem_ax", "sem_gs", "sem_pcg_solve", "sem_destroy",
                     "sem_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_mirrors_every_declared_symbol(lib):
    import paper_2503_02134_gb300 as sem
    for n in declared_functions():
        assert n in sem.EXPORTED, n
        assert callable(getattr(sem, n))


def test_null_arguments_are_rejected_without_a_gpu(lib):
    import paper_2503_02134_gb300 as sem
    lib.sem_ax.restype = ctypes.c_int
    lib.sem_ax.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_int]
    assert lib.sem_ax(None, None, None, 0) == sem.SEM_EINVAL
    assert "invalid" in sem.sem_last_error()
