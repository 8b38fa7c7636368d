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


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/sem.h compiles as strict C99, a C program links every declared
    entry point against the library, and a call with a null handle returns
    SEM_EINVAL with a message (no GPU touched)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    import __graft_entry__
    so = __graft_entry__._build_module().LIB
    refs = ",\n".join(f"    (void (*)(void)){n}" for n in declared_functions())
    prog = tmp_path / "abi_check.c"
    prog.write_text(
        '#include "sem.h"\n#include <stdio.h>\n'
        "int main(void) {\n"
        f"  void (*fns[])(void) = {{\n{refs}\n  }};\n"
        "  int rc = sem_ax((sem_handle)0, 0, 0, SEM_FP64);\n"
        '  printf("%d %d %s\\n", (int)(sizeof(fns) / sizeof(fns[0])), rc, sem_last_error());\n'
        "  return rc == SEM_EINVAL ? 0 : 1;\n}\n")
    exe = tmp_path / "abi_check"
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(prog), so,
                    "-Wl,-rpath," + os.path.dirname(so), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    count, rc, msg = out.stdout.split(" ", 2)
    assert int(count) == len(declared_functions()) and int(rc) == -1 and "invalid" in msg
