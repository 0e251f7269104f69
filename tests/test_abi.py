"""The C-ABI library loads and exports everything include/*.h declares.

CPU only: nothing here launches a kernel or touches a device.  The argument
checks exercised below all fail before the library makes any CUDA call.
"""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(fmm_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["fmm_plan_create", "fmm_plan_destroy", "fmm_sddmm", "fmm_spmm",
                     "fmm_spmm_t", "fmm_fusedmm", "fmm_fusedmm_t", "fmm_fusedmm_bwd",
                     "fmm_fusedmm_t_bwd", "fmm_csr_validate", "fmm_status_string"]:
        assert required in names


def test_library_exports_every_declared_symbol(fmm_lib):
    lib = fmm_lib.lib()
    names = declared_functions()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", fmm_lib.LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert names <= exported, names - exported


def test_binding_covers_the_header(fmm_lib):
    assert declared_functions() <= set(fmm_lib._SIGNATURES)


def test_status_strings_and_version(fmm_lib):
    lib = fmm_lib.lib()
    for code in (0, -1, -2, -3, -4, -5):
        assert lib.fmm_status_string(code)
    assert lib.fmm_status_string(-99) == b"unknown status"
    assert lib.fmm_version() == (1 << 16)


def test_host_side_argument_errors(fmm_lib):
    lib = fmm_lib.lib()
    out = ctypes.c_void_p(1)
    # NULL pattern: rejected before any CUDA call
    assert lib.fmm_plan_create(None, 32, 0, None, None, ctypes.byref(out)) == fmm_lib.FMM_EINVAL
    assert out.value is None
    csr = fmm_lib._Csr(4, 4, 1 << 31, 0, 0)
    assert lib.fmm_plan_create(ctypes.byref(csr), 32, 0, None, None,
                               ctypes.byref(out)) == fmm_lib.FMM_EOVERFLOW
    csr = fmm_lib._Csr(-1, 4, 0, 8, 0)
    assert lib.fmm_plan_create(ctypes.byref(csr), 32, 0, None, None,
                               ctypes.byref(out)) == fmm_lib.FMM_EINVAL
    csr = fmm_lib._Csr(4, 4, 0, 8, 0)
    assert lib.fmm_plan_create(ctypes.byref(csr), 0, 0, None, None,
                               ctypes.byref(out)) == fmm_lib.FMM_EUNSUPPORTED
    assert lib.fmm_plan_create(ctypes.byref(csr), 8, 7, None, None,
                               ctypes.byref(out)) == fmm_lib.FMM_EUNSUPPORTED
    opt = fmm_lib._Options(0, 0, 333)
    assert lib.fmm_plan_create(ctypes.byref(csr), 8, 0, ctypes.byref(opt), None,
                               ctypes.byref(out)) == fmm_lib.FMM_EINVAL
    opt = fmm_lib._Options(0, -1, 0)
    assert lib.fmm_plan_create(ctypes.byref(csr), 8, 0, ctypes.byref(opt), None,
                               ctypes.byref(out)) == fmm_lib.FMM_EINVAL
    assert lib.fmm_plan_create(ctypes.byref(csr), 8, 0, None, None, None) == fmm_lib.FMM_EINVAL
    assert lib.fmm_plan_get_info(None, None) == fmm_lib.FMM_EINVAL
    assert lib.fmm_plan_destroy(None) == fmm_lib.FMM_OK
    assert lib.fmm_fusedmm(None, None, None, None, None, None) == fmm_lib.FMM_EINVAL
    assert b"NULL" in lib.fmm_last_error()
    assert lib.fmm_csr_validate(None, None, None) == fmm_lib.FMM_EINVAL


def test_product_path_has_no_oracle_or_cpu_fallback():
    # the package and the CUDA sources never reference the oracle
    pkg = os.path.join(ROOT, "paper_2203_07673_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "fmm_oracle" not in text, path


def test_missing_library_fails_loudly(monkeypatch, fmm_lib):
    monkeypatch.setattr(fmm_lib, "_lib", None)
    monkeypatch.setattr(fmm_lib, "LIB_PATH", "/nonexistent/libfmm.so")
    with pytest.raises(RuntimeError, match="not built"):
        fmm_lib.lib()


def test_header_compiles_as_c_and_links(fmm_lib, tmp_path):
    """A C11 caller: include/fmm.h compiles as plain C (no C++ or CUDA headers
    needed), links against libfmm.so, and its host-side checks answer through
    the C ABI without a GPU."""
    import shutil
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "caller.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "fmm.h"
int main(void)
{
    fmm_plan *plan = (fmm_plan *)1;
    fmm_csr csr;
    memset(&csr, 0, sizeof csr);
    csr.m = -1; csr.n = 4;
    if (fmm_plan_create(NULL, 32, FMM_F32, NULL, NULL, &plan) != FMM_EINVAL || plan) return 1;
    if (fmm_plan_create(&csr, 32, FMM_F32, NULL, NULL, &plan) != FMM_EINVAL) return 2;
    if (fmm_plan_destroy(NULL) != FMM_OK) return 3;
    if (fmm_fusedmm(NULL, NULL, NULL, NULL, NULL, NULL) != FMM_EINVAL) return 4;
    if (fmm_version() <= 0 || !fmm_status_string(FMM_EINVAL)[0]) return 5;
    printf("%d %s\n", (int)fmm_version(), fmm_status_string(FMM_EOVERFLOW));
    return 0;
}
''')
    lib_dir = os.path.dirname(fmm_lib.LIB_PATH)
    exe = tmp_path / "caller"
    res = subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-pedantic",
                          "-I" + os.path.join(ROOT, "include"),
                          str(src), "-o", str(exe), f"-L{lib_dir}", "-l:libfmm.so",
                          f"-Wl,-rpath,{lib_dir}"], capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0, (run.returncode, run.stderr)
