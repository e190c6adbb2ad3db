"""CPU-side checks of the C ABI: the library builds for sm_103a, loads,
exports every entry point that include/lbm.h declares, its descriptor structs
have the layout the Python binding assumes, and it refuses to run without a
GPU instead of falling back to anything."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


@pytest.fixture(scope="module")
def lbm():
    from paper_1906_05445_gb300 import build
    build.build()
    from paper_1906_05445_gb300 import lbm as L
    return L


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_api():
    names = declared_functions()
    for must in ("lbm_create", "lbm_step", "lbm_get_velocity", "lbm_get_force_torque",
                 "lbm_set_scheme", "lbm_add_solid", "lbm_run_to_steady"):
        assert must in names


def test_library_exports_every_declared_symbol(lbm):
    out = subprocess.run(["nm", "-D", "--defined-only", lbm._LIB_PATH],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r" T (lbm_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    for n in declared_functions():
        getattr(lbm.lib, n)


def test_struct_layout_matches_header(lbm, tmp_path):
    prog = tmp_path / "sizes.c"
    prog.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "lbm.h"\n'
                    'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n",'
                    ' sizeof(lbm_lattice_desc),'
                    ' sizeof(lbm_solid_desc), sizeof(lbm_scheme_desc), sizeof(lbm_info),'
                    ' offsetof(lbm_lattice_desc, body_force), offsetof(lbm_solid_desc, fluid_inside),'
                    ' sizeof(lbm_domain_desc), sizeof(lbm_request), sizeof(lbm_result),'
                    ' offsetof(lbm_request, deadline_s), offsetof(lbm_result, device_bytes));'
                    'return 0;}\n')
    exe = tmp_path / "sizes"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)], check=True)
    got = list(map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                       check=True).stdout.split()))
    want = [C.sizeof(lbm.lbm_lattice_desc), C.sizeof(lbm.lbm_solid_desc),
            C.sizeof(lbm.lbm_scheme_desc), C.sizeof(lbm.lbm_info),
            lbm.lbm_lattice_desc.body_force.offset, lbm.lbm_solid_desc.fluid_inside.offset,
            C.sizeof(lbm.lbm_domain_desc), C.sizeof(lbm.lbm_request), C.sizeof(lbm.lbm_result),
            lbm.lbm_request.deadline_s.offset, lbm.lbm_result.device_bytes.offset]
    assert got == want


def test_version_and_null_arguments(lbm):
    assert b"sm_103a" in lbm.lbm_version()
    assert lbm.lbm_create(None, None, None) == -1      # LBM_ERR_ARG
    assert lbm.lbm_step(None, 1) == -1
    assert lbm.lbm_sync(None) == -1


def test_create_without_gpu_fails_loudly(lbm):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    d = lbm.lbm_lattice_desc()
    d.lattice, d.nx, d.ny, d.nz, d.tau, d.precision = 1, 8, 8, 8, 0.8, 1
    h = C.c_void_p()
    assert lbm.lbm_create(C.byref(h), C.byref(d), None) == -3   # LBM_ERR_CUDA
    with pytest.raises(lbm.LbmError):
        lbm.Lattice(1, 8, 8, 8, 0.8)


def test_invalid_descriptors_rejected_before_device_work(lbm):
    d = lbm.lbm_lattice_desc()
    d.lattice, d.nx, d.ny, d.nz, d.tau = 1, 8, 8, 8, 0.5   # tau must exceed 1/2
    h = C.c_void_p()
    assert lbm.lbm_create(C.byref(h), C.byref(d), None) == -1
    d.tau, d.lattice = 0.8, 7
    assert lbm.lbm_create(C.byref(h), C.byref(d), None) == -1
    d.lattice, d.nx = 1, 0
    assert lbm.lbm_create(C.byref(h), C.byref(d), None) == -1
    # more nodes than a 32-bit node index holds: refused before any device call
    d.nx, d.ny, d.nz = 2048, 2048, 1024
    assert lbm.lbm_create(C.byref(h), C.byref(d), None) == -4   # LBM_ERR_UNSUPPORTED
    d.nx, d.ny, d.nz, d.precision = 8, 8, 8, 9                # unknown precision
    assert lbm.lbm_create(C.byref(h), C.byref(d), None) == -1
    d.precision, d.collision = 1, 5                            # unknown collision
    assert lbm.lbm_create(C.byref(h), C.byref(d), None) == -1


def test_header_is_plain_c(tmp_path):
    """include/lbm.h compiles as strict C99 (no C++ or compiler extensions in
    the ABI), so a C caller can use it as it is."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "use.c"
    src.write_text('#include "include/lbm.h"\n'
                   "int main(void) {\n"
                   "  lbm_lattice_desc d; lbm_request r; lbm_result s; lbm_domain_desc f;\n"
                   "  (void)d; (void)r; (void)s; (void)f;\n"
                   "  return 0;\n"
                   "}\n")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-I", root, "-c", str(src), "-o", str(tmp_path / "use.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
