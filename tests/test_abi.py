"""The C-ABI library: it builds, loads and exports every symbol the public header declares; host-side
argument and model-format checks that need no GPU."""
import ctypes
import os
import re

import pytest

from paper_1605_03262_b300 import build as pjbuild
from paper_1605_03262_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def _declared_symbols():
    names = set()
    for fn in os.listdir(HEADER_DIR):
        if fn.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, fn)).read()
            names |= set(re.findall(r"PJ_API\s+[\w\s\*]*?\b(pj_\w+)\s*\(", text))
    return names


@pytest.fixture(scope="module")
def lib():
    path = pjbuild.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for must in ("pj_mech_load", "pj_mech_load_file", "pj_mech_free", "pj_mech_info", "pj_eval_dydt",
                 "pj_eval_jacobian", "pj_eval_jacobian_host", "pj_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared_symbols()) if not hasattr(lib, n)]
    assert not missing, missing


def test_model_format_errors_are_reported_without_a_gpu(lib):
    lib.pj_mech_load.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_void_p)]
    lib.pj_mech_load.restype = ctypes.c_int
    lib.pj_last_error.restype = ctypes.c_char_p
    blob = synth.to_bytes(synth.config_model(0))
    h = ctypes.c_void_p()
    for bad in (blob[:-5], b"XXXXXXXX" + blob[8:], blob + b"\0\0"):
        buf = ctypes.create_string_buffer(bad, len(bad))
        assert lib.pj_mech_load(buf, len(bad), ctypes.byref(h)) == -2       # PJ_EFORMAT
        assert lib.pj_last_error()
    assert lib.pj_mech_load(None, 0, ctypes.byref(h)) == -1                # PJ_EINVAL


def test_null_model_arguments_are_rejected(lib):
    lib.pj_eval_jacobian.restype = ctypes.c_int
    lib.pj_eval_jacobian.argtypes = [ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 3 + \
        [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    assert lib.pj_eval_jacobian(None, 4, None, None, None, 13, None, 196, None, 0, None) == -1
    lib.pj_mech_info.restype = ctypes.c_int
    assert lib.pj_mech_info(None, None, None, None) == -1


def test_oversized_stoichiometry_is_unsupported(lib):
    from paper_1605_03262_b300.synth import KIND_ELEMENTARY, REV_IRREVERSIBLE, Reaction
    from tests import mechs
    r = Reaction(kind=KIND_ELEMENTARY, rev_mode=REV_IRREVERSIBLE, reac=[(0, 5)], prod=[(1, 1)], arr=(1.0, 0.0, 0.0))
    model = mechs.one_reaction_model(r, [(1, 0), (5, 0)])
    blob = synth.to_bytes(model)
    buf = ctypes.create_string_buffer(blob, len(blob))
    h = ctypes.c_void_p()
    assert lib.pj_mech_load(buf, len(blob), ctypes.byref(h)) == -6          # PJ_EUNSUPPORTED


def test_fd_entry_points_reject_null_model(lib):
    lib.pj_eval_jacobian_fd.restype = ctypes.c_int
    lib.pj_eval_jacobian_fd.argtypes = [ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 3 + \
        [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    assert lib.pj_eval_jacobian_fd(None, 4, None, None, None, 13, None, 196, None, 0, None) == -1
    lib.pj_fd_workspace_bytes.restype = ctypes.c_int
    lib.pj_fd_workspace_bytes.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]
    b = ctypes.c_size_t()
    assert lib.pj_fd_workspace_bytes(None, 4, ctypes.byref(b)) == -1


def test_cv_entry_points_reject_null_model(lib):
    for name in ("pj_eval_dydt_cv", "pj_eval_jacobian_cv"):
        fn = getattr(lib, name)
        fn.restype = ctypes.c_int
    lib.pj_eval_dydt_cv.argtypes = [ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 3 + \
        [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    lib.pj_eval_jacobian_cv.argtypes = [ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 3 + \
        [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    assert lib.pj_eval_dydt_cv(None, 4, None, None, None, 13, None, 14, None) == -1
    assert lib.pj_eval_jacobian_cv(None, 4, None, None, None, 13, None, 196, None, 0, None) == -1


def test_concentration_basis_entry_points_reject_null_model(lib):
    lib.pj_conc_pattern.restype = ctypes.c_int
    lib.pj_conc_pattern.argtypes = [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p, ctypes.c_void_p]
    nnz = ctypes.c_int64(-7)
    assert lib.pj_conc_pattern(None, ctypes.byref(nnz), None, None) == -1
    lib.pj_eval_jacobian_conc.restype = ctypes.c_int
    lib.pj_eval_jacobian_conc.argtypes = [ctypes.c_void_p, ctypes.c_int64] + [ctypes.c_void_p] * 4 + \
        [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]
    assert lib.pj_eval_jacobian_conc(None, 4, None, None, None, None, 12, None, 300, None, 0, None) == -1


def test_header_and_library_work_from_plain_c(tmp_path):
    """The ABI is C: the header compiles as C99 with warnings as errors, and a C program linked
    against the library gets the documented status codes and error text (no GPU needed)."""
    import shutil
    import subprocess
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_1605_03262_b300 import build
    src = tmp_path / "t.c"
    src.write_text(
        '#include <string.h>\n#include "pyjac_b300.h"\n'
        "int main(void) {\n"
        "    if (pj_version() <= 0) return 1;\n"
        "    if (pj_eval_jacobian(NULL, 4, NULL, NULL, NULL, 13, NULL, 196, NULL, 0, NULL) != PJ_EINVAL) return 2;\n"
        "    if (strlen(pj_last_error()) == 0) return 3;\n"
        "    if (pj_eval_jacobian_cv(NULL, 4, NULL, NULL, NULL, 13, NULL, 196, NULL, 0, NULL) != PJ_EINVAL) return 4;\n"
        "    if (pj_mech_specialize(NULL, 1) != PJ_EINVAL) return 5;\n"
        "    return 0;\n}\n")
    exe = tmp_path / "t"
    libdir = os.path.dirname(build.LIB)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(build.ROOT, "include"),
                    str(src), "-L", libdir, "-lpyjacb300", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    assert subprocess.run([str(exe)]).returncode == 0
