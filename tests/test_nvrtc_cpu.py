"""The device code that the library embeds for its run-time specialised kernels compiles on its own
under NVRTC (no host headers), for sm_103a, the way pj_mech_specialize compiles it. NVRTC needs no
GPU, so this runs on the CPU."""
import ctypes
import os

import pytest

from paper_1605_03262_b300 import build

NVRTC_SUCCESS = 0


def _nvrtc():
    for name in ("libnvrtc.so.13", "libnvrtc.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libnvrtc is not loadable here")


def _compile(source: str, headers: dict):
    lib = _nvrtc()
    prog = ctypes.c_void_p()
    names = list(headers)
    hs = (ctypes.c_char_p * len(names))(*[headers[n].encode() for n in names])
    hn = (ctypes.c_char_p * len(names))(*[n.encode() for n in names])
    assert lib.nvrtcCreateProgram(ctypes.byref(prog), source.encode(), b"t.cu", len(names), hs, hn) == 0
    opts = [b"-arch=sm_103a", b"-std=c++17", b"-default-device"]
    rc = lib.nvrtcCompileProgram(prog, len(opts), (ctypes.c_char_p * len(opts))(*opts))
    n = ctypes.c_size_t()
    lib.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    log = ctypes.create_string_buffer(n.value + 1)
    lib.nvrtcGetProgramLog(prog, log)
    size = ctypes.c_size_t()
    if rc == NVRTC_SUCCESS:
        lib.nvrtcGetCUBINSize(prog, ctypes.byref(size))
    lib.nvrtcDestroyProgram(ctypes.byref(prog))
    return rc, log.value.decode(errors="replace"), size.value


def _headers():
    return {fn: open(os.path.join(build.SRC_DIR, fn)).read() for _, fn in build.EMBEDDED}


def test_embedded_sources_have_no_raw_string_delimiter(tmp_path):
    build.write_embedded(str(tmp_path))
    text = (tmp_path / "pj_embedded_src.inc").read_text()
    for name, fn in build.EMBEDDED:
        assert "const char %s[] = R\"PJSRC(" % name in text
    assert text.count(")PJSRC\"") == len(build.EMBEDDED)


def test_device_code_compiles_standalone_with_model_constants():
    src = ('#include "pj_device_kernels.cuh"\n'
           'extern "C" __global__ void __launch_bounds__(512, 1) k(const __grid_constant__ pj::KParams p) {\n'
           '    pj::KParams q = p;\n'
           '    q.m.N = 13; q.m.R = 27; q.m.rpc = 4; q.groups = 8;\n'
           '    pj::eval_kernel_body<true, 1, false>(q);\n'
           '    pj::eval_kernel_body<false, 2, true>(q);\n'
           '    pj::eval_kernel_body<true, 2, false, true>(q);\n'
           '}\n')
    rc, log, size = _compile(src, _headers())
    assert rc == NVRTC_SUCCESS, log[:3000]
    assert size > 10000
