"""Build of libpyjacb300.so (sm_103a) with nvcc, in the package directory."""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC_DIR = os.path.join(HERE, "csrc")
SOURCES = ["pj_model.cu", "pj_kernels.cu", "pj_api.cu", "pj_host.cu", "pj_batch.cu", "pj_fd.cu", "pj_nvrtc.cu"]
HEADERS = ["pj_internal.h", "pj_device.h", "pj_device_kernels.cuh", "pj_fastmath.cuh"]
# device sources the library embeds for its run-time specialised kernels (pj_nvrtc.cu)
EMBEDDED = [("kSrcFastmath", "pj_fastmath.cuh"), ("kSrcDevice", "pj_device.h"),
            ("kSrcDeviceKernels", "pj_device_kernels.cuh")]
LIB = os.path.join(HERE, "libpyjacb300.so")
CALIB_SRC = "pj_calib.cu"
CALIB_LIB = os.path.join(HERE, "libpjcalib.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-shared", "--expt-relaxed-constexpr",
         "-Xcompiler", "-fvisibility=hidden", "-Xcompiler", "-Wall"]


def sources():
    return [os.path.join(SRC_DIR, s) for s in SOURCES]


def _inputs():
    return sources() + [os.path.join(SRC_DIR, h) for h in HEADERS] + [os.path.join(ROOT, "include", "pyjac_b300.h")]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build_calib(force: bool = False) -> str:
    """Measurement kernels for the benchmark's roofline denominators (libpjcalib.so)."""
    src = os.path.join(SRC_DIR, CALIB_SRC)
    deps = [src, os.path.join(SRC_DIR, "pj_fastmath.cuh")]
    if not force and os.path.exists(CALIB_LIB) and os.path.getmtime(CALIB_LIB) >= max(map(os.path.getmtime, deps)):
        return CALIB_LIB
    tmp = CALIB_LIB + ".tmp.%d" % os.getpid()
    cmd = [os.environ.get("NVCC", "nvcc")] + ARCH + ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
                                                     "-Xcompiler", "-fvisibility=hidden", "-o", tmp, src]
    subprocess.run(cmd, check=True)
    os.replace(tmp, CALIB_LIB)
    return CALIB_LIB


def write_embedded(directory: str) -> None:
    """pj_embedded_src.inc: the device sources as raw string literals, for the NVRTC path."""
    out = []
    for name, fn in EMBEDDED:
        text = open(os.path.join(SRC_DIR, fn)).read()
        if ")PJSRC" in text:
            raise RuntimeError("%s contains the raw-string delimiter" % fn)
        out.append('const char %s[] = R"PJSRC(%s)PJSRC";\n' % (name, text))
    with open(os.path.join(directory, "pj_embedded_src.inc"), "w") as f:
        f.write("".join(out))


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    build_calib(force=force)
    if not force and not needs_build():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    tmp = LIB + ".tmp.%d" % os.getpid()
    with tempfile.TemporaryDirectory(prefix="pjb300_") as gen:
        write_embedded(gen)
        cmd = [nvcc] + ARCH + FLAGS + list(extra) + ["-I", os.path.join(ROOT, "include"), "-I", gen, "-o", tmp] + \
            sources()
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    extra = sys.argv[1:]
    print(build(force=True, verbose=True, extra=extra))
