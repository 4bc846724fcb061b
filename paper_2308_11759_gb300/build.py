"""Builds libpcz.so (the CUDA library behind include/pcz.h) in this directory.

nvcc compiles every translation unit for sm_103a (GB300) in parallel and links
them into one shared library with the CUDA runtime linked statically.  No
floating-point contraction, no flush-to-zero, IEEE division and square root.
"""
import os
import shutil
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpcz.so")
LIB_DEBUG = os.path.join(HERE, "libpcz_debug.so")  # with the PCZ_DEBUG buffer checks
SOURCES = ["pcz_api.cu", "pcz_compress.cu", "pcz_retrieve.cu", "pcz_misc.cu", "pcz_noalloc.cu", "pcz_small.cu", "pcz_serve.cu", "pcz_batch.cu", "pcz_schedule.cu", "pcz_fd.cu"]
HEADERS = ["pcz_device.cuh", "pcz_kernels.h", "pcz_host.h", "pcz_chunk3.cuh", "pcz_chunk_small.cuh", os.path.join("..", "..", "include", "pcz.h")]

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-fmad=false", "-ftz=false",
         "-prec-div=true", "-prec-sqrt=true"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Builds libpcz.so, and with debug=True also libpcz_debug.so (PCZ_DEBUG
    buffer checks); every translation unit of both compiles in parallel."""
    variants = [(LIB, [])] + ([(LIB_DEBUG, ["-DPCZ_DEBUG"])] if debug else [])
    todo = [(lib, extra) for lib, extra in variants if force or _stale(lib)]
    if not todo:
        return LIB
    nvcc = _nvcc()
    with tempfile.TemporaryDirectory(prefix="pcz_build_") as tmp:
        procs = []
        objs = {lib: [] for lib, _ in todo}
        for lib, extra in todo:
            tag = os.path.basename(lib).replace(".so", "")
            for src in SOURCES:
                obj = os.path.join(tmp, tag + "_" + src.replace(".cu", ".o"))
                objs[lib].append(obj)
                cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
                if verbose:
                    cmd.insert(1, "-Xptxas=-v")
                procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        errors = []
        for src, pr in procs:
            out, _ = pr.communicate()
            if verbose and out:
                print(out)
            if pr.returncode != 0:
                errors.append(f"{src}:\n{out}")
        if errors:
            raise RuntimeError("libpcz build failed:\n" + "\n".join(errors))
        for lib, _ in todo:
            tmp_lib = os.path.join(tmp, os.path.basename(lib))
            link = [nvcc, *ARCH, "-shared", "-o", tmp_lib, *objs[lib], "-cudart", "static"]
            r = subprocess.run(link, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("libpcz link failed:\n" + r.stdout + r.stderr)
            shutil.copy2(tmp_lib, lib + ".tmp")
            os.replace(lib + ".tmp", lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))
