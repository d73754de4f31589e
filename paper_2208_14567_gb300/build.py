"""Builds the CUDA library ``_lib/liblinks.so`` in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel, then linked into one shared library
that exports the C ABI of ``include/links.h``.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "liblinks.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-ffp-contract=off", "-Xcompiler", "-fvisibility=hidden",
              "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblinks.so")
    return path


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(ROOT, "include", "links.h"),
                                                                 os.path.abspath(__file__)]


# Device headers that the run-time compiled (topology-specialised) kernels include,
# embedded in the library as string literals.
EMBEDDED = ("dw_core.cuh", "step.cuh")


def embed_headers():
    out = ["// Generated by build.py from csrc/ headers: the run-time compiler's include files."]
    for i, name in enumerate(EMBEDDED):
        text = open(os.path.join(CSRC, name)).read()
        if ')LINKSRAW"' in text:
            raise RuntimeError(f"{name} contains the raw-string delimiter")
        out.append(f'static const char kEmbeddedName{i}[] = "{name}";')
        out.append(f'static const char kEmbeddedText{i}[] = R"LINKSRAW({text})LINKSRAW";')
    out.append(f"static const int kEmbeddedCount = {len(EMBEDDED)};")
    out.append("static const char* const kEmbeddedNames[] = {" +
               ", ".join(f"kEmbeddedName{i}" for i in range(len(EMBEDDED))) + "};")
    out.append("static const char* const kEmbeddedTexts[] = {" +
               ", ".join(f"kEmbeddedText{i}" for i in range(len(EMBEDDED))) + "};")
    path = os.path.join(OUT_DIR, "embedded_headers.inc")
    text = "\n".join(out) + "\n"
    if not os.path.exists(path) or open(path).read() != text:
        open(path, "w").write(text)


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    flags = NVCC_FLAGS + (extra or [])

    def compile_one(src):
        obj = os.path.join(OUT_DIR, os.path.basename(src).replace(".cu", ".o"))
        cmd = [cc, *ARCH, *flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    embed_headers()
    flags = flags + ["-I", OUT_DIR]
    with ThreadPoolExecutor(max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB + f".tmp{os.getpid()}"
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(cc))), "lib64")
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "shared", "-lpthread",
           # run-time compilation of topology-specialised kernels
           "-L", cuda_lib, "-lnvrtc", "-Xlinker", "-rpath", "-Xlinker", cuda_lib]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
