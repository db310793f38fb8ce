"""Build libfcsph.so in-tree for sm_103a.

    python -m paper_2606_06247_gb300.build        (or call build())

Host C++ (tables, C ABI) goes through g++, the kernels through nvcc with
-gencode arch=compute_103a,code=sm_103a; the translation units compile in
parallel and link into paper_2606_06247_gb300/libfcsph.so.
"""
import os
import platform
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfcsph.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _cuda_home():
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.isdir(c):
            return c
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("CUDA toolkit not found (set CUDA_HOME)")


def _sources():
    return [os.path.join(CSRC, f) for f in ("fcsph_tables.cpp", "fcsph_api.cpp", "fcsph_batch.cpp", "fcsph_kernels.cu", "fcsph_noalloc.cu")]


def _needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "fcsph.h")]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, verbose=False):
    if not force and not _needs_build():
        return LIB
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = ["-I" + os.path.join(cuda, "include"), "-I" + os.path.join(HERE, "..", "include")]
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    objs = []
    for src in _sources():
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        objs.append(obj)
        if src.endswith(".cu"):
            cmd = [nvcc, ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v"] + inc + ["-c", src, "-o", obj]
        else:
            cmd = ["g++", "-O2", "-std=gnu++17", "-fPIC"] + inc + ["-c", src, "-o", obj]
        jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    for cmd, p in jobs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("compile failed: " + " ".join(cmd) + "\n" + out)
        if verbose and out:
            print(out)
        if "-Xptxas" in cmd:
            with open(os.path.join(BUILD, os.path.basename(cmd[-3]) + ".ptxas.txt"), "w") as f:
                f.write(out)
    libs = ["-cudart=static"]
    if platform.machine() == "x86_64":
        libs.append("-lquadmath")
    tmp = LIB + ".tmp"
    cmd = [nvcc, ARCH, "-shared", "-o", tmp] + objs + ["-L" + os.path.join(cuda, "lib64")] + libs
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: " + " ".join(cmd) + "\n" + r.stdout)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
