"""Build the in-tree CUDA library libhbi.so for sm_103a (nvcc, no cmake).

Translation units are compiled in parallel, then linked against the shared CUDA runtime
so that the process shares one runtime with PyTorch.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libhbi.so")
SOURCES = ["hbi_host.cpp", "hbi_entry.cu", "hbi_recompress.cu", "hbi_hmvm.cu", "hbi_multi.cu", "hbi_ode.cu", "hbi_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _compile(src, verbose=False, out=OUT, defines=()):
    obj = os.path.join(out, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-lineinfo", *ARCH, *defines,
           "-I", os.path.join(HERE, "..", "include"), "-c", os.path.join(CSRC, src), "-o", obj]
    if verbose and src.endswith(".cu"):
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "hbi.h")]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, checked=False):
    """Build libhbi.so; checked=True builds the bounds-checked variant (HBI_BOUNDS_CHECK: the
    product kernels check every table entry and gather index against their buffers and count
    violations, hbi_bounds_violations) into _build/checked/."""
    out = os.path.join(OUT, "checked") if checked else OUT
    lib = os.path.join(out, "libhbi.so")
    os.makedirs(out, exist_ok=True)
    if not force and not _stale(lib):
        return lib
    defines = ("-DHBI_BOUNDS_CHECK",) if checked else ()
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, out, defines), SOURCES))
    if verbose:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc(), "-shared", *ARCH, "-cudart", "shared", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
