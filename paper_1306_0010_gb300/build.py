"""Build librhd.so (the C-ABI library of the radiation subcycle) in-tree for sm_103a.

Each CUDA translation unit is compiled in parallel with nvcc, then linked into
paper_1306_0010_gb300/librhd.so.  No CMake; needs only nvcc and a host compiler.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "librhd.so")
SOURCES = ["rhd_api.cu", "k_fp64.cu", "k_split.cu", "k_aux.cu", "k_rsla.cu", "k_gas.cu", "rhd_noalloc.cu"]
# librhd_debug.so: the kernel translation units again with -DRHD_BOUNDS_CHECK (index checks that count
# out-of-range indices and redirect the access), linked with the other objects of the release build
DEBUG_LIB = os.path.join(PKG, "librhd_debug.so")
DEBUG_SOURCES = ["k_fp64.cu", "k_split.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _newest_input() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "rhd.h"), __file__]
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False) -> str:
    newest = _newest_input()
    if (not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest and os.path.exists(DEBUG_LIB)
            and os.path.getmtime(DEBUG_LIB) >= newest):
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(job):
        src, debug = job
        obj = os.path.join(BUILD, src.replace(".cu", "_dbg.o" if debug else ".o"))
        cmd = [cc, *common, *(["-DRHD_BOUNDS_CHECK"] if debug else []), "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    jobs = [(s, False) for s in SOURCES] + [(s, True) for s in DEBUG_SOURCES]
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(compile_one, jobs))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    objs = [o for o, _ in results[:len(SOURCES)]]
    dbg = {src: o for (src, _), (o, _) in zip(jobs[len(SOURCES):], results[len(SOURCES):])}
    debug_objs = [dbg.get(s, o) for s, o in zip(SOURCES, objs)]
    for lib, lib_objs in ((LIB, objs), (DEBUG_LIB, debug_objs)):
        tmp = lib + ".tmp"
        cmd = [cc, "-shared", *ARCH, "-o", tmp, *lib_objs, "-cudart", "static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
