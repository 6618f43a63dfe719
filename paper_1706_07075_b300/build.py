"""Build librecon.so (the CUDA library behind include/recon.h) in-tree.

nvcc compiles every csrc/*.cu for sm_103a only and links one shared library
against the shared CUDA runtime, so streams handed over from PyTorch (which
loads the same libcudart.so.13) are valid inside the library.
"""
import concurrent.futures as cf
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "librecon.so")
OBJ_DIR = os.path.join(HERE, "_build")
# bounds-checked build: every voxel index of the walks checked before use (RECON_BOUNDS_CHECK)
CHECK_LIB = os.path.join(HERE, "librecon_check.so")
CHECK_OBJ_DIR = os.path.join(HERE, "_build_check")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-Wall", "--expt-relaxed-constexpr",
         "-I" + INCLUDE, "-I" + CSRC]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(lib=LIB):
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def _compile(src, verbose, checked=False):
    obj = os.path.join(CHECK_OBJ_DIR if checked else OBJ_DIR, os.path.basename(src)[:-3] + ".o")
    cmd = [NVCC] + ARCH + FLAGS + (["-DRECON_BOUNDS_CHECK"] if checked else []) + \
        (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


PROBE_DIR = os.path.join(CSRC, "probe")
PROBE_LIB = os.path.join(HERE, "librecon_probe.so")


def build_probe(force=False):
    """Compile librecon_probe.so (roofline probes used by bench.py)."""
    srcs = sorted(glob.glob(os.path.join(PROBE_DIR, "*.cu")))
    deps = srcs + glob.glob(os.path.join(PROBE_DIR, "*.h"))
    if not force and os.path.exists(PROBE_LIB) and all(os.path.getmtime(p) <= os.path.getmtime(PROBE_LIB) for p in deps):
        return PROBE_LIB
    tmp = PROBE_LIB + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + FLAGS + ["-I" + PROBE_DIR, "-shared", "-cudart", "shared", "-o", tmp] + srcs + \
        ["-Xlinker", "-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"probe build failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


def build(force=False, verbose=False, checked=False):
    """Compile and link librecon.so (checked: librecon_check.so, the bounds-checked
    build) unless it is newer than every source."""
    lib = CHECK_LIB if checked else LIB
    if not checked:
        build_probe(force)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(CHECK_OBJ_DIR if checked else OBJ_DIR, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, checked), _sources()))
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [NVCC] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + [o for o, _ in results] + \
        ["-Xlinker", "-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
