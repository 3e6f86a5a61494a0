"""Build the CUDA library libgp_sscn.so (sm_103a) in-tree.

The translation units compile in parallel with nvcc, then link into one shared
library with the CUDA runtime linked statically, so the library carries no
dependency on the runtime version PyTorch ships.  Output:
paper_1605_03958_gb300/_build/libgp_sscn.so.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC_DIR = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libgp_sscn.so")
# the same library with the kernels' bounds checks on (-DGP_CHECK): an index outside
# its buffer records a status the host reports as GP_ERR_BOUNDS instead of faulting
LIB_CHECK = os.path.join(OUT_DIR, "libgp_sscn_check.so")
SOURCES = ["gp_api.cu", "gp_sweeps.cu", "gp_sweeps64.cu", "gp_reduce.cu", "gp_noalloc.cu",
           "gp_batch.cu"]
HEADERS = ["gp_device.cuh", "gp_internal.h", "gp_arena.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgp_sscn.so")
    return path


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = [os.path.join(SRC_DIR, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(HERE, "..", "include", "gp.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=(), check: bool = False) -> str:
    """Compile (if sources changed) and return the path of libgp_sscn.so, or with
    check=True of the bounds-checked libgp_sscn_check.so."""
    lib = LIB_CHECK if check else LIB
    if not force and not extra_flags and not _stale(lib):
        return lib
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    flags = [*FLAGS, *extra_flags, *(["-DGP_CHECK"] if check else [])]

    def compile_one(src):
        obj = os.path.join(OUT_DIR, src.replace(".cu", ".check.o" if check else ".o"))
        cmd = [cc, *ARCH, *flags, "-c", os.path.join(SRC_DIR, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp"
    r = subprocess.run([cc, *ARCH, "-shared", "-cudart", "static", *objs, "-o", tmp],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    flags = [a for a in sys.argv[1:] if a.startswith("-X") or a.startswith("--")]
    print(build(force=True, verbose=True, check="--check" in flags,
                extra_flags=[f for f in flags if f not in ("--force", "--check")]))
