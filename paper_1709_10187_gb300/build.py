"""Build the CUDA library ``_build/librddmc.so`` for sm_103a with nvcc.

Each translation unit of ``csrc/`` is compiled by its own nvcc process (in
parallel), then linked into one shared library exporting the C-ABI of
``include/rddmc.h``.  The FP64 tables (leakage thresholds, eq. R_discrete
thresholds) are compiled with ``--fmad=false`` so their products and sums stay
rounded as written; the walk kernels keep fused multiply-adds for their FP32
arithmetic (their FP64 escape geometry rounds each step explicitly).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "librddmc.so")
# translation units whose device code must not contract a*b+c into an FMA
NO_FMA = {"precompute.cu", "redist.cu"}
SOURCES = ["api.cu", "precompute.cu", "walk.cu", "timewalk.cu", "redist.cu", "batch.cu", "learned.cu", "noalloc.cu", "gather.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return p


def _flags():
    # RDDMC_NVCC_EXTRA: extra nvcc options for tuning builds (e.g. -DRDDMC_WALK_MIN_BLOCKS=4)
    extra = os.environ.get("RDDMC_NVCC_EXTRA", "").split()
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC] + extra


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "rddmc.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    """Compile and link the library if missing or stale; return its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    cc = nvcc()
    flags = _flags() + list(extra_flags or [])

    def compile_one(src):
        obj = os.path.join(OUT, src.replace(".cu", ".o"))
        fma = ["--fmad=false"] if src in NO_FMA else []
        cmd = [cc] + flags + fma + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    if verbose:
        for _, err in results:
            if err.strip():
                print(err)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, extra_flags=sys.argv[1:]))
