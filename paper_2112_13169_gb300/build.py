"""Build libvg.so (the C-ABI voxel-grid library) for sm_103a, in-tree.

Each .cu translation unit is compiled by nvcc in parallel with one
-gencode (compute_103a -> sm_103a) and linked into
paper_2112_13169_gb300/_build/libvg.so.  The files that carry the method's
FP32 arithmetic (K1, K3) are also built with -fmad=false so that no
multiply-add is ever contracted.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libvg.so")

SOURCES = ["vg_api.cu", "k_voxelize.cu", "k_inflate.cu", "k_raytrace.cu", "k_merge.cu", "k_batch.cu",
           "vg_noalloc.cu", "vg_server.cu"]
NO_FMAD = {"k_voxelize.cu", "k_raytrace.cu", "k_batch.cu"}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc"),
            shutil.which("nvcc") or ""]
    for c in cand:
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: libvg.so cannot be built")


def _flags(src):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
                "-I", os.path.join(ROOT, "include"), "-I", CSRC, "--expt-relaxed-constexpr"]
    if src in NO_FMAD:
        f += ["-fmad=false"]
    if os.environ.get("VG_PTXAS_VERBOSE"):
        f += ["-Xptxas", "-v"]
    return f


def _stale(out, deps):
    return not os.path.exists(out) or any(os.path.getmtime(d) > os.path.getmtime(out) for d in deps)


def build(force=False, verbose=False):
    """Compile and link libvg.so if any source changed; return its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    headers = [os.path.join(CSRC, h) for h in ("vg_internal.cuh", "vg_units.cuh", "vg_rt.cuh", "vg_sync.cuh",
                                               "vg_host.h")]
    headers.append(os.path.join(ROOT, "include", "vg.h"))
    objs, jobs = [], []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s, os.path.join(HERE, "build.py")] + headers):
            jobs.append([cc] + _flags(src) + ["-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max(1, len(jobs))) as ex:
        list(ex.map(run, jobs))
    if jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        run([cc] + ARCH + ["-shared", "-o", tmp] + objs)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
