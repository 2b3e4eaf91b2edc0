"""Build libqgeom.so in-tree for sm_103a with nvcc (no cmake, no torch
extension machinery): each .cu is compiled in parallel, then linked."""
import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libqgeom.so")
# (source, object, extra flags): the persistent 1-D propagator is compiled once
# per occupancy, its shared-memory cluster form once per cluster size and the
# 2-D one once per precision form, so the large instantiations build in
# parallel.  In the 2-D kernels CTAs read data other
# CTAs wrote in the same launch, so their global loads are cached in L2 only.
UNITS = [
    ("qg_propagate.cu", "qg_propagate_b1.o", ["-DQG_MINB=1"]),
    ("qg_propagate.cu", "qg_propagate_b2.o", ["-DQG_MINB=2"]),
    ("qg_propagate2d.cu", "qg_propagate2d_f64.o", ["-DQG_PREC=0", "-Xptxas", "-dlcm=cg"]),
    ("qg_propagate2d.cu", "qg_propagate2d_mixed.o", ["-DQG_PREC=1", "-Xptxas", "-dlcm=cg"]),
    ("qg_kernels2d.cu", "qg_kernels2d.o", ["-Xptxas", "-dlcm=cg"]),
    ("qg_propagate_cluster.cu", "qg_propagate_cluster_g1.o", ["-DQG_CLUSTER_G=1"]),
    ("qg_propagate_cluster.cu", "qg_propagate_cluster_g2.o", ["-DQG_CLUSTER_G=2"]),
    ("qg_propagate_cluster.cu", "qg_propagate_cluster_g4.o", ["-DQG_CLUSTER_G=4"]),
    ("qg_propagate_cluster.cu", "qg_propagate_cluster_g8.o", ["-DQG_CLUSTER_G=8"]),
    ("qg_propagate_cluster.cu", "qg_propagate_cluster_g16.o", ["-DQG_CLUSTER_G=16"]),
    ("qg_noalloc.cu", "qg_noalloc.o", []),
    ("qg_probe.cu", "qg_probe.o", []),
    ("qg_kernels.cu", "qg_kernels.o", []),
    ("qg_api.cu", "qg_api.o", []),
]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _deps_mtime():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "qgeom.h")]
    return max(os.path.getmtime(f) for f in files)


def build(force=False, verbose=False):
    """Compile and link; skipped when the library is newer than every source."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps_mtime():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(unit):
        src, obj, extra = unit
        obj = os.path.join(BUILD, obj)
        cmd = [nvcc] + ARCH + FLAGS + extra + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with cf.ThreadPoolExecutor(len(UNITS)) as ex:
        objs = list(ex.map(compile_one, UNITS))
    tmp = LIB + ".tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
