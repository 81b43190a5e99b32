"""Build the in-tree CUDA library liblbm.so for sm_103a (nvcc, no torch types).

Each lattice's kernels live in their own translation unit so the four
compiles run in parallel; the result is paper_2409_10399_gb300/_build/liblbm.so.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "liblbm.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
SOURCES = ["lbm_capi.cu", "lbm_d1q3.cu", "lbm_d2q9.cu", "lbm_d3q19.cu",
           "lbm_ref_d1q3.cu", "lbm_ref_d2q9.cu", "lbm_ref_d3q19.cu", "lbm_noalloc.cu", "lbm_batch.cu",
           "lbm_fno.cu"]
# the FP64 reference path is compiled without floating-point contraction;
# the fast paths use approximate single-precision division and square root
FAST = ["-prec-div=false", "-prec-sqrt=false"]
PER_FILE_FLAGS = {"lbm_ref_d1q3.cu": ["-fmad=false"], "lbm_ref_d2q9.cu": ["-fmad=false"],
                  "lbm_ref_d3q19.cu": ["-fmad=false"], "lbm_d1q3.cu": FAST, "lbm_d2q9.cu": FAST,
                  "lbm_d3q19.cu": FAST}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-Xcompiler", "-ffp-contract=off",
              "--expt-relaxed-constexpr", "-I" + INCLUDE]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "lbm.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def build(force=False, verbose=False, extra_flags=()):
    """Compile (if stale) and return the path of liblbm.so."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= _deps():
        return SO
    nvcc = _nvcc()
    procs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        cmd = [nvcc] + ARCH + NVCC_FLAGS + PER_FILE_FLAGS.get(src, []) + list(extra_flags) + \
            ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    tmp = SO + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl", "-lpthread"])
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
