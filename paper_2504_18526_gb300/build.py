"""Build the CUDA library libsisdc.so in-tree for sm_103a.

Each translation unit is compiled by nvcc in parallel, then linked into
``paper_2504_18526_gb300/_lib/libsisdc.so``.  Nothing is installed.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libsisdc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]
SOURCES = (["ops_sipg.cu", "ops_conv.cu", "ops_misc.cu", "ops_av.cu", "tables.cpp", "sisdc.cu", "noalloc.cu", "mlp.cu", "mlp_tc.cu",
            "sweep_dispatch.cu", "sweep_cd_1dhi.cu", "stab.cu", "ensemble.cu", "ens_lo.cu", "ens_hi.cu", "ens_lo_mix.cu", "ens_hi_mix.cu"] +
           ["sweep_%s_%s%s.cu" % (p, h, m) for p in ("cd", "bu", "eu", "ns") for h in ("lo", "hi") for m in ("", "_mix")])


def nvcc():
    exe = shutil.which("nvcc")
    if exe:
        return exe
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(ROOT, "include", "sisdc.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def _compile(src, extra, verbose):
    srcp = os.path.join(CSRC, src)
    obj = os.path.join(BUILD_DIR, src + ".o")
    if not _stale(obj, srcp):
        return obj, ""
    cmd = [nvcc()] + ARCH + FLAGS + extra + ["-c", srcp, "-o", obj]
    if src.endswith(".cpp"):
        cmd = [nvcc()] + FLAGS + extra + ["-x", "c++", "-c", srcp, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    return obj, (r.stdout + r.stderr) if verbose else ""


def build(verbose=False, ptxas_info=False):
    os.makedirs(OUT_DIR, exist_ok=True)
    os.makedirs(BUILD_DIR, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra, verbose or ptxas_info), SOURCES))
    objs = [o for o, _ in results]
    for _, log in results:
        if log:
            sys.stdout.write(log)
    if not os.path.exists(LIB_PATH) or any(os.path.getmtime(o) > os.path.getmtime(LIB_PATH) for o in objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB_PATH] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: %s\n%s" % (r.stdout, r.stderr))
    return LIB_PATH


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="--ptxas" in sys.argv))
