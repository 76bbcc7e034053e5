"""Builds libeh.so in-tree with nvcc for sm_103a (one -gencode, parallel TUs),
and libeh_check.so: the same library with the count kernels' loads checked
against their arrays (count.cu compiled with -DEH_CHECK_LOADS)."""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libeh.so")
LIB_CHECK = os.path.join(HERE, "libeh_check.so")
CHECKED_SOURCES = ("count.cu",)   # compiled a second time with EH_CHECK_LOADS
OBJ = os.path.join(ROOT, "_build", "eh")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _deps():
    return sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))] + \
        [os.path.join(ROOT, "include", "eh.h")]


def up_to_date():
    if not os.path.exists(LIB) or not os.path.exists(LIB_CHECK):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(LIB_CHECK))
    return all(os.path.getmtime(d) <= t for d in _deps())


def _compile(src, extra, suffix=""):
    obj = os.path.join(OBJ, os.path.basename(src) + suffix + ".o")
    cmd = [NVCC] + ARCH + FLAGS + extra + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stdout + r.stderr))
    return obj, r.stderr


def build(force=False, verbose=False, extra=()):
    if not force and up_to_date():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    srcs = sources()
    checked = [x for x in srcs if os.path.basename(x) in CHECKED_SOURCES]
    jobs = [(x, list(extra), "") for x in srcs] + [(x, list(extra) + ["-DEH_CHECK_LOADS"], ".check") for x in checked]
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        res = list(ex.map(lambda j: _compile(*j), jobs))
    if verbose:
        for _, err in res:
            if err.strip():
                sys.stderr.write(err)
    plain = [o for o, _ in res[:len(srcs)]]
    check = {os.path.basename(o).replace(".check.o", ".o"): o for o, _ in res[len(srcs):]}
    for lib, objs in ((LIB, plain), (LIB_CHECK, [check.get(os.path.basename(o), o) for o in plain])):
        tmp = lib + ".tmp%d" % os.getpid()
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s" % (r.stdout + r.stderr))
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, extra=["-Xptxas", "-v"] if "--ptxas" in sys.argv else [])
    print(LIB)
