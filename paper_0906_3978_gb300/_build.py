"""Build libwf.so (CUDA C++ for sm_103a) in-tree with nvcc, translation units in parallel."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import re
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libwf.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off", "--expt-relaxed-constexpr",
         "-I", INC, "-I", CSRC]


def sizes():
    src = open(os.path.join(CSRC, "wf_ctx.h")).read()
    m = re.search(r"#define WF_SIZES\(X\)(.*?)\n\n", src, re.S)
    return [int(v) for v in re.findall(r"X\((\d+)\)", m.group(1))]


def units():
    out = []
    for f in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        name = os.path.basename(f)[:-3]
        if name == "wf_solver_inst":
            for n in sizes():
                out.append((f, os.path.join(BUILD, "%s_%d.o" % (name, n)), ["-DWF_N=%d" % n]))
        else:
            out.append((f, os.path.join(BUILD, name + ".o"), []))
    return out


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    headers = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INC, "*.h"))
    jobs = []
    for src, obj, defs in units():
        if _stale(obj, [src] + headers):
            cmd = [NVCC] + ARCH + FLAGS + list(extra) + defs + ["-c", src, "-o", obj]
            jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=max(1, os.cpu_count() or 1)) as ex:
            res = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        failed = [(c, r) for c, r in zip(jobs, res) if r.returncode != 0]
        for c, r in zip(jobs, res):
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(c[-3:]) + "\n" + r.stdout + r.stderr)
        if failed:
            raise RuntimeError("nvcc failed for %d unit(s)" % len(failed))
    objs = [o for _, o, _ in units()]
    if _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        r = subprocess.run([NVCC] + ARCH + ["-shared", "-Xlinker", "--no-undefined", "-o", tmp] + objs, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
