"""Build the FAM CUDA library (libfam.so) in-tree for sm_103a.

    python -m paper_2609_26194_b300.build [--force] [-j N]

Compiles csrc/fam_api.cu, csrc/fam_probe.cu and one instantiation unit of
csrc/fam_inst.cu per (dimension, precision, order) in parallel with nvcc
(-gencode arch=compute_103a,code=sm_103a), then links them into
paper_2609_26194_b300/libfam.so.  Object files go to paper_2609_26194_b300/_build/.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libfam.so")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xptxas", "-v,-warn-spills",
         "--expt-relaxed-constexpr"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def units():
    out = [("fam_api", os.path.join(CSRC, "fam_api.cu"), []),
           ("fam_probe", os.path.join(CSRC, "fam_probe.cu"), []),
           ("fam_batch", os.path.join(CSRC, "fam_batch.cu"), []),
           ("fam_batch2d_p64", os.path.join(CSRC, "fam_batch2d.cu"), ["-DFAM_P=64"]),
           ("fam_batch2d_p32", os.path.join(CSRC, "fam_batch2d.cu"), ["-DFAM_P=32"]),
           ("fam_noalloc", os.path.join(CSRC, "fam_noalloc.cu"), []),
           ("fam_adjoint2d", os.path.join(CSRC, "fam_adjoint2d.cu"), [])]
    for d in (1, 2):
        for p in (64, 32):
            for k in (3, 4, 5, 6):
                out.append((f"fam_inst_d{d}_p{p}_k{k}", os.path.join(CSRC, "fam_inst.cu"),
                            [f"-DFAM_D={d}", f"-DFAM_P={p}", f"-DFAM_K={k}"]))
    return out


def _deps():
    files = glob.glob(os.path.join(CSRC, "*.cu*")) + [os.path.join(INCLUDE, "fam.h")]
    return max(os.path.getmtime(f) for f in files)


def _compile(job, force):
    name, src, defs = job
    obj = os.path.join(BUILD, name + ".o")
    if not force and os.path.exists(obj) and os.path.getmtime(obj) >= _deps():
        return name, obj, "", True
    cmd = [nvcc(), *ARCH, *FLAGS, *defs, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr[-6000:]}")
    return name, obj, r.stderr, False


def build(force: bool = False, jobs: int | None = None, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    jobs = jobs or max(1, os.cpu_count() or 1)
    objs, logs = [], []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        for name, obj, log, cached in ex.map(lambda j: _compile(j, force), units()):
            objs.append(obj)
            if not cached:
                logs.append((name, log))
    stale = (not os.path.exists(LIB)) or max(os.path.getmtime(o) for o in objs) > os.path.getmtime(LIB)
    if logs or stale or force:
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stderr[-4000:])
        os.replace(tmp, LIB)
        with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
            for name, log in logs:
                f.write(f"==== {name}\n{log}\n")
    if verbose:
        for name, log in logs:
            print(f"==== {name}\n{log}")
    return LIB


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--force", action="store_true")
    ap.add_argument("-j", type=int, default=None)
    ap.add_argument("-v", action="store_true")
    a = ap.parse_args()
    print(build(a.force, a.j, a.v))
    sys.exit(0)
