"""Build the in-tree CUDA library libknnwarp.so for sm_103a.

Each translation unit is compiled by nvcc in parallel and the objects are
linked into one shared library next to this file.  No CMake, no setuptools:
a plain compile that works the same on x86_64 and aarch64 hosts.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
LIB = os.path.join(HERE, "libknnwarp.so")
BUILD = os.path.join(HERE, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-fvisibility=hidden",
              "--expt-relaxed-constexpr", "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


# Point widths with DP kernels compiled (one translation unit each, so that
# nvcc compiles them in parallel); the units are generated from DP_UNIT.
DP_WIDTHS = (1, 2, 3, 4, 5, 6, 7, 8, 16)
GEN = os.path.join(BUILD, "gen")
DP_UNIT = """// Generated by build.py: DP kernel instantiations for d = {D}.
#include "dp.cuh"
#include "dp_variants.h"

namespace knn {{

namespace {{
template <int DD, int PP>
bool try_launch(const DpArgs &a, int P, int kind, int n_sm, cudaStream_t st)
{{
    if constexpr (DD == {D}) {{
        if (P == PP)
            return dp_launch_tpl<DD, PP>(a, kind, n_sm, st);
    }}
    return false;
}}
template <int DD, int PP>
int try_occ(int P, int kind)
{{
    if constexpr (DD == {D}) {{
        if (P == PP)
            return dp_occupancy_tpl<DD, PP>(kind);
    }}
    return 0;
}}
}}  // namespace

bool dp_launch_d{D}(const DpArgs &a, int P, int kind, int n_sm, cudaStream_t st)
{{
#define KNN_X(DD, PP) if (try_launch<DD, PP>(a, P, kind, n_sm, st)) return true;
    KNN_DP_VARIANTS(KNN_X)
#undef KNN_X
    return false;
}}

int dp_occ_d{D}(int P, int kind)
{{
    int v = 0;
#define KNN_X(DD, PP) v += try_occ<DD, PP>(P, kind);
    KNN_DP_VARIANTS(KNN_X)
#undef KNN_X
    return v;
}}

}}  // namespace knn
"""


def generated_units() -> list[str]:
    """Write the per-width DP units (only when their text changes)."""
    os.makedirs(GEN, exist_ok=True)
    out = []
    for d in DP_WIDTHS:
        path = os.path.join(GEN, f"dp_d{d}.cu")
        text = DP_UNIT.format(D=d)
        if not os.path.exists(path) or open(path).read() != text:
            with open(path, "w") as f:
                f.write(text)
        out.append(path)
    return out


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _digest(paths) -> str:
    h = hashlib.sha256()
    for p in sorted(paths):
        with open(p, "rb") as f:
            h.update(p.encode() + b"\0" + f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS).encode())
    h.update(DP_UNIT.encode() + repr(DP_WIDTHS).encode())
    return h.hexdigest()


def _all_inputs():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)
             if f.endswith((".cu", ".cuh", ".h"))]
    files.append(os.path.join(INCLUDE, "knnwarp.h"))
    return files


def build(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile (if sources changed) and return the path of libknnwarp.so."""
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "stamp")
    digest = _digest(_all_inputs())
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    cc = nvcc()
    srcs = sources() + generated_units()
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]

    def compile_one(pair):
        src, obj = pair
        cmd = [cc, *ARCH, *NVCC_FLAGS, "-I" + CSRC, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    jobs = jobs or min(len(srcs), max(2, os.cpu_count() or 2))
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        list(ex.map(compile_one, zip(srcs, objs)))
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
