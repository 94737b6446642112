"""Build the CUDA library libfpt.so in-tree with nvcc (sm_103a only).

Each .cu file under csrc/ is compiled to an object in parallel (k_bfgs_pat.cu
once per BFGS pattern range), then linked into a shared library next to this
file.  Re-running skips objects whose
sources and headers are older than the object.
"""

from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import re
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfpt.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _pattern_ranges() -> list[tuple[int, int, int]]:
    """(order, first pattern, count) of every BFGS pattern object, read from FPT_BFGS_RANGES in bfgs.cuh."""
    with open(os.path.join(CSRC, "bfgs.cuh")) as f:
        text = f.read()
    m = re.search(r"#define FPT_BFGS_RANGES\(X\)((?:[^\n]*\\\n)*[^\n]*)", text)
    if not m:
        raise RuntimeError("FPT_BFGS_RANGES not found in bfgs.cuh")
    return [tuple(int(v) for v in t) for t in re.findall(r"X\((\d+),\s*(\d+),\s*(\d+)\)", m.group(1))]


def _units() -> list[tuple[str, str, list[str]]]:
    """(source, object, extra defines) of every translation unit."""
    units = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        base = os.path.basename(src)[:-3]
        if base == "k_high":
            for n in range(6, 11):
                units.append((src, os.path.join(OUT, f"{base}_o{n}.o"), [f"-DFPT_HIGH_ORDER={n}"]))
        elif base == "k_bfgs_pat":
            for n, q0, qn in _pattern_ranges():
                units.append((src, os.path.join(OUT, f"{base}_o{n}_q{q0}.o"),
                              [f"-DFPT_BFGS_ORDER={n}", f"-DFPT_BFGS_Q0={q0}u", f"-DFPT_BFGS_QN={qn}u"]))
        else:
            units.append((src, os.path.join(OUT, base + ".o"), []))
    return units


def build(verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    os.makedirs(OUT, exist_ok=True)
    headers = sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
                     glob.glob(os.path.join(ROOT, "include", "*.h")))
    flags = NVCC_FLAGS + (extra_flags or [])
    units = _units()
    jobs = []
    for src, obj, defs in units:
        if _stale(obj, [src] + headers):
            jobs.append([_nvcc(), *ARCH, *flags, *defs, "-c", src, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for cmd, res in zip(jobs, ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs)):
            if verbose or res.returncode != 0:
                print(" ".join(cmd))
                print(res.stdout + res.stderr)
            if res.returncode != 0:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    objs = [obj for _, obj, _ in units]
    if _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = [_nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            print(" ".join(cmd))
            print(res.stdout + res.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
