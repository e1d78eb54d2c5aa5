"""Build the CUDA library in-tree: one nvcc process per translation unit, in parallel.

Output: ``paper_2202_03933_gb300/_build/libmortar_gb300.so`` (sm_103a only).
Run ``python -m paper_2202_03933_gb300.build`` or call :func:`build`.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmortar_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
          "-extended-lambda"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


# Sources whose pair kernels are built once per element-type combination
# (slave nodes, master nodes): the same file is compiled into a main object
# and one object per combination, so the large kernel templates compile in
# parallel (see the part declarations in csrc/context.h).
SPLIT = ("k_adjoint.cu", "k_integrate.cu", "k_tangent.cu")
COMBOS = ((4, 4), (4, 3), (3, 4), (3, 3))


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _units():
    """(source, object name, extra nvcc flags) for every object of the library."""
    units = []
    for src in _sources():
        base = os.path.basename(src)[:-3]
        units.append((src, base, []))
        if os.path.basename(src) in SPLIT:
            for ns, nm in COMBOS:
                units.append((src, f"{base}_p{ns}{nm}", [f"-DMORTAR_PAIR_NS={ns}", f"-DMORTAR_PAIR_NM={nm}"]))
    return units


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(os.path.dirname(HERE), "include", "mortar.h"), os.path.abspath(__file__)]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    units = _units()
    extra = ["-Xptxas", "-v"] if ptxas_verbose else []

    def compile_one(unit):
        src, name, defs = unit
        obj = os.path.join(OUT_DIR, name + ".o")
        cmd = [nvcc, *ARCH, *CFLAGS, *extra, *defs, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src} {' '.join(defs)}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    # the slowest units first, so that they do not start last
    units.sort(key=lambda u: (not u[2], -os.path.getsize(u[0])))
    with cf.ThreadPoolExecutor(max_workers=min(len(units), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, units))
    if verbose or ptxas_verbose:
        for _, err in results:
            if err:
                sys.stderr.write(err)
    objs = [o for o, _ in results]
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv)
    print(LIB)
