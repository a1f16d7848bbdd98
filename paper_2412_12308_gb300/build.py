"""Build ``libfsolve.so`` in-tree with nvcc for sm_103a (no cmake).

Each CUDA translation unit compiles in its own process (in parallel), then
one link step produces the shared library next to this file.  Re-running is
incremental on source modification times.
"""

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfsolve.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-rdc=true", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]
# register tile sizes instantiated per element type (see fs_units.cuh)
TILE_E = {"float": (4, 5, 6, 8, 10, 12, 16, 20, 24), "double": (4, 5, 6, 8, 10, 12, 16)}


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _jobs():
    """(source, extra flags, object name) for every compilation."""
    out = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        name = os.path.basename(src)
        if name == "fs_units_inst.cu":
            for t, tiles in TILE_E.items():
                for e in tiles:
                    # the units are called from kernels launched with <= 512 threads
                    out.append((src, [f"-DFS_T={t}", f"-DFS_E={e}", "-maxrregcount=128"],
                                f"units_{t}_e{e}.o"))
        elif name == "fs_mixed_f32.cu":
            # one object per family (3 x 2^k, 5 x 2^k); units called from <= 512-thread kernels
            for odd in (3, 5):
                out.append((src, [f"-DFS_MX_ODD={odd}", "-maxrregcount=128"], f"mixed_f32_{odd}.o"))
        elif name in ("fs_pow2_f32.cu", "fs_pow2_src_f32.cu"):
            # its device units are called from kernels launched with <= 512 threads
            out.append((src, ["-maxrregcount=128"], name + ".o"))
        else:
            out.append((src, [], name + ".o"))
    return out


def _headers_mtime():
    hs = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    hs += glob.glob(os.path.join(HERE, "..", "include", "*.h"))
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _compile(job, verbose):
    src, extra, oname = job
    obj = os.path.join(BUILD, oname)
    hm = _headers_mtime()
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), hm):
        return obj, ""
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
    return obj, r.stderr


def build(verbose=False, jobs=None):
    """Compile every TU and link libfsolve.so; returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    todo = _jobs()
    # largest translation units first
    todo.sort(key=lambda j: 0 if "kernels" in j[2] else (1 if "e2" in j[2] or "e1" in j[2] else 2))
    jobs = jobs or min(len(todo), os.cpu_count() or 4)
    logs = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = []
        for obj, log in ex.map(lambda j: _compile(j, verbose), todo):
            objs.append(obj)
            if log:
                logs.append(log)
    newest = max(os.path.getmtime(o) for o in objs)
    if not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        cmd = [nvcc(), *ARCH, "-rdc=true", "-shared", "-o", LIB + ".tmp", *objs,
               "-lcudart_static", "-lrt", "-ldl", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(LIB + ".tmp", LIB)
    if verbose:
        sys.stderr.write("".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
