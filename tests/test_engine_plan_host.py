"""The compile-time FFT engine follows the runtime engine's radix plan (CPU).

The kernels with compile-time transform lengths (powers of two with register
tile 16; 3 x 2^k with 24 and 5 x 2^k with 20) derive their stage radices with
the constexpr functions ct::nstages / ct::radix of fs_fft.cuh.  For every
compiled power-of-two length those radices equal the plan of the runtime
engine (fs_radix_plan, exported by the library), stage for stage, so both
engines apply the same butterflies and twiddles (Sec. II.C's splitting,
generalised to mixed radix).  For 3 x 2^k / 5 x 2^k lengths the
compile-time engine takes the runtime plan's leading stages and merges its
trailing power-of-two stage(s) and the odd stage into one composite last
stage (radix m 2^j dividing the tile), which saves one shared-memory
exchange.  The constexpr side is evaluated by a small host program that nvcc
builds from the same header; no GPU is involved.
"""

import os
import shutil
import subprocess

import pytest

from paper_2412_12308_gb300 import fsolve

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2412_12308_gb300", "csrc")

POW2 = [128 << k for k in range(7)]  # 128 .. 8192
MIXED = [160, 192, 320, 384, 640, 768, 1280, 1536, 2560, 3072, 5120, 6144]

_PROGRAM = r"""
#include <cstdio>
#include "fs_fft.cuh"
#include "fs_mixed.h"

template <int L, int E, int ST>
void stages() {
  if constexpr (ST < fs::ct::nstages(L, E)) {
    std::printf(" %d", fs::ct::radix(L, E, ST));
    stages<L, E, ST + 1>();
  }
}
template <int L, int E>
void plan() {
  static_assert(fs::ct::ok(L, E), "length and tile accepted by the compile-time engine");
  std::printf("%d %d %d :", L, E, fs::ct::nstages(L, E));
  stages<L, E, 0>();
  std::printf("\n");
}
int main() {
@CALLS@
  return 0;
}
"""


def _calls():
    out = [f"  plan<{L}, 16>();" for L in POW2]
    # 3 x 2^k / 5 x 2^k lengths with the family's tile (fs_mixed.h)
    out += [f"  plan<{L}, fs::mx_e({L})>();" for L in MIXED]
    return "\n".join(out)


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    return None


@pytest.fixture(scope="module")
def ct_plans(tmp_path_factory):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("ctplan")
    src, exe = d / "ctplan.cu", d / "ctplan"
    src.write_text(_PROGRAM.replace("@CALLS@", _calls()))
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC, "-o", str(exe), str(src)],
                   check=True, capture_output=True, timeout=600)
    lines = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout.splitlines()
    plans = {}
    for line in lines:
        head, radices = line.split(":")
        L, E, n = (int(x) for x in head.split())
        rs = [int(x) for x in radices.split()]
        assert len(rs) == n
        plans[(L, E)] = rs
    return plans


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(fsolve.LIB_PATH):
        import __graft_entry__

        __graft_entry__.build()
    return fsolve.load()


def test_every_compiled_length_has_a_plan(ct_plans):
    assert sorted(L for L, _ in ct_plans) == sorted(POW2 + MIXED)
    for (L, E), rs in ct_plans.items():
        prod = 1
        for r in rs:
            prod *= r
            assert E % r == 0, (L, E, rs)
        assert prod == L, (L, E, rs)
        # the odd radix, if any, is the last stage
        assert all(r in (2, 4, 8, 16) for r in rs[:-1]), (L, E, rs)


def _odd(x):
    while x % 2 == 0:
        x //= 2
    return x


def test_compile_time_plan_follows_runtime_plan(ct_plans, lib):
    for (L, E), rs in ct_plans.items():
        rt = fsolve.fs_radix_plan(L, E)
        if _odd(L) == 1:
            assert rt == rs, (L, E, rs, rt)
            continue
        # leading stages identical; the runtime plan's remaining stages (at
        # least two: power-of-two stage(s) and the odd one) form the last one
        n = len(rs)
        assert rs[:-1] == rt[:n - 1], (L, E, rs, rt)
        tail = rt[n - 1:]
        prod = 1
        for r in tail:
            prod *= r
        assert len(tail) >= 2 and prod == rs[-1], (L, E, rs, rt)
        assert _odd(rs[-1]) == _odd(L) and E % rs[-1] == 0, (L, E, rs)
