"""Host-side checks of the C-ABI library (no GPU needed).

The library must load, export every entry point that include/fsolve.h
declares, and reject bad arguments before touching a device.
"""

import ctypes
import os
import re

import pytest

from paper_2412_12308_gb300 import fsolve, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fsolve.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(fs_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(fsolve.LIB_PATH):
        import __graft_entry__

        __graft_entry__.build()
    return fsolve.load()


def test_header_declares_entry_points():
    names = _declared()
    for must in ("fs_plan_create", "fs_poisson_solve", "fs_diffusion_advance", "fs_wave_advance",
                 "fs_state_create", "fs_batch_submit", "fs_batch_wait", "fs_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, f"declared in include/fsolve.h but not exported: {missing}"


def test_binding_names_match_header():
    declared = set(_declared())
    for name in fsolve.exported_symbols():
        assert name in declared, name


def test_size_rule_matches_generator(lib):
    for n in range(0, 8200, 2):
        assert fsolve.fs_size_supported(n) == workloads.is_supported_size(n), n
    for n in (7, 9, 14, 28, 56, 8194, 16384, -8):
        assert not fsolve.fs_size_supported(n)


@pytest.mark.parametrize("L,e", [(4, 4), (8, 8), (16, 16), (32, 16), (2048, 16), (4096, 16), (8192, 16),
                                 (6, 6), (12, 12), (24, 24), (48, 24), (3072, 24), (6144, 24),
                                 (5, 5), (10, 10), (20, 20), (40, 20), (5120, 20), (8192, 8)])
def test_radix_plan_product_and_divisibility(lib, L, e):
    r = fsolve.fs_radix_plan(L, e)
    assert r, (L, e)
    prod = 1
    for x in r:
        assert x in (2, 3, 4, 5, 8, 16)
        assert e % x == 0, (L, e, r)
        prod *= x
    assert prod == L


def test_radix_plan_rejects_bad_lengths(lib):
    assert fsolve.fs_radix_plan(7, 8) == []
    assert fsolve.fs_radix_plan(24, 16) == []  # odd factor 3 does not divide the tile
    assert fsolve.fs_radix_plan(0, 16) == []


@pytest.mark.parametrize("nx,ny", [(7, 8), (8, 14), (8194, 8), (6, 8), (8, 0), (9, 9)])
def test_plan_create_rejects_sizes_without_device(lib, nx, ny):
    h = ctypes.c_void_p()
    st = lib.fs_plan_create(nx, ny, 1.0, 1.0, 0, ctypes.byref(h))
    assert st == -2  # FS_ERR_SIZE, decided on the host before any CUDA call
    assert not h.value
    assert b"unsupported size" in lib.fs_last_error()


def test_plan_create_rejects_bad_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.fs_plan_create(64, 64, 0.0, 1.0, 0, ctypes.byref(h)) == -1
    assert lib.fs_plan_create(64, 64, 1.0, -1.0, 0, ctypes.byref(h)) == -1
    assert lib.fs_plan_create(64, 64, 1.0, 1.0, 7, ctypes.byref(h)) == -1
    assert lib.fs_plan_create(64, 64, 1.0, 1.0, 0, None) == -1


def test_null_handles_are_rejected(lib):
    assert lib.fs_poisson_solve(None, None, None, None) == -1
    assert lib.fs_diffusion_advance(None, 0.1, 0.0, None, None) == -1
    assert lib.fs_wave_advance(None, 1.0, 0.0, None, None, None) == -1
    assert lib.fs_plan_destroy(None) == 0
    assert lib.fs_state_destroy(None) == 0
    assert lib.fs_state_set_source(None, None, None) == -1
    assert lib.fs_rk4_step(None, 0.1, 1, None) == -1
    assert lib.fs_rk4_output(None, None, None, None) == -1
    assert lib.fs_rk4_destroy(None) == 0
    assert lib.fs_poisson_solve_c(None, None, None, None) == -1
    assert lib.fs_state_load(None, None, 0, None) == -1
    assert lib.fs_state_save(None, None, 0, None) == -1
    assert lib.fs_rows_forward(None, 4, None, None, None) == -1
    assert lib.fs_rows_inverse(None, 4, None, None, None) == -1
    assert lib.fs_columns_apply(None, 0, 1, 0, 0.0, 0.0, 0.0, None, None) == -1
    assert lib.fs_operator_factors(None, 0, 0.0, 0.0, 0.0, 0, None, None) == -1


def test_binding_raises_with_message(lib):
    with pytest.raises(fsolve.FsError) as ei:
        fsolve.fs_plan_create(10, 7, 1.0, 1.0, fsolve.FS_F32)
    assert ei.value.status == -2
    assert "unsupported size" in str(ei.value)


def test_batch_rejects_bad_requests_on_host(lib):
    assert lib.fs_batch_submit(None, 0, None, None) == -1
    r = fsolve.FsRequest(0, None, None, None, None, None, None, 0.0, 0.0, 0.0)
    arr = (fsolve.FsRequest * 1)(r)
    t = ctypes.c_uint64()
    assert lib.fs_batch_submit(arr, 1, ctypes.byref(t), None) == -1  # no plan
    assert lib.fs_batch_wait(12345678, 0) == -1  # unknown ticket


def test_tune_cache_file_roundtrip(lib, tmp_path):
    """The autotuner's cache is JSON lines keyed by (gpu, nx, ny, dtype): load
    skips lines that are not entries, save writes every entry back."""
    src = tmp_path / "in.jsonl"
    src.write_text(
        '{"gpu": "NVIDIA GB300", "nx": 4096, "ny": 4096, "dtype": 0, "e_row": 16, "e_col": 16, "rows": 4, '
        '"cols": 1, "us": 186.2}\n'
        'not json at all\n'
        '{"gpu": "NVIDIA GB300", "nx": 1536, "ny": 1536, "dtype": 1, "e_row": 12, "e_col": 12, "rows": 8, '
        '"cols": 2, "us": 900.5}\n'
        '{"gpu": "NVIDIA GB300", "nx": 64}\n')
    lib.fs_tune_cache_clear()
    assert lib.fs_tune_cache_load(str(src).encode()) == 2
    dst = tmp_path / "out.jsonl"
    assert lib.fs_tune_cache_save(str(dst).encode()) == 2
    lines = sorted(dst.read_text().strip().splitlines())
    assert len(lines) == 2 and '"nx": 1536' in lines[0] and '"e_row": 12' in lines[0] and '"rows": 4' in lines[1]
    assert lib.fs_tune_cache_load(str(tmp_path / "missing.jsonl").encode()) == -1
    assert lib.fs_tune_cache_clear() == 2

