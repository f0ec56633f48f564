"""Host book-keeping of the fixed-budget device arena (gabor_arena_*), on the CPU.

gabor_arena_wrap over a made-up aligned address: the arena only does arithmetic on the
address, so first fit, alignment, merging and budget refusal are checked without a GPU.
"""
import ctypes

import pytest

from paper_1704_05231_gb300.bank import STATUS_CODE, load_library

BASE = 1 << 40


@pytest.fixture
def arena():
    lib = load_library()
    h = ctypes.c_void_p()
    assert lib.gabor_arena_wrap(ctypes.byref(h), ctypes.c_void_p(BASE), 4096) == 0
    yield lib, h
    lib.gabor_arena_destroy(h)


def _alloc(lib, h, n):
    p = ctypes.c_void_p()
    rc = lib.gabor_arena_alloc(h, n, ctypes.byref(p))
    return rc, (p.value - BASE if p.value else None)


def _stats(lib, h):
    c, u, f = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    assert lib.gabor_arena_stats(h, ctypes.byref(c), ctypes.byref(u), ctypes.byref(f)) == 0
    return c.value, u.value, f.value


def test_first_fit_alignment_and_budget(arena):
    lib, h = arena
    assert _alloc(lib, h, 1) == (0, 0)
    assert _alloc(lib, h, 300) == (0, 256)          # rounded to 256-byte ranges
    assert _alloc(lib, h, 1000) == (0, 768)
    assert _stats(lib, h) == (4096, 256 + 512 + 1024, 4096 - 1792)
    rc, off = _alloc(lib, h, 4096)
    assert rc == STATUS_CODE["GB_ERR_BUDGET"] and off is None


def test_free_merges_neighbours(arena):
    lib, h = arena
    offs = [_alloc(lib, h, 1024)[1] for _ in range(4)]
    assert offs == [0, 1024, 2048, 3072]
    assert _alloc(lib, h, 256)[0] == STATUS_CODE["GB_ERR_BUDGET"]
    assert lib.gabor_arena_free(h, ctypes.c_void_p(BASE + 1024)) == 0
    assert lib.gabor_arena_free(h, ctypes.c_void_p(BASE + 2048)) == 0
    assert _stats(lib, h)[2] == 2048                  # the two freed ranges merged
    assert _alloc(lib, h, 2048) == (0, 1024)
    for off in (0, 1024, 3072):
        assert lib.gabor_arena_free(h, ctypes.c_void_p(BASE + off)) == 0
    assert _stats(lib, h) == (4096, 0, 4096)


def test_bad_frees_and_arguments(arena):
    lib, h = arena
    assert lib.gabor_arena_free(h, ctypes.c_void_p(BASE + 256)) == STATUS_CODE["GB_ERR_INVALID_ARG"]
    assert _alloc(lib, h, 0)[0] == STATUS_CODE["GB_ERR_INVALID_ARG"]
    h2 = ctypes.c_void_p()
    assert lib.gabor_arena_wrap(ctypes.byref(h2), ctypes.c_void_p(BASE + 8), 4096) == STATUS_CODE["GB_ERR_INVALID_ARG"]
    assert lib.gabor_arena_destroy(None) == 0
