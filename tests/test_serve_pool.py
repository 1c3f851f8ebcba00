"""CPU tests of the serving loop's host bookkeeping (csrc/serve_pool.h): the
first-fit arena allocator and the LRU cache of resident RFP arrays, compiled
with g++ through tests/host_emu/serve_pool_harness.cpp."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pool(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("pool") / "libpool.so")
    src = os.path.join(ROOT, "tests", "host_emu", "serve_pool_harness.cpp")
    subprocess.run(["g++", "-std=c++17", "-O1", "-fPIC", "-shared", src, "-o", so], check=True)
    lib = ctypes.CDLL(so)
    v, i64, sz = ctypes.c_void_p, ctypes.c_int64, ctypes.c_size_t
    sigs = {"arena_new": ([sz], v), "arena_free": ([v], None), "arena_alloc": ([v, sz], i64),
            "arena_release": ([v, i64], ctypes.c_int), "arena_in_use": ([v], sz),
            "arena_largest_free": ([v], sz), "arena_free_ranges": ([v], sz),
            "arena_capacity": ([v], sz), "cache_new": ([v], v), "cache_free": ([v], None),
            "cache_put": ([v, i64, sz, ctypes.c_int], i64), "cache_has": ([v, i64], ctypes.c_int),
            "cache_unpin": ([v, i64], ctypes.c_int), "cache_erase": ([v, i64], ctypes.c_int),
            "cache_evictions": ([v], i64), "cache_entries": ([v], sz), "cache_bytes": ([v], sz)}
    for name, (args, res) in sigs.items():
        f = getattr(lib, name)
        f.argtypes, f.restype = args, res
    return lib


def test_arena_random_alloc_free_never_overlaps_and_coalesces(pool):
    cap = 1 << 20
    a = pool.arena_new(cap)
    rng = np.random.default_rng(0)
    live = {}
    for step in range(4000):
        if live and (rng.random() < 0.45 or len(live) > 60):
            off = list(live)[rng.integers(len(live))]
            assert pool.arena_release(a, off) == 1
            del live[off]
        else:
            size = int(rng.integers(1, 40000))
            off = pool.arena_alloc(a, size)
            if off < 0:
                assert pool.arena_largest_free(a) < (size + 255) // 256 * 256
                continue
            assert off % 256 == 0 and off + size <= cap
            for o, s in live.items():        # no overlap with any live block
                assert off + size <= o or o + s <= off
            live[off] = (size + 255) // 256 * 256
        assert pool.arena_in_use(a) == sum(live.values())
    for off in list(live):
        assert pool.arena_release(a, off) == 1
    assert pool.arena_in_use(a) == 0
    assert pool.arena_free_ranges(a) == 1 and pool.arena_largest_free(a) == cap
    assert pool.arena_release(a, 12345) == 0            # not a live block
    pool.arena_free(a)


def test_cache_evicts_least_recently_used_and_never_pinned(pool):
    a = pool.arena_new(10 * 4096)
    c = pool.cache_new(a)
    for k in range(10):                                  # fill: 10 blocks of 4 KB, unpinned
        assert pool.cache_put(c, k, 4096, 0) >= 0
    assert pool.cache_entries(c) == 10 and pool.cache_bytes(c) == 10 * 4096
    assert pool.cache_has(c, 0)                          # touch 0: now most recently used
    assert pool.cache_put(c, 100, 4096, 0) >= 0          # evicts 1, the least recently used
    assert not pool.cache_has(c, 1) and pool.cache_has(c, 0)
    assert pool.cache_evictions(c) == 1
    # pin everything, then nothing can be evicted
    a2 = pool.arena_new(4 * 4096)
    c2 = pool.cache_new(a2)
    for k in range(4):
        assert pool.cache_put(c2, k, 4096, 1) >= 0
    assert pool.cache_put(c2, 9, 4096, 0) == -1
    assert pool.cache_erase(c2, 2) == 0                  # pinned: not erased
    assert pool.cache_unpin(c2, 2) == 1
    assert pool.cache_put(c2, 9, 4096, 0) >= 0           # now 2 goes
    assert not pool.cache_has(c2, 2) and pool.cache_has(c2, 9)
    # a block larger than the arena is refused without evicting anything
    before = pool.cache_entries(c)
    assert pool.cache_put(c, 555, 11 * 4096, 0) == -1
    assert pool.cache_entries(c) == before and pool.cache_evictions(c) == 1
    for h in (c, c2):
        pool.cache_free(h)
    for h in (a, a2):
        pool.arena_free(h)
