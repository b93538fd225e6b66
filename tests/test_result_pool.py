"""The result pool (HiVision Sec. 4.2 Result Pool; Sec. 4.1 Parse Tasks drops
tiles already rendered): a host-memory store of tiles keyed by request and
style, with least-recently-used eviction under a byte capacity and a time to
live.  Host code only, so these run without a GPU."""
import time

import numpy as np
import pytest

from paper_2005_12489_gb300 import hv


@pytest.fixture(scope="module")
def lib():
    from paper_2005_12489_gb300 import build
    build.build()
    return hv


def req(z, x, y, r16, mode=hv.HV_MODE_COVERAGE, layer=0):
    r = np.zeros(1, dtype=hv.REQ_DTYPE)
    r["z"], r["x"], r["y"], r["r16"], r["mode"], r["layer"] = z, x, y, r16, mode, layer
    return r


def tile(seed, n=65536):
    return np.random.default_rng(seed).integers(0, 256, n, dtype=np.uint8)


def test_put_get_and_keys(lib):
    pool = hv.hv_result_pool_create(1 << 20)
    try:
        s1, s2 = hv.make_style((1, 2, 3), (4, 5, 6)), hv.make_style((9, 9, 9), (4, 5, 6))
        a = tile(1)
        hv.hv_result_pool_put(pool, req(5, 3, 4, 16), s1, a)
        out = np.zeros(65536, np.uint8)
        assert hv.hv_result_pool_get(pool, req(5, 3, 4, 16), s1, out) and np.array_equal(out, a)
        # the style is part of the key in RGBA mode only
        assert hv.hv_result_pool_get(pool, req(5, 3, 4, 16), s2, out)
        for other in (req(5, 3, 4, 17), req(5, 4, 3, 16), req(6, 3, 4, 16), req(5, 3, 4, 16, layer=1),
                      req(5, 3, 4, 16, mode=hv.HV_MODE_MASK)):
            assert not hv.hv_result_pool_get(pool, other, s1, out)
        b = tile(2, 262144)
        hv.hv_result_pool_put(pool, req(5, 3, 4, 16, hv.HV_MODE_RGBA), s1, b)
        big = np.zeros(262144, np.uint8)
        assert hv.hv_result_pool_get(pool, req(5, 3, 4, 16, hv.HV_MODE_RGBA), s1, big) and np.array_equal(big, b)
        assert not hv.hv_result_pool_get(pool, req(5, 3, 4, 16, hv.HV_MODE_RGBA), s2, big)
        with pytest.raises(hv.HVError):                       # output too small for the tile
            hv.hv_result_pool_get(pool, req(5, 3, 4, 16, hv.HV_MODE_RGBA), s1, out)
        # a second put of the same key replaces the tile
        c = tile(3)
        hv.hv_result_pool_put(pool, req(5, 3, 4, 16), s1, c)
        assert hv.hv_result_pool_get(pool, req(5, 3, 4, 16), None, out) and np.array_equal(out, c)
        st = hv.hv_result_pool_stats(pool)
        assert st["entries"] == 2 and st["bytes"] == 65536 + 262144 and st["inserts"] == 3
        assert st["hits"] == 5 and st["misses"] == 6
        hv.hv_result_pool_clear(pool)
        assert hv.hv_result_pool_stats(pool)["entries"] == 0
        assert not hv.hv_result_pool_get(pool, req(5, 3, 4, 16), s1, out)
    finally:
        hv.hv_result_pool_destroy(pool)


def test_lru_eviction_under_capacity(lib):
    pool = hv.hv_result_pool_create(3 * 65536)
    try:
        out = np.zeros(65536, np.uint8)
        for k in range(3):
            hv.hv_result_pool_put(pool, req(8, k, 0, 16), None, tile(k))
        assert hv.hv_result_pool_get(pool, req(8, 0, 0, 16), None, out)     # 0 is now most recent
        hv.hv_result_pool_put(pool, req(8, 3, 0, 16), None, tile(3))        # evicts 1, the least recent
        assert not hv.hv_result_pool_get(pool, req(8, 1, 0, 16), None, out)
        for k in (0, 2, 3):
            assert hv.hv_result_pool_get(pool, req(8, k, 0, 16), None, out) and np.array_equal(out, tile(k))
        st = hv.hv_result_pool_stats(pool)
        assert st["evictions"] == 1 and st["entries"] == 3 and st["bytes"] <= st["capacity"]
        with pytest.raises(hv.HVError) as e:                                # larger than the pool
            hv.hv_result_pool_put(pool, req(8, 9, 0, 16, hv.HV_MODE_RGBA), None, tile(9, 262144))
        assert e.value.status == hv.HV_ENOMEM
        assert hv.hv_result_pool_stats(pool)["rejected"] == 1
    finally:
        hv.hv_result_pool_destroy(pool)


def test_time_to_live(lib):
    pool = hv.hv_result_pool_create(1 << 20, ttl_ms=150)
    try:
        out = np.zeros(65536, np.uint8)
        hv.hv_result_pool_put(pool, req(9, 1, 1, 16), None, tile(1))
        assert hv.hv_result_pool_get(pool, req(9, 1, 1, 16), None, out)
        time.sleep(0.3)
        assert not hv.hv_result_pool_get(pool, req(9, 1, 1, 16), None, out)
        st = hv.hv_result_pool_stats(pool)
        assert st["expirations"] == 1 and st["entries"] == 0
    finally:
        hv.hv_result_pool_destroy(pool)


def test_bad_arguments(lib):
    L = hv.lib()
    assert L.hv_result_pool_create(0, 0, None) == hv.HV_EINVAL
    assert L.hv_result_pool_destroy(None) == hv.HV_EINVAL
    assert L.hv_result_pool_get(None, None, None, None, 0, None) == hv.HV_EINVAL
