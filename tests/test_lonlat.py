"""The host quantiser from longitude / latitude to the grid (Web Mercator,
the projection of the tile pyramid; Sec. 3.2 gives resolution(Z) in
Web-Mercator metres), checked at points whose grid values follow by hand
(no GPU)."""
import math

import numpy as np
import pytest

from paper_2005_12489_gb300 import hv

HALF = 1 << 30


@pytest.fixture(scope="module")
def lib():
    from paper_2005_12489_gb300 import build
    build.build()
    return hv


def test_known_points(lib):
    lat_max = math.degrees(math.atan(math.sinh(math.pi)))
    got = hv.hv_lonlat_to_grid([[0, 0], [90, 0], [-90, 0], [-180, 0], [180, 0],
                                [0, lat_max], [0, -lat_max], [-180, lat_max]])
    want = [[0, 0], [1 << 29, 0], [-(1 << 29), 0], [-HALF, 0], [HALF - 1, 0],
            [0, -HALF], [0, HALF - 1], [-HALF, -HALF]]
    assert np.array_equal(got, np.array(want, dtype=np.int32))


def test_against_the_log_tan_form(lib):
    """v = (1 - ln(tan(pi/4 + lat/2)) / pi) / 2, the textbook form, away from
    unit boundaries; north is negative y (y grows southward)."""
    rng = np.random.default_rng(5)
    ll = np.stack([rng.uniform(-179, 179, 500), rng.uniform(-84, 84, 500)], 1)
    got = hv.hv_lonlat_to_grid(ll).astype(np.int64)
    for (lon, lat), (x, y) in zip(ll, got):
        u = (lon + 180) / 360 * 2 ** 31
        v = (1 - math.log(math.tan(math.pi / 4 + math.radians(lat) / 2)) / math.pi) / 2 * 2 ** 31
        assert abs(x - (u - HALF)) <= 1 and abs(y - (v - HALF)) <= 1
    assert (got[ll[:, 1] > 0, 1] < 0).all() and (got[ll[:, 1] < 0, 1] >= 0).all()
    # monotone in both coordinates
    o = np.argsort(ll[:, 0])
    assert (np.diff(got[o, 0]) >= 0).all()


def test_range_errors(lib):
    for bad in ([181, 0], [-180.5, 0], [0, 85.06], [0, -89], [float("nan"), 0]):
        with pytest.raises(hv.HVError) as e:
            hv.hv_lonlat_to_grid([[0, 0], bad])
        assert e.value.status == hv.HV_ERANGE
