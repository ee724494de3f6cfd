"""Oracle pins against printed values stored under tests/golden/: published
tables of K_0 and K_1 (the special function of Eq. 2), and the paper's own
figure for the length of one degree in the region of its soil-moisture
application (Section 4), which the great-circle distance (Section 7.4) has to
reproduce."""
import math
from pathlib import Path

import numpy as np

import oracle

GOLDEN = Path(__file__).parent / "golden"


def _rows(name):
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if line and not line.startswith("#"):
            yield line.split()


def test_bessel_k_table():
    rows = list(_rows("bessel_k_table.txt"))
    assert len(rows) == 10
    for nu, x, want in rows:
        got = float(oracle.bessel_k(float(nu), np.array([float(x)]))[0])
        assert abs(got - float(want)) <= 1e-10 * float(want), (nu, x, got, want)


def _degree_of_longitude(lat, radius=oracle.EARTH_RADIUS_KM):
    a = np.array([[0.0], [lat]])
    b = np.array([[1.0], [lat]])
    return float(oracle.gcd_dist(a, b, radius)[0, 0])


def _latitude_for(km, radius=oracle.EARTH_RADIUS_KM):
    """Latitude in [0, 89] N whose one-degree longitude arc is km long, by
    bisection (the arc shrinks monotonically towards the pole); None if the
    arc is shorter than km even on the equator."""
    lo, hi = 0.0, 89.0
    if _degree_of_longitude(lo, radius) < km:
        return None
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if _degree_of_longitude(mid, radius) > km:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def test_one_degree_in_the_mississippi_basin():
    g = {k: float(v) for k, v in _rows("gcd_one_degree.txt")}
    lat = _latitude_for(g["km_per_degree"])
    assert lat is not None and g["basin_lat_min"] <= lat <= g["basin_lat_max"], lat
    # the reading: a degree of latitude is ~111 km, far from the printed figure
    dlat = float(oracle.gcd_dist(np.array([[-90.0], [35.0]]), np.array([[-90.0], [36.0]]))[0, 0])
    assert abs(dlat - 111.19) < 0.01
    # the pin separates plausible mistakes: a radius in miles, or the haversine
    # without its factor 2, has no latitude at all with an 87.5 km degree
    assert _latitude_for(g["km_per_degree"], radius=3958.8) is None
    assert _latitude_for(g["km_per_degree"], radius=oracle.EARTH_RADIUS_KM / 2) is None
    assert math.isclose(_degree_of_longitude(0.0), math.pi / 180 * oracle.EARTH_RADIUS_KM, rel_tol=1e-12)
