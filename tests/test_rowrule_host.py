"""CPU checks of the numpy restatement of the FP32 row rule used by the tile
list checks: its fused multiply-add is correctly rounded (one rounding of the
exact a b + c, checked against exact rational arithmetic, including values
that land exactly on a rounding midpoint), and the rule lists a disk-only
footprint in exactly the tiles a hand count gives."""
from fractions import Fraction

import numpy as np

from tests import rowrule as rr


def _round32(x: Fraction) -> np.float32:
    """Correct round-to-nearest-even of an exact rational to binary32."""
    f = np.float32(float(x))  # float(x) rounds once to binary64; fix it up exactly below
    cands = [f, np.nextafter(f, np.float32(np.inf)), np.nextafter(f, np.float32(-np.inf))]
    best = min(cands, key=lambda c: (abs(Fraction(float(c)) - x),
                                     int(np.asarray(c, np.float32).view(np.int32)) & 1))
    return np.float32(best)


def test_fma32_is_one_rounding():
    rng = np.random.default_rng(5)
    a = rng.normal(size=3000).astype(np.float32) * np.float32(2.0) ** rng.integers(-20, 20, 3000)
    b = rng.normal(size=3000).astype(np.float32)
    c = rng.normal(size=3000).astype(np.float32) * np.float32(2.0) ** rng.integers(-20, 20, 3000)
    # cases whose exact value is a binary32 midpoint plus or minus a tiny term
    ulp = np.float32(2.0 ** -23)
    a[:4] = np.float32(1.0) + ulp
    b[:4] = np.float32(1.0) + ulp
    c[:4] = np.array([-(1.0 + 2 * 2.0 ** -23), 0.0, -2.0 ** -46, 2.0 ** -60], np.float32)
    got = rr.fma32(a, b, c)
    for i in range(a.size):
        exact = Fraction(float(a[i])) * Fraction(float(b[i])) + Fraction(float(c[i]))
        assert got[i] == _round32(exact), (i, a[i], b[i], c[i], got[i])


def test_disk_only_footprint_tiles():
    """A footprint with no ellipse (hy < 0) is the screen-filter disk: centre
    (40.3, 20.7), radius 2.12 px reaches pixel centres x in [38.5, 42.5]
    and rows 19..22: tile columns 2 (x < 48) and rows 1 (y 16..31)."""
    words = np.zeros((1, 14), np.int32)
    f = np.array([40.3, 0.0, 20.7, 0.0, 0.0, 0.0, -1.0, 0.0, 0.0, 0.0], np.float32)
    words[0, :10] = f.view(np.int32)
    words[0, 10:] = [38, 42, 19, 22]
    s, t = rr.instances(words, np.array([0]), tiles_x=10, rf=np.float32(np.sqrt(4.5)))
    assert s.tolist() == [0] and t.tolist() == [1 * 10 + 2]
