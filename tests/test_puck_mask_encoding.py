"""The child-occupancy mask that the distance search keeps in the low 8
mantissa bits of a puck's radius: the radius is first rounded up to a
multiple of 256 units in the last place, then the mask is or-ed in, so the
stored radius is never below the true one (the lower bound stays
conservative) and exceeds it by at most 2^-14 relative.  Checked on the bits
of IEEE-754 binary32 values, from the rule's definition."""
import numpy as np


def encode(r, mask):
    bits = r.astype(np.float32).view(np.uint32)
    up = (bits + np.uint32(0xFF)) & np.uint32(0xFFFFFF00)
    return (up | mask.astype(np.uint32)).view(np.float32)


def test_radius_never_shrinks_and_stays_within_two_to_minus_14():
    rng = np.random.default_rng(0)
    # radii over the whole positive normal range, plus zero and subnormals
    r = np.concatenate([
        np.float32(2.0) ** rng.uniform(-126, 127, 200_000).astype(np.float32),
        np.array([0.0, 1e-45, 1e-40, 1.0, 3.0e38], np.float32),
    ]).astype(np.float32)
    for mask in (np.zeros_like(r, np.uint32), np.full(r.shape, 0xFF, np.uint32),
                 rng.integers(0, 256, r.shape).astype(np.uint32)):
        s = encode(r, mask)
        assert np.all(np.isfinite(s))
        assert np.all(s >= r)
        big = r > 1e-37
        assert np.all((s[big].astype(np.float64) - r[big]) <= 2.0 ** -14 * r[big].astype(np.float64))
        assert np.array_equal(s.view(np.uint32) & 0xFF, mask)


def test_empty_marker_keeps_its_sign():
    # empty nodes carry radius -1 and are never encoded; the sign bit is what
    # the search and the mask pass test, and the encoding of a non-negative
    # radius never sets it
    r = np.array([0.0, 0.5, 7.0], np.float32)
    s = encode(r, np.array([1, 2, 255], np.uint32))
    assert np.all(np.signbit(s) == False)  # noqa: E712
