"""The exact centroid sums (the update step of Lloyd's algorithm, §I) add each scaled
coordinate v in [0, 1] as the integer rne(v 2^32) (32.32 fixed point, ties to even).  The
kernels form it with two 32-bit conversions: s = v 2^16 (exact), hi = floor(s), and
lo = rne((s - hi) 2^16), the fraction and its product being exact in float32, so that
hi 2^16 + lo = rne(v 2^32).  This restates those float32 steps in numpy and checks them
against the definition on every float32 of a binade sample, the ends of the range and
values whose product lies exactly half-way (an exhaustive run over all 2^30 float32 values
in [0, 1] found no difference either)."""
import numpy as np


def fix_parts(v):
    v = np.asarray(v, np.float32)
    s = v * np.float32(65536.0)
    hi = np.floor(s).astype(np.uint64)
    lo = np.rint((s - hi.astype(np.float32)) * np.float32(65536.0)).astype(np.uint64)
    return hi, lo


def _check(v):
    hi, lo = fix_parts(v)
    ref = np.rint(np.asarray(v, np.float32).astype(np.float64) * 2.0 ** 32).astype(np.uint64)
    np.testing.assert_array_equal((hi << np.uint64(16)) + lo, ref)
    assert lo.max() <= 65536          # the halves stay within 32 bits over 32768 rows


def test_every_float_of_sampled_binades():
    for e in (-149, -126, -40, -33, -32, -31, -17, -9, -8, -1):
        lo_bits = np.float32(2.0 ** e).view(np.uint32)
        bits = np.arange(int(lo_bits), int(lo_bits) + (1 << 20), dtype=np.uint32)
        _check(bits.view(np.float32))


def test_ends_and_half_way_products():
    ends = np.array([0.0, 1.0, np.nextafter(np.float32(1), np.float32(0)), np.float32(2.0 ** -149),
                     np.float32(2.0 ** -33), np.float32(3 * 2.0 ** -34)], np.float32)
    _check(ends)
    # m 2^-33 with m odd: v 2^32 = m / 2 lies half-way between two integers
    m = np.arange(1, 1 << 20, 2, dtype=np.float64)
    _check((m * 2.0 ** -33).astype(np.float32))


def test_random_values():
    g = np.random.default_rng(3)
    _check(g.random(1 << 22, dtype=np.float32))
