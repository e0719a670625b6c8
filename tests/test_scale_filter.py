"""The float-float filter of the scaling kernel, restated on the CPU: where it decides, its
value must equal the float64 definition (the oracle's min-max scaling) bit for bit.

The kernel computes RN_T((double(x) - mn) * inv), inv = RN(1/range), without float64
arithmetic for most values: x - mn = s + e exactly (TwoSum), the product with inv = ih + il
in float-float (s*ih = p + pe exactly, as the FMA gives it), and the T value nearest
z = zh + zl is taken when z is farther than the product's error bound from every rounding
midpoint of T (a margin of 2^-16 of a half-spacing for float32, 2^-12 for bfloat16).  The
steps below are the kernel's float32 operations, each rounded once (numpy float32), and
the exact FMA residual taken from float64 (the 48-bit product is exact there)."""
import numpy as np
import pytest

import oracle

F, D = np.float32, np.float64


def _filter(x, mn, inv, bf16, drop_il=False, bf16_margin=2.0 ** -12):
    """(decided mask, value) of the kernel's float-float path; x is (n, d) float32, mn and
    inv are per attribute (float64)."""
    ok_attr = (inv >= 2.0 ** -60) & (inv <= 2.0 ** 60)
    ih = np.where(ok_attr, inv.astype(F), F(0))
    il = np.where(ok_attr, (inv - ih.astype(D)).astype(F), F(0))
    if drop_il:
        il = np.zeros_like(il)
    mnf = mn.astype(F)
    with np.errstate(all="ignore"):
        s = x - mnf
        bb = s - x
        e = (x - (s - bb)) + (-mnf - bb)
        p = s * ih
        pe = (s.astype(D) * ih.astype(D) - p.astype(D)).astype(F)
        t = pe + (s * il + e * ih)
        zh = p + t
        zl = t - (zh - p)
        rng = (zh >= F(2.0 ** -90)) & (zh < F(2.0 ** 100))
        b = zh.view(np.uint32).astype(np.int64)
        if not bf16:
            hs = (((b >> 23) - 24).clip(1) << 23).astype(np.uint32).view(F)
            hs = np.where((b & 0x7FFFFF) == 0, hs * F(0.5), hs)
            dec = rng & (np.abs(zl) <= hs - hs * F(2.0 ** -16))
            val = zh
        else:
            cb = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
            c = cb.view(F)
            u = (zh - c) + zl
            hs = ((((cb.astype(np.int64) >> 23) - 8).clip(1)) << 23).astype(np.uint32).view(F)
            hs = np.where((cb & 0x7FFFFF) == 0, hs * F(0.5), hs)
            dec = rng & (np.abs(u) <= hs - hs * F(bf16_margin))
            val = c
    zero = s == 0
    return dec | zero, np.where(zero, F(0), val)


def _matrix(seed, n=8192, d=256):
    """Attributes of every scale (minimum and range from 2^-40 to 2^40, both signs), rows 0
    and 1 their minimum and maximum, then values spread over the range, a few ulps above the
    minimum and below the maximum."""
    rng = np.random.default_rng(seed)
    mn = ((rng.random(d) * 2 - 1) * 2.0 ** rng.integers(-40, 41, d)).astype(F)
    mn[: d // 8] = 0
    mx = (mn.astype(D) + (rng.random(d) + 0.5) * 2.0 ** rng.integers(-40, 41, d)).astype(F)
    mx = np.where(mx > mn, mx, np.nextafter(mn, F(np.inf)))
    x = (mn.astype(D) + rng.random((n, d)) * (mx.astype(D) - mn.astype(D))).astype(F)
    k = n // 8
    x[2:k] = (mn.view(np.uint32) + rng.integers(0, 64, (k - 2, d)).astype(np.uint32)).view(F)
    x[k:2 * k] = (mx.view(np.uint32) - rng.integers(0, 64, (k, d)).astype(np.uint32)).view(F)
    x = np.clip(x, mn, mx)
    x[0], x[1] = mn, mx
    return np.ascontiguousarray(x)


def _reference(x, bf16):
    exp, mn, mx = oracle.scale(x, bf16=bf16)
    rng = mx - mn
    inv = np.where(rng > 0, 1.0 / np.where(rng > 0, rng, 1.0), 0.0)
    return exp, mn, inv


@pytest.mark.parametrize("bf16", [False, True])
def test_filter_decisions_equal_the_float64_definition(bf16):
    x = _matrix(1234 + bf16)
    exp, mn, inv = _reference(x, bf16)
    dec, val = _filter(x, mn, inv, bf16)
    live = inv > 0
    dec &= live
    assert dec.mean() > 0.95                   # the float64 fallback stays rare
    np.testing.assert_array_equal(val[dec].view(np.uint32), exp[dec].view(np.uint32))


def test_planted_mistakes_are_caught():
    """The comparison above has teeth: dropping the low part of 1/range, or a bfloat16 margin
    on the wrong side of the half-spacing, gives values that differ from the definition."""
    x = _matrix(99)
    exp, mn, inv = _reference(x, False)
    dec, val = _filter(x, mn, inv, False, drop_il=True)
    assert np.any(val[dec].view(np.uint32) != exp[dec].view(np.uint32))
    exp, mn, inv = _reference(x, True)
    dec, val = _filter(x, mn, inv, True, bf16_margin=-2.0 ** -4)
    assert np.any(val[dec].view(np.uint32) != exp[dec].view(np.uint32))
