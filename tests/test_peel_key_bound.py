"""The peel's float32 landmark keys and their error bound (Algorithm 1 step 2, Eq. 1 distances
in float64 as the definition), checked on the CPU with the kernel's arithmetic emulated.

A full pass keys a point by the float32 FMA chain acc = RN(RN(x_j - L_j)^2 + acc) over
ascending attributes, within eps0 = (d+4) 2^-23 (relative) and ea0 = 2^-120 of the float64
distance.  After a landmark change in a few attributes J the kernel instead adds the change
of the squared distance, sum_J (l_j - o_j)(l_j + o_j - 2 x_j), as an FMA chain in float32
(o_j old, l_j new value), clamps at 0, and carries the bound as
    eps' = eps + 2^-23,   ea' = ea + (5 eps + (16 + 4|J|) 2^-24) sum_J (l_j - o_j).
Here every key of a run of such updates must stay within eps*key + ea of the float64
distance to the current landmark, on data shaped like the peel's inputs (min-max scaled
mixtures) and on adversarial ones (large jumps, values crowding the landmark).  A float32
FMA is emulated as one rounding of the exact double product plus the addend, exact except
for rare double roundings of 2^-53 relative, far inside the bound's margins."""
import numpy as np
import pytest

U = 2.0 ** -24


def fma32(a, b, c):
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


def full_keys(x, L):
    acc = np.zeros(len(x), np.float32)
    for j in range(x.shape[1]):
        t = (x[:, j] - L[j]).astype(np.float32)
        acc = fma32(t, t, acc)
    return acc


def delta64(x, L):
    s = np.zeros(len(x), np.float64)
    for j in range(x.shape[1]):
        diff = x[:, j].astype(np.float64) - np.float64(L[j])
        s = s + diff * diff
    return s


def update_keys(keys, x, J, old, new):
    acc = np.zeros(len(x), np.float32)
    for j, o, l in zip(J, old, new):
        c = np.float32(np.float32(l) - np.float32(o))
        sm = np.float32(np.float32(l) + np.float32(o))
        inner = fma32(np.full(len(x), -2.0, np.float32), x[:, j], np.full(len(x), sm, np.float32))
        acc = fma32(np.full(len(x), c, np.float32), inner, acc)
    k = (keys + acc).astype(np.float32)
    return np.where(k > 0, k, np.float32(0.0))


def carried(eps, ea, J, old, new):
    cs = float(sum(float(np.float32(np.float32(l) - np.float32(o))) for o, l in zip(old, new)))
    return eps + 2.0 ** -23, ea + (5.0 * eps + (16.0 + 4.0 * len(J)) * U) * cs * (1.0 + 2.0 ** -20)


def scaled_mixture(rng, n, d, blobs):
    c = rng.normal(size=(blobs, d)) * 3.0
    x = c[rng.integers(0, blobs, n)] + rng.normal(size=(n, d)) * rng.uniform(0.2, 1.0, (n, 1))
    mn, mx = x.min(0), x.max(0)
    return ((x - mn) / (mx - mn)).astype(np.float32)


def check_chain(x, rng, steps, max_moved, jump):
    n, d = x.shape
    L = x.min(0).astype(np.float32)
    keys = full_keys(x, L)
    eps, ea = (d + 4) * 2.0 ** -23, 2.0 ** -120
    worst = 0.0
    for _ in range(steps):
        ref = delta64(x, L)
        bound = eps * keys.astype(np.float64) + ea
        err = np.abs(keys.astype(np.float64) - ref)
        assert np.all(err <= bound), (float((err - bound).max()), eps, ea)
        worst = max(worst, float((err / np.maximum(bound, 1e-300)).max()))
        J = np.sort(rng.choice(d, rng.integers(1, max_moved + 1), replace=False))
        old = L[J].copy()
        new = np.minimum(np.float32(1.0), old + jump(rng, len(J))).astype(np.float32)
        keys = update_keys(keys, x, J, old, new)
        eps, ea = carried(eps, ea, J, old, new)
        L[J] = new
    return worst


@pytest.mark.parametrize("d", [4, 16, 64])
def test_updates_stay_within_the_carried_bound(d):
    rng = np.random.default_rng(11 + d)
    x = scaled_mixture(rng, 6000, d, 24)
    # small moves, as a landmark's next holder value: the regime the kernel updates in
    worst = check_chain(x, rng, steps=(d + 4) // 2, max_moved=3,
                        jump=lambda r, m: r.exponential(1e-3, m).astype(np.float32))
    assert worst <= 1.0


@pytest.mark.parametrize("d", [8, 32])
def test_large_jumps_and_points_at_the_landmark(d):
    # jumps up to half the range, and a third of the points sharing coordinates with the
    # landmark path (keys that cancel to 0 or near it)
    rng = np.random.default_rng(5 + d)
    x = scaled_mixture(rng, 4000, d, 8)
    x[rng.choice(len(x), len(x) // 3, replace=False)] = x.min(0)
    x[:50] = np.float32(1.0)
    worst = check_chain(x, rng, steps=12, max_moved=8,
                        jump=lambda r, m: r.uniform(0.0, 0.5, m).astype(np.float32))
    assert worst <= 1.0


def test_the_bound_is_not_vacuous():
    # the emulated update does err: some keys differ from the float64 distance after a
    # chain of updates, by more than a plain recomputation would (the carried terms matter)
    rng = np.random.default_rng(3)
    x = scaled_mixture(rng, 6000, 16, 24)
    L = x.min(0).astype(np.float32)
    keys = full_keys(x, L)
    for _ in range(8):
        J = np.sort(rng.choice(16, 2, replace=False))
        new = np.minimum(np.float32(1.0), L[J] + np.float32(0.01)).astype(np.float32)
        keys = update_keys(keys, x, J, L[J].copy(), new)
        L[J] = new
    err = np.abs(keys.astype(np.float64) - delta64(x, L))
    assert err.max() > 0.0
    fresh = np.abs(full_keys(x, L).astype(np.float64) - delta64(x, L))
    assert err.max() >= fresh.max()


@pytest.mark.parametrize("d", [16, 64])
def test_cancellation_needs_the_carried_absolute_term(d):
    # points far from the landmark in attribute 0 only, where the landmark then jumps: the
    # new keys are tiny differences of large old ones, whose rounding error is only covered
    # by the carried absolute term (a relative bound on the new key alone fails here)
    rng = np.random.default_rng(17 + d)
    n = 4000
    x = (rng.random((n, d)) * 1e-3).astype(np.float32)
    x[:, 0] = (0.75 + rng.random(n) * 1e-3).astype(np.float32)
    x[0] = 0.0
    L = x.min(0).astype(np.float32)
    keys = full_keys(x, L)
    eps, ea = (d + 4) * 2.0 ** -23, 2.0 ** -120
    J = np.array([0])
    old, new = L[J].copy(), np.array([0.75], np.float32)
    keys = update_keys(keys, x, J, old, new)
    L[J] = new
    err = np.abs(keys.astype(np.float64) - delta64(x, L))
    ne, na = carried(eps, ea, J, old, new)
    assert np.all(err <= ne * keys.astype(np.float64) + na)
    assert np.any(err > ne * keys.astype(np.float64) + ea)
