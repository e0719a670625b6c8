"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a hand-worked example,
a published generator vector, a closed form, an invariant of the algorithm or brute
force on tiny inputs.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_1412_1947_gb300 import synth
from tests.golden_io import arr, load


# ----------------------------------------------------------------------------------
# Worked example: every step of the method (Algorithm 1, §I, §V) on 10 points.
# ----------------------------------------------------------------------------------
def test_hand_example_every_step():
    g = load("hand_2d.txt")
    N, lk, fk, T = (int(v) for v in g["params"][0])
    raw = arr(g["raw"], np.float32)
    r = oracle.two_level(raw, N, lk, fk, T, seed=0, first_k=True)
    np.testing.assert_array_equal(r.scaled, arr(g["scaled"], np.float32))
    segs = [np.array([int(v) for v in row]) for row in g["segments"]]
    assert len(r.seg_off) - 1 == len(segs)
    for s, seg in enumerate(segs):
        np.testing.assert_array_equal(r.perm[r.seg_off[s]:r.seg_off[s + 1]], seg)
    np.testing.assert_array_equal(r.landmarks, arr(g["landmarks"], np.float32))
    np.testing.assert_array_equal(r.local_centers, arr(g["local_centers"]))
    np.testing.assert_array_equal(r.local_sse[:, -1], arr(g["local_sse_last"]))
    np.testing.assert_allclose(r.final_sse_hist, arr(g["final_sse_hist"]), rtol=1e-15, atol=0)
    np.testing.assert_array_equal(r.final_sse_hist[1:], arr(g["final_sse_hist"])[1:])
    np.testing.assert_array_equal(r.final_centers, arr(g["final_centers"]))
    np.testing.assert_array_equal(r.labels, arr(g["labels"]).astype(np.int32))
    assert r.sse == float(g["sse"][0][0])


def test_hand_example_round0_distances():
    g = load("hand_2d.txt")
    x = arr(g["scaled"], np.float32)
    # distances of round 0: the landmark is the origin after min-max scaling
    lab, best, _ = oracle.assign(x, np.zeros((1, 2)))
    np.testing.assert_array_equal(best, arr(g["round0_delta"]))


# ----------------------------------------------------------------------------------
# SplitMix64: the published first outputs from state 0 (Steele et al. 2014; the
# reference C implementation by Vigna).
# ----------------------------------------------------------------------------------
def test_splitmix64_published_vector():
    assert oracle.splitmix64(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_init_indices_is_a_partial_shuffle():
    for m, k in [(1, 1), (7, 7), (100, 10), (4096, 64), (5, 1)]:
        idx = oracle.init_indices(1234, 0, 3, m, k)
        assert len(set(idx.tolist())) == k and idx.min() >= 0 and idx.max() < m
    full = oracle.init_indices(99, 1, 0, 50, 50)
    assert sorted(full.tolist()) == list(range(50))
    a = oracle.init_indices(99, 0, 1, 1000, 16)
    b = oracle.init_indices(99, 0, 2, 1000, 16)
    c = oracle.init_indices(99, 1, 1, 1000, 16)
    assert not np.array_equal(a, b) and not np.array_equal(a, c)
    np.testing.assert_array_equal(a, oracle.init_indices(99, 0, 1, 1000, 16))


def test_init_indices_first_draw_closed_form():
    # step 0 swaps position 0 with r0 mod m, so the first index is r0 mod m where r0 is
    # the first output of the keyed stream
    seed, stage, seg, m = 0xABCDEF, 0, 5, 977
    st = oracle.lib().or_init_state(seed, stage, seg)
    r0 = oracle.splitmix64(st, 1)[0]
    assert oracle.init_indices(seed, stage, seg, m, 1)[0] == r0 % m


# ----------------------------------------------------------------------------------
# Feature scaling (Algorithm 1 step 1): closed form of min-max.
# ----------------------------------------------------------------------------------
def test_scale_closed_form():
    g = np.random.default_rng(1)
    raw = g.normal(size=(333, 5)).astype(np.float32) * 7 + 3
    raw[:, 2] = 4.5                         # a constant attribute
    raw[:, 3] = np.arange(333) * 0.25       # an exactly representable ramp
    s, mn, mx = oracle.scale(raw)
    for j in (0, 1, 4):
        assert s[:, j].min() == 0.0 and s[:, j].max() == 1.0
        assert np.all(np.argsort(raw[:, j], kind="stable") == np.argsort(s[:, j], kind="stable"))
    assert np.all(s[:, 2] == 0.0)
    np.testing.assert_array_equal(s[:, 3], (np.arange(333) / 332.0).astype(np.float32))
    np.testing.assert_array_equal(mn, raw.min(0).astype(np.float64))


# ----------------------------------------------------------------------------------
# The peel (Algorithm 1 steps 2-5).
# ----------------------------------------------------------------------------------
def _check_partition(perm, seg_off, n, N):
    assert sorted(perm.tolist()) == list(range(n))
    sizes = np.diff(seg_off)
    assert np.all(sizes[:-1] == N) and 1 <= sizes[-1] <= N
    for s in range(len(sizes)):
        seg = perm[seg_off[s]:seg_off[s + 1]]
        assert np.all(np.diff(seg) > 0)


def test_peel_one_dimension_is_sorting():
    # d = 1: L is the smallest remaining value, so every round takes the N smallest
    # values left; the segments are consecutive chunks of the (value, index) order.
    g = np.random.default_rng(2)
    x = g.integers(0, 40, size=(301, 1)).astype(np.float32) / 40  # many exact ties
    perm, seg_off, _ = oracle.peel(x, 25)
    order = np.lexsort((np.arange(301), x[:, 0]))
    _check_partition(perm, seg_off, 301, 25)
    for s in range(len(seg_off) - 1):
        np.testing.assert_array_equal(perm[seg_off[s]:seg_off[s + 1]],
                                      np.sort(order[seg_off[s]:seg_off[s + 1]]))


@pytest.mark.parametrize("n,d,N", [(500, 3, 37), (256, 8, 64), (1000, 2, 1000), (97, 5, 1),
                                   (64, 4, 200)])
def test_peel_invariants(n, d, N):
    x, _, _ = oracle.scale(synth.mixture(n, d, 4, seed=n + d))
    perm, seg_off, lm = oracle.peel(x, N)
    _check_partition(perm, seg_off, n, N)
    # after min-max scaling the first landmark is the origin
    assert np.all(lm[0] == 0.0)
    remaining = np.ones(n, bool)
    prev = None
    for s in range(len(seg_off) - 1):
        seg = perm[seg_off[s]:seg_off[s + 1]]
        rest = np.flatnonzero(remaining)
        # landmark = per-attribute minimum of what remains
        np.testing.assert_array_equal(lm[s], x[rest].min(0))
        if prev is not None:
            assert np.all(lm[s] >= prev)          # minima over shrinking sets never fall
        prev = lm[s]
        # selection: every chosen point precedes every remaining one in (distance, index)
        delta = ((x[rest].astype(np.float64) - lm[s].astype(np.float64)) ** 2).sum(1)
        key = dict(zip(rest.tolist(), delta.tolist()))
        chosen = set(seg.tolist())
        worst_in = max((key[i], i) for i in chosen)
        others = [(key[i], i) for i in rest if i not in chosen]
        if others:
            assert worst_in < min(others)
        remaining[seg] = False
    assert not remaining.any()


def test_peel_brute_force_tiny():
    # brute force: enumerate rounds with a full sort of all remaining points
    g = np.random.default_rng(3)
    for trial in range(20):
        n = int(g.integers(1, 13))
        d = int(g.integers(1, 4))
        N = int(g.integers(1, n + 2))
        x = (g.integers(0, 5, size=(n, d)) / 4).astype(np.float32)   # ties galore
        perm, seg_off, _ = oracle.peel(x, N)
        rem = list(range(n))
        out = []
        while rem:
            L = np.min(x[rem], axis=0)
            cand = sorted(rem, key=lambda i: (float(sum((float(x[i, j]) - float(L[j])) ** 2
                                                        for j in range(d))), i))
            out.append(sorted(cand[:N]))
            rem = sorted(cand[N:])
        assert [perm[seg_off[s]:seg_off[s + 1]].tolist() for s in range(len(seg_off) - 1)] == out


# ----------------------------------------------------------------------------------
# Lloyd (§I).
# ----------------------------------------------------------------------------------
def test_lloyd_sse_never_increases():
    x, _, _ = oracle.scale(synth.mixture(3000, 6, 9, seed=11))
    c0 = x[oracle.init_indices(5, 0, 0, 3000, 12)].astype(np.float64)
    _, _, hist, _, _, _ = oracle.lloyd(x, c0, 30)
    assert np.all(np.diff(hist) <= 1e-12 * hist[:-1])


def test_lloyd_fixed_point():
    # after convergence every point is with its nearest center and every center is the
    # mean of its points
    x, _, _ = oracle.scale(synth.mixture(800, 3, 5, sigma=0.3, seed=12))
    c0 = x[oracle.init_indices(8, 0, 0, 800, 5)].astype(np.float64)
    c, lab, hist, cnt, _, _ = oracle.lloyd(x, c0, 200)
    assert hist[-1] == hist[-2]
    dist = ((x[:, None, :].astype(np.float64) - c[None]) ** 2).sum(-1)
    np.testing.assert_array_equal(lab, dist.argmin(1))
    for j in range(5):
        if cnt[j]:
            np.testing.assert_allclose(c[j], x[lab == j].astype(np.float64).mean(0), rtol=0, atol=1e-15)


def test_lloyd_brute_force_optimum():
    # enumerate every partition of a tiny set: Lloyd's SSE is never below the optimum and
    # reaches it on separated blobs started with one center per blob
    g = np.random.default_rng(4)
    for trial in range(6):
        k = 2 + trial % 2
        m = 8
        means = g.uniform(0, 1, size=(k, 2)) * 10
        lab_true = np.arange(m) % k
        x = (means[lab_true] + g.normal(scale=0.05, size=(m, 2))).astype(np.float32)
        best = np.inf
        for assign in itertools.product(range(k), repeat=m):
            a = np.array(assign)
            sse = 0.0
            for j in range(k):
                if np.any(a == j):
                    p = x[a == j].astype(np.float64)
                    sse += ((p - p.mean(0)) ** 2).sum()
            best = min(best, sse)
        c0 = x[:k].astype(np.float64)                 # points 0..k-1 are in distinct blobs
        c, lab, hist, _, _, _ = oracle.lloyd(x, c0, 10)
        assert hist[-1] >= best * (1 - 1e-12)
        assert abs(hist[-1] - best) <= 1e-12 * max(best, 1e-300) + 1e-15
        rand = x[[0, 1] + [k] * (k - 2)][:k].astype(np.float64)
        _, _, h2, _, _, _ = oracle.lloyd(x, rand, 10)
        assert h2[-1] >= best * (1 - 1e-12)


def test_lloyd_ties_and_empty_clusters():
    x = np.array([[0, 0], [1, 0], [0, 1]], np.float32)
    # two identical centers: every point goes to the lower index, the other one is empty
    c0 = np.array([[5, 5], [5, 5], [9, 9]], np.float64)
    c, lab, _, cnt, _, _ = oracle.lloyd(x, c0, 1)
    np.testing.assert_array_equal(lab, [0, 0, 0])
    np.testing.assert_array_equal(cnt, [3, 0, 0])
    np.testing.assert_array_equal(c[1], [5, 5])        # empty: keeps its center
    np.testing.assert_array_equal(c[2], [9, 9])
    np.testing.assert_allclose(c[0], [1 / 3, 1 / 3], rtol=0, atol=1e-16)


def test_local_k_one_gives_subcluster_means():
    raw = synth.mixture(1000, 4, 6, seed=21)
    r = oracle.two_level(raw, 128, 1, 2, 5, seed=3)
    packed = r.scaled[r.perm].astype(np.float64)
    for s in range(len(r.seg_off) - 1):
        np.testing.assert_allclose(r.local_centers[s], packed[r.seg_off[s]:r.seg_off[s + 1]].mean(0),
                                   rtol=0, atol=1e-15)


def test_two_level_reduces_to_standard_kmeans():
    # one subcluster holding every point and one local center per point: the pooled set
    # is the data itself (reordered) and the final Lloyd is plain Lloyd on all points
    raw = synth.mixture(300, 3, 4, seed=31)
    n, k, T, seed = 300, 4, 15, 77
    r = oracle.two_level(raw, n, n, k, T, seed=seed)
    pooled = r.local_centers.astype(np.float32)
    assert sorted(map(tuple, pooled.tolist())) == sorted(map(tuple, r.scaled.tolist()))
    init = pooled[oracle.init_indices(seed, 1, 0, n, k)].astype(np.float64)
    # against the separately written one-level k-means (numpy), not the oracle's own Lloyd
    c, lab, hist = oracle.standard_kmeans(r.scaled, init, T)
    np.testing.assert_allclose(r.final_centers, c, rtol=0, atol=1e-14)
    np.testing.assert_allclose(r.final_sse_hist, hist, rtol=1e-13, atol=0)


def test_standard_kmeans_on_a_hand_worked_case():
    # four points on a line, two centers: assignments and means by hand
    x = np.array([[0.0], [1.0], [9.0], [10.0]])
    c, lab, hist = oracle.standard_kmeans(x, np.array([[0.0], [1.0]]), 2)
    # iteration 1: {0} -> 0, {1, 9, 10} -> 1 (mean 20/3); iteration 2: {0, 1} -> 0 (0.5),
    # {9, 10} -> 1 (9.5)
    np.testing.assert_array_equal(lab, [0, 0, 1, 1])
    np.testing.assert_allclose(c, [[0.5], [9.5]])
    np.testing.assert_allclose(hist, [(1 - 20 / 3) ** 2 + (9 - 20 / 3) ** 2 + (10 - 20 / 3) ** 2, 4 * 0.25])


def test_two_level_one_iteration_matches_vectorised_lloyd():
    raw = synth.mixture(2000, 5, 8, seed=41)
    r = oracle.two_level(raw, 250, 16, 8, 1, seed=9)
    packed = r.scaled[r.perm].astype(np.float64)
    for s in range(len(r.seg_off) - 1):
        p = packed[r.seg_off[s]:r.seg_off[s + 1]]
        init = p[oracle.init_indices(9, 0, s, len(p), 16)]
        lab = ((p[:, None, :] - init[None]) ** 2).sum(-1).argmin(1)
        exp = np.stack([p[lab == j].mean(0) if np.any(lab == j) else init[j] for j in range(16)])
        got = r.local_centers[s * 16:(s + 1) * 16]
        np.testing.assert_allclose(got, exp, rtol=0, atol=1e-14)


def test_replay_follows_only_near_ties():
    x, _, _ = oracle.scale(synth.mixture(500, 3, 4, seed=51))
    c0 = x[:4].astype(np.float64)
    _, lab, _, _, _, _ = oracle.lloyd(x, c0, 1)
    # its own labels: nothing forced, nothing bad
    *_, nf, nb = oracle.lloyd(x, c0, 1, force=lab[None, :], tie_tol=1e-5)
    assert (nf, nb) == (0, 0)
    # a clearly wrong label is reported, not followed
    bad = lab.copy()
    bad[7] = (bad[7] + 1) % 4
    *_, nf, nb = oracle.lloyd(x, c0, 1, force=bad[None, :], tie_tol=1e-5)
    assert (nf, nb) == (0, 1)
    # an exact tie: a duplicated center, the other side picked the higher index
    cdup = np.vstack([c0, c0[2:3]])
    _, lab2, _, _, _, _ = oracle.lloyd(x, cdup, 1)
    f = lab2.copy()
    f[lab2 == 2] = 4
    *_, nf, nb = oracle.lloyd(x, cdup, 1, force=f[None, :], tie_tol=1e-5)
    assert nb == 0 and nf == int((lab2 == 2).sum()) > 0


@pytest.mark.parametrize("n,d,N,grid", [(2000, 3, 128, 0), (3001, 2, 97, 6), (1024, 8, 1, 0), (777, 4, 1000, 0),
                                        (5000, 1, 333, 4), (4096, 16, 256, 0)])
def test_select_peel_equals_sorted_peel(n, d, N, grid):
    # the O(n_r) selection form of the peel is the same function as the sort form,
    # ties included (grid > 0: coordinates on a coarse grid, thousands of equal distances)
    g = np.random.default_rng(n + d)
    if grid:
        raw = g.integers(0, grid, size=(n, d)).astype(np.float32)
    else:
        raw = synth.mixture(n, d, 5, outlier_frac=0.01, seed=n)
    x, _, _ = oracle.scale(raw)
    a = oracle.peel(x, N)
    b = oracle.peel(x, N, select=True)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


def test_two_level_select_peel_flag_changes_nothing():
    raw = synth.mixture(3000, 4, 6, outlier_frac=0.01, seed=61)
    a = oracle.two_level(raw, 256, 8, 5, 4, seed=2)
    b = oracle.two_level(raw, 256, 8, 5, 4, seed=2, select_peel=True)
    np.testing.assert_array_equal(a.perm, b.perm)
    np.testing.assert_array_equal(a.final_centers, b.final_centers)
    assert a.sse == b.sse


# ---------------------------------------------------------------- Algorithm 2 grouping
def test_unequal_grouping_1d_closed_form():
    # data spanning [0, 1]: 4 landmarks at 1/8, 3/8, 5/8, 7/8, a point x joins landmark
    # ceil(4x) - 1 (0 for x = 0); x = 1/4, 1/2, 3/4 lie exactly between two landmarks and
    # join the lower one
    xs = np.array([0, 1, 0.25, 0.5, 0.75, 0.1, 0.3, 0.6, 0.9, 0.2499, 0.2501, 0.125, 0.5, 0.75],
                  np.float32)[:, None]
    perm, off, lm, g = oracle.group_unequal(xs, 4)
    np.testing.assert_array_equal(lm[:, 0], np.array([0.125, 0.375, 0.625, 0.875], np.float32))
    expect = np.maximum(np.ceil(xs[:, 0].astype(np.float64) * 4) - 1, 0).astype(np.int32)
    np.testing.assert_array_equal(g, expect)
    # groups in landmark order, ascending index inside each
    sizes = np.bincount(expect, minlength=4)
    np.testing.assert_array_equal(np.diff(off), sizes[sizes > 0])
    for s in range(len(off) - 1):
        seg = perm[off[s]:off[s + 1]]
        assert np.all(np.diff(seg) > 0) and len(set(expect[seg])) == 1


def test_unequal_landmarks_lie_on_the_segment_from_L_to_H():
    # L = (0, 3, -2), H = (1, 3, 6): the constant attribute stays 3 on every landmark
    x = np.array([[0, 3, 6], [1, 3, -2], [0.5, 3, 0], [0.2, 3, 1]], np.float32)
    _, _, lm, _ = oracle.group_unequal(x, 5)
    for i in range(5):
        t = (i + 0.5) / 5
        np.testing.assert_array_equal(lm[i], np.array([t, 3, -2 + 8 * t], np.float32))


def test_unequal_empty_groups_are_skipped_and_m1_is_one_group():
    rng = np.random.default_rng(4)
    x = np.concatenate([rng.uniform(0, 0.05, (50, 2)), rng.uniform(0.95, 1.0, (50, 2))]).astype(np.float32)
    perm, off, _, g = oracle.group_unequal(x, 10)
    assert len(off) - 1 == len(np.unique(g)) < 10 and np.all(np.diff(off) > 0)
    assert sorted(perm.tolist()) == list(range(100))
    perm1, off1, _, g1 = oracle.group_unequal(x, 1)
    np.testing.assert_array_equal(perm1, np.arange(100))
    np.testing.assert_array_equal(off1, [0, 100])
    assert not g1.any()


def test_unequal_two_level_uses_the_grouping():
    raw = synth.mixture(600, 3, 4, outlier_frac=0.05, seed=77)
    o = oracle.two_level(raw, 0, 4, 3, 5, 9, unequal_m=12)
    perm, off, _, _ = oracle.group_unequal(o.scaled, 12)
    np.testing.assert_array_equal(o.perm, perm)
    np.testing.assert_array_equal(o.seg_off, off)
    assert o.local_centers.shape[0] == sum(min(4, int(v)) for v in np.diff(off))


# ---------------------------------------------------------------- bfloat16 storage
def test_bf16_storage_rounds_once_to_nearest_even():
    # raw [0, 512, 257, 259, 384, 171]: scaled = v / 512 exactly, then 8 significant bits:
    #   257/512 = 0.5 + 2^-9, halfway between 0.5 and 0.5 + 2^-8 -> 0.5 (even)
    #   259/512 = 0.5 + 1.5 * 2^-8, halfway -> 0.5 + 2^-7 (even)
    #   384/512 = 0.75 exact; 171/512 = 0.333984375 exact (0x3EAB)
    raw = np.array([[0.0], [512.0], [257.0], [259.0], [384.0], [171.0]], np.float32)
    xs, _, _ = oracle.scale(raw, bf16=True)
    np.testing.assert_array_equal(xs[:, 0], np.array([0, 1, 0.5, 0.5078125, 0.75, 0.333984375], np.float32))
    # 1/3 from [0, 3]: 1.0101010101..b x 2^-2, the bit after the 8th is 1 with more set bits
    # after it -> rounds up to 1.0101011b x 2^-2 = 0.333984375
    xs2, _, _ = oracle.scale(np.array([[0.0], [3.0], [1.0]], np.float32), bf16=True)
    assert xs2[2, 0] == np.float32(0.333984375)
    # float32 storage keeps 24 bits
    xs3, _, _ = oracle.scale(np.array([[0.0], [3.0], [1.0]], np.float32))
    assert xs3[2, 0] == np.float32(1.0 / 3.0)


# ----------------------------------------------------------------------------------
# Count-weighted pooled Lloyd (the abstract: the second level clusters the subclusters'
# means; weighing each local center by its cluster's size makes those the weighted means).
# ----------------------------------------------------------------------------------
def test_weighted_lloyd_with_unit_weights_is_plain_lloyd():
    x, _, _ = oracle.scale(synth.mixture(600, 4, 6, seed=31))
    c0 = x[:7].astype(np.float64)
    a = oracle.lloyd(x, c0, 9)
    b = oracle.lloyd(x, c0, 9, weights=np.ones(600, np.int64))
    for u, v in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(u, v)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_weighted_lloyd_equals_lloyd_on_the_replicated_multiset(seed):
    # integer weights w_p: Lloyd on the multiset holding point p w_p times (zero: absent)
    # moves the centers identically, its labels are the weighted run's labels repeated,
    # and its SSE is the weighted SSE
    rng = np.random.default_rng(seed)
    x, _, _ = oracle.scale(synth.mixture(120, 3, 5, seed=40 + seed))
    w = rng.integers(0, 5, size=120).astype(np.int64)
    w[:6] = 1 + np.arange(6)                        # the initial centers carry weight
    c0 = x[:6].astype(np.float64)
    cw, lw, hw, _, _, _ = oracle.lloyd(x, c0, 12, weights=w)
    xr = np.repeat(x, w, axis=0)
    cr, lr, hr, _, _, _ = oracle.lloyd(xr, c0, 12)
    np.testing.assert_allclose(cw, cr, rtol=0, atol=1e-14)
    np.testing.assert_array_equal(np.repeat(lw, w), lr)
    np.testing.assert_allclose(hw, hr, rtol=1e-13, atol=0)


def test_pooled_weights_are_the_local_cluster_sizes():
    # the two-level run with pool_weighted: its final centers are those of plain Lloyd on
    # the pooled local centers, each repeated as often as its cluster has members in the
    # last local iteration (first-k init, so both runs start from the same centers)
    raw = synth.mixture(3000, 3, 8, seed=51)
    N, lk, fk, T = 400, 12, 6, 8
    r = oracle.two_level(raw, N, lk, fk, T, seed=0, first_k=True, pool_weighted=True)
    sizes = np.concatenate([np.bincount(r.local_labels[r.seg_off[s]:r.seg_off[s + 1]], minlength=r.local_k_eff[s])
                            for s in range(len(r.seg_off) - 1)])
    assert sizes.sum() == 3000 and len(sizes) == len(r.local_centers)
    pool = r.local_centers.astype(np.float32)
    cr, _, _, _, _, _ = oracle.lloyd(np.repeat(pool, sizes, axis=0), pool[:fk].astype(np.float64), T)
    np.testing.assert_allclose(r.final_centers, cr, rtol=0, atol=1e-14)
    u = oracle.two_level(raw, N, lk, fk, T, seed=0, first_k=True)
    np.testing.assert_array_equal(u.local_centers, r.local_centers)       # the first level is unchanged
    assert np.abs(u.final_centers - r.final_centers).max() > 1e-6        # the weights do act
