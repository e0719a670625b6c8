"""The CUDA peel's epoch scheme restated on the CPU and checked against the oracle's peel.

The kernel computes the landmark distances once per epoch and lets them serve up to K
rounds: with the same landmark, round r+1 takes the next N points of the same order by
(distance, index) (Algorithm 1 steps 2-5, repeated on the points left out as §II
describes).  An epoch commits its rounds up to the first one after which some attribute
has no remaining point holding its landmark value (the only way the per-attribute minimum
L can change), counting holders per attribute exactly as the kernel does: live holders
counted when the distances are computed, holders per tentative round counted when the
rounds are assigned.  This file restates that bookkeeping (exact float64 distances, so
only the scheme is under test, not the float32 filter) and checks that it gives the
oracle's partition bit for bit, including inputs with heavy ties in values and distances.
"""
import numpy as np
import pytest

import oracle
from paper_1412_1947_gb300 import synth


def _delta64(x, L):
    acc = np.zeros(len(x), np.float64)
    for j in range(x.shape[1]):
        t = x[:, j].astype(np.float64) - np.float64(L[j])
        acc = acc + t * t
    return acc


def epoch_peel(x, N, K, stats=None, predict=False):
    """The kernel's epoch bookkeeping in plain numpy; returns (perm, seg_off).  With
    predict, an epoch resolves only the rounds up to the one in which the last holder of
    some attribute's landmark value leaves at the latest: m = the smallest over the
    attributes of their holders' largest distance (taken at the pass), c = the live
    distances <= m, the last round (c - 1) // N (the kernel reads c off its histograms,
    an upper bound of the same kind)."""
    n, d = x.shape
    rnd = np.full(n, -1, np.int64)
    live = np.ones(n, bool)
    L = x.min(axis=0)                     # the first landmark (0 for scaled data)
    r0, passes, epochs, short = 0, 0, 0, 0
    need_keys = True
    chold = None
    delta = None
    hmax = None
    while True:
        ids = np.flatnonzero(live)
        if len(ids) <= N:
            rnd[ids] = r0
            break
        Ke = min(K, -(-len(ids) // N) - 1)
        if need_keys:
            delta = _delta64(x, L)
            chold = (x[ids] == L[None, :]).sum(axis=0)      # live holders per attribute
            held = x[ids] == L[None, :]
            hmax = np.array([delta[ids][held[:, j]].max() if held[:, j].any() else 0.0 for j in range(d)])
            passes += 1
        cap = Ke
        if predict:
            c = int(np.sum(delta[ids] <= hmax.min()))
            Ke = min(Ke, (max(c, 1) - 1) // N + 1)
        epochs += 1
        order = ids[np.lexsort((ids, delta[ids]))]
        tent = {}
        for q in range(Ke):
            for i in order[q * N:(q + 1) * N]:
                tent[int(i)] = q
        hcnt = np.zeros((d, Ke), np.int64)
        for i, q in tent.items():
            hcnt[:, q] += x[i] == L
        # q* = the first round after which some attribute has no holder left
        qs = Ke
        for j in range(d):
            acc = np.cumsum(hcnt[j])
            hit = np.flatnonzero(acc >= chold[j])
            if len(hit):
                qs = min(qs, int(hit[0]))
        kcommit = qs + 1 if qs < Ke else Ke
        changed = qs < Ke
        for i, q in tent.items():
            if q < kcommit:
                rnd[i] = r0 + q
                live[i] = False
        if changed:
            L = x[live].min(axis=0)
        else:
            chold = chold - hcnt[:, :kcommit].sum(axis=1)
            short += Ke < cap          # an epoch the prediction cut before the landmark changed
        need_keys = changed
        r0 += kcommit
    S = r0 + 1
    perm = np.lexsort((np.arange(n), rnd))          # by round, ascending index inside
    seg_off = np.array([np.sum(rnd < r) for r in range(S + 1)], np.int64)
    if stats is not None:
        stats.update(passes=passes, epochs=epochs, rounds=S, short=short)
    return perm, seg_off


def _check(raw, N, K):
    x, _, _ = oracle.scale(raw)
    perm, off = epoch_peel(x, N, K)
    operm, ooff, _ = oracle.peel(x, N)
    np.testing.assert_array_equal(off, ooff)
    np.testing.assert_array_equal(perm, operm)


@pytest.mark.parametrize("K", [1, 2, 3, 8, 16])
def test_epochs_equal_the_per_round_peel(K):
    raw = synth.mixture(3000, 4, 6, outlier_frac=0.02, seed=4242)
    _check(raw, 97, K)


@pytest.mark.parametrize("K", [1, 4, 16])
def test_epochs_with_tied_values_and_distances(K):
    # a coarse integer grid: many points share each attribute's minimum (several holders)
    # and thousands share each distance (ties decided by index)
    g = np.random.default_rng(9)
    raw = g.integers(0, 5, size=(2500, 3)).astype(np.float32)
    _check(raw, 64, K)


def test_epochs_with_a_constant_attribute():
    # every point holds the constant attribute's minimum: it never ends an epoch
    g = np.random.default_rng(10)
    raw = g.normal(size=(1200, 3)).astype(np.float32)
    raw[:, 1] = 2.5
    _check(raw, 50, 8)


def test_epochs_on_the_worked_example():
    # the hand-worked example: rounds 0 and 1 share the landmark (0, 0), so one epoch
    # (one pass of distances) serves both, and round 2 takes the two points left
    from tests.golden_io import arr, load
    g = load("hand_2d.txt")
    raw = arr(g["raw"], np.float32)
    x, _, _ = oracle.scale(raw)
    st = {}
    perm, off = epoch_peel(x, 4, 8, st)
    np.testing.assert_array_equal(perm, [0, 1, 2, 3, 5, 7, 8, 9, 4, 6])
    np.testing.assert_array_equal(off, [0, 4, 8, 10])
    assert st["passes"] == 1 and st["epochs"] == 1


def test_epochs_save_distance_passes_on_the_headline_shape():
    # the headline recipe at 1/16 size: far fewer distance passes than rounds
    raw = synth.mixture(65536, 16, 64, outlier_frac=0.01, seed=synth.BASE_SEED + 1)
    x, _, _ = oracle.scale(raw)
    st = {}
    perm, off = epoch_peel(x, 4096, 8, st)
    operm, ooff, _ = oracle.peel(x, 4096)
    np.testing.assert_array_equal(perm, operm)
    assert st["passes"] < st["rounds"]


@pytest.mark.parametrize("K", [2, 8, 32])
def test_predicted_epochs_equal_the_per_round_peel(K):
    raw = synth.mixture(3000, 4, 6, outlier_frac=0.02, seed=4243)
    x, _, _ = oracle.scale(raw)
    perm, off = epoch_peel(x, 97, K, predict=True)
    operm, ooff, _ = oracle.peel(x, 97)
    np.testing.assert_array_equal(off, ooff)
    np.testing.assert_array_equal(perm, operm)


def test_predicted_epochs_with_tied_values_and_distances():
    g = np.random.default_rng(11)
    raw = g.integers(0, 5, size=(2500, 3)).astype(np.float32)
    x, _, _ = oracle.scale(raw)
    perm, off = epoch_peel(x, 64, 32, predict=True)
    operm, ooff, _ = oracle.peel(x, 64)
    np.testing.assert_array_equal(off, ooff)
    np.testing.assert_array_equal(perm, operm)


def test_the_prediction_never_cuts_an_epoch_short():
    # in exact arithmetic the predicted last round is at or after the round in which the
    # landmark changes, so every epoch ends with a change or with its cap: one epoch per
    # landmark whenever no landmark serves more rounds than the cap
    raw = synth.mixture(65536, 16, 64, outlier_frac=0.01, seed=synth.BASE_SEED + 1)
    x, _, _ = oracle.scale(raw)
    st = {}
    perm, off = epoch_peel(x, 4096, 32, st, predict=True)
    operm, ooff, _ = oracle.peel(x, 4096)
    np.testing.assert_array_equal(perm, operm)
    assert st["short"] == 0
    assert st["epochs"] == st["passes"]
