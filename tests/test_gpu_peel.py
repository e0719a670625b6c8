"""The peel's partition (Algorithm 1 steps 2-5, repeated on the points left out as §II
describes) against the oracle's, bit for bit, for every number of rounds one pass of
distances may serve (PSCL_OPT_PEEL_ROUNDS: a tuning choice that must not change the
result), on inputs that stress the epochs: many tiny rounds, boundaries whose bands
overlap (heavy distance ties), several holders of each attribute's minimum, a constant
attribute, and wide points."""
import numpy as np
import pytest

import oracle
from paper_1412_1947_gb300 import binding as B
from paper_1412_1947_gb300 import synth

pytestmark = pytest.mark.gpu


def _peel_gpu(raw, N, rounds):
    with B.Job(raw) as j:
        j.option(B.PSCL_OPT_PEEL_ROUNDS, rounds)
        j.steps(N, 2, 2, 1, 3)
        perm, off = j.partition()
        x = j.scaled()
    return perm, off, x


def _check(raw, N, rounds):
    perm, off, x = _peel_gpu(raw, N, rounds)
    operm, ooff, _ = oracle.peel(x, N, select=len(raw) > 50000)
    np.testing.assert_array_equal(off, ooff)
    np.testing.assert_array_equal(perm, operm)


@pytest.mark.parametrize("rounds", [1, 2, 5, 16, 32])
def test_mixture(rounds):
    _check(synth.mixture(30000, 16, 20, outlier_frac=0.01, seed=600), 1000, rounds)


@pytest.mark.parametrize("rounds", [1, 8, 16])
def test_integer_grid_ties(rounds):
    # thousands of equal distances per round, several holders of each minimum
    g = np.random.default_rng(601)
    raw = g.integers(0, 6, size=(20000, 2)).astype(np.float32)
    _check(raw, 1024, rounds)


@pytest.mark.parametrize("rounds", [3, 16])
def test_tiny_rounds(rounds):
    # N = 7: boundaries a few points apart, so their bands overlap and merge into groups
    _check(synth.mixture(5000, 4, 5, seed=602), 7, rounds)


def test_constant_attribute():
    g = np.random.default_rng(603)
    raw = g.normal(size=(12000, 8)).astype(np.float32)
    raw[:, 3] = 1.25
    _check(raw, 500, 8)


def test_wide_points():
    _check(synth.mixture(16384, 64, 32, seed=604), 1024, 8)


def test_generic_attribute_count():
    _check(synth.mixture(9001, 5, 7, outlier_frac=0.02, seed=605), 333, 8)


def test_duplicated_points():
    # every point twice: every distance tied in pairs
    base = synth.mixture(6000, 8, 6, seed=606)
    raw = np.concatenate([base, base])
    _check(raw, 512, 8)


@pytest.mark.parametrize("cap", [1, 7, 16, 19, 76])
def test_partition_does_not_depend_on_the_grid(cap):
    # PSCL_OPT_PEEL_GRID caps the cooperative launch (a grid under 16 CTAs has no
    # landmark-only CTAs, every CTA then does both); the partition is the oracle's
    raw = synth.mixture(6000, 16, 8, outlier_frac=0.01, seed=91)
    N = 250
    with B.Job(raw) as j:
        j.option(B.PSCL_OPT_PEEL_GRID, cap)
        j.steps(N, 4, 4, 1, 3)
        perm, off = j.partition()
        x = j.scaled()
    operm, ooff, _ = oracle.peel(x, N)
    np.testing.assert_array_equal(off, ooff)
    np.testing.assert_array_equal(perm, operm)


@pytest.mark.parametrize("n,d,blobs,N", [(1 << 17, 64, 256, 1024), (1 << 18, 16, 64, 1024),
                                         (1 << 18, 128, 256, 8192)])
def test_key_updates_keep_the_partition(n, d, blobs, N):
    # 128 and 256 rounds on the two measured shapes' recipes, scaled down: most landmark changes
    # move one or two attributes, so most passes update the keys from those attributes
    # (with the carried error bound) instead of recomputing them; the partition is still
    # the oracle's bit for bit.  The third case (128 MB of points, more than L2 holds)
    # reads the moved attributes from the copy of the points by attribute
    raw = synth.mixture(n, d, blobs, seed=607 + d)
    with B.Job(raw) as j:
        j.steps(N, 2, 2, 1, 3)
        perm, off = j.partition()
        x = j.scaled()
        epochs, passes, updates, barriers = j.peel_stats()
    print(f"epochs {epochs} passes {passes} key updates {updates} barriers {barriers}")
    assert 0 < updates < passes <= epochs
    # the bucket lists: 3 (after the counts, their scan and the places); every epoch 5,
    # and one more with a distance pass
    assert barriers == 3 + 5 * epochs + passes
    operm, ooff, _ = oracle.peel(x, N, select=True)
    np.testing.assert_array_equal(off, ooff)
    np.testing.assert_array_equal(perm, operm)
