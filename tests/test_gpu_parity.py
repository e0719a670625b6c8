"""The CUDA path against the oracle, element by element, on seeded inputs."""
import numpy as np
import pytest

import oracle
from paper_1412_1947_gb300 import binding as B
from paper_1412_1947_gb300 import synth
from tests.golden_io import arr, load
from tests.parity import compare, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def test_hand_example_exact():
    g = load("hand_2d.txt")
    N, lk, fk, T = (int(v) for v in g["params"][0])
    raw = arr(g["raw"], np.float32)
    r = run_gpu(raw, N, lk, fk, T, seed=0, first_k=True)
    np.testing.assert_array_equal(r.scaled, arr(g["scaled"], np.float32))
    segs = [int(v) for row in g["segments"] for v in row]
    np.testing.assert_array_equal(r.perm, segs)
    np.testing.assert_array_equal(r.local_centers, arr(g["local_centers"], np.float32))
    np.testing.assert_array_equal(r.final_centers, arr(g["final_centers"], np.float32))
    np.testing.assert_array_equal(r.labels, arr(g["labels"]).astype(np.int32))
    assert r.sse == float(g["sse"][0][0])


@pytest.mark.parametrize("n,d,outl", [(4096, 4, 0.0), (5000, 5, 0.01), (3333, 16, 0.01), (777, 3, 0.0),
                                      (20000, 32, 0.0), (1, 7, 0.0)])
def test_scaling_bit_exact(n, d, outl):
    raw = synth.mixture(n, d, 5, outlier_frac=outl, seed=100 + n + d)
    if d > 2:
        raw[:, 1] = 2.5                        # a constant attribute
    with B.Job(raw) as j:
        B.pscl_scale_features(j.h)
        got = j.scaled()
    exp, _, _ = oracle.scale(raw)
    np.testing.assert_array_equal(got, exp)


def _hard_columns(n, seed):
    """Attributes that drive the scaling's float-float filter to its edges: sixty decades of
    magnitude of both signs, a minimum repeated by 30 % of the rows, a range of 1e30 (1/range
    below 2^-60, subnormal scaled values), a range of 1e-19 (1/range above 2^60), values a few
    ulps from mid-range power-of-two results, a constant, and a plain uniform attribute."""
    rng = np.random.default_rng(seed)
    cols = [
        rng.uniform(-1, 1, n) * 10.0 ** rng.integers(-30, 30, n),
        np.where(rng.random(n) < 0.3, -5.0, rng.uniform(-5, 1e-6, n)),
        np.concatenate([[0.0, 1e30], rng.uniform(0, 1e-8, n - 2)]),
        rng.uniform(0, 1e-19, n),
        np.concatenate([[0.0, 3.0], 1.5 + rng.integers(-64, 64, n - 2) * 2.0 ** -23,]),
        np.full(n, 2.5),
        rng.uniform(-3, 7, n),
    ]
    return np.stack(cols, axis=1).astype(np.float32)


@pytest.mark.parametrize("d", [7, 8])
def test_scaling_hard_attributes_bit_exact(d):
    """float32 and bfloat16 storage, vectorised (d % 4 == 0) and scalar passes: every scaled
    value bit for bit equal to the float64 definition."""
    from tests.test_gpu_bf16 import to_bf16
    n = 200_003
    raw = _hard_columns(n, 41 + d)
    raw = np.concatenate([raw, raw[:, : d - raw.shape[1]]], axis=1) if d > raw.shape[1] else raw[:, :d]
    raw = np.ascontiguousarray(raw)
    with B.Job(raw) as j:
        B.pscl_scale_features(j.h)
        got = j.scaled()
    exp, _, _ = oracle.scale(raw)
    np.testing.assert_array_equal(got.view(np.uint32), exp.view(np.uint32))
    bits, vals = to_bf16(raw)
    with B.Job(bits) as j:
        B.pscl_scale_features(j.h)
        got = j.scaled()
    exp, _, _ = oracle.scale(vals, bf16=True)
    np.testing.assert_array_equal(got.view(np.uint32), exp.view(np.uint32))


def test_small_workload_parity():
    w = synth.SMALL
    raw = w.points()
    g = run_gpu(raw, w.N, w.local_k, w.final_k, w.iters, seed=11)
    o = run_oracle(raw, w.N, w.local_k, w.final_k, w.iters, seed=11, gpu=g)
    stats = compare(g, o)
    assert stats["local_center_err"] < 1e-6


@pytest.mark.parametrize("n,d,N,lk,fk,T", [
    (65536, 16, 4096, 64, 64, 25),      # the headline recipe at 1/16 size: 16 rounds
    (10000, 3, 768, 20, 10, 8),         # ragged tail, generic attribute count
    (9001, 8, 1000, 64, 30, 10),        # ragged, units smaller than a subcluster
    (3000, 4, 5000, 16, 4, 5),          # N >= n: a single subcluster
    (1500, 2, 7, 3, 12, 4),             # many tiny rounds, tail of 2 points
    (2048, 64, 512, 32, 16, 6),         # wide points
    (1200, 128, 300, 8, 8, 3),          # widest specialisation
    (999, 16, 100, 200, 50, 4),         # local_k > N: every point is a local center
])
def test_two_level_parity(n, d, N, lk, fk, T):
    raw = synth.mixture(n, d, 12, outlier_frac=0.01, seed=1000 + n + d)
    g = run_gpu(raw, N, lk, fk, T, seed=5 + n)
    o = run_oracle(raw, N, lk, fk, T, seed=5 + n, gpu=g)
    compare(g, o)


def test_partition_with_massive_ties():
    # points on a coarse integer grid: thousands of exactly equal distances per round,
    # decided by index inside the float64 band
    g0 = np.random.default_rng(7)
    raw = g0.integers(0, 6, size=(20000, 2)).astype(np.float32)
    g = run_gpu(raw, 1024, 8, 8, 3, seed=3)
    o = run_oracle(raw, 1024, 8, 8, 3, seed=3, gpu=g)
    compare(g, o)


def test_partition_all_points_equal():
    raw = np.full((3000, 4), 0.5, np.float32)
    raw[:, 0] = 1.0
    g = run_gpu(raw, 256, 4, 2, 2, seed=1)
    o = run_oracle(raw, 256, 4, 2, 2, seed=1, gpu=g)
    np.testing.assert_array_equal(g.perm, np.arange(3000))
    compare(g, o)


def test_plain_and_batched_are_bitwise_equal():
    raw = synth.mixture(30000, 16, 20, outlier_frac=0.01, seed=77)
    a = run_gpu(raw, 2048, 32, 16, 10, seed=9, trace=False)
    b = run_gpu(raw, 2048, 32, 16, 10, seed=9, trace=False, plain=True)
    np.testing.assert_array_equal(a.local_centers, b.local_centers)
    np.testing.assert_array_equal(a.final_centers, b.final_centers)
    np.testing.assert_array_equal(a.labels, b.labels)
    assert a.sse == b.sse


def test_graph_replay_equals_eager():
    raw = synth.mixture(20000, 16, 20, outlier_frac=0.01, seed=78)
    a = run_gpu(raw, 1024, 32, 16, 6, seed=4, trace=False)
    b = run_gpu(raw, 1024, 32, 16, 6, seed=4, trace=False, graph=True, runs=3)
    np.testing.assert_array_equal(a.perm, b.perm)
    np.testing.assert_array_equal(a.final_centers, b.final_centers)
    assert a.sse == b.sse


def test_device_input_equals_host_input():
    raw = synth.mixture(12345, 8, 9, seed=79)
    a = run_gpu(raw, 1000, 16, 8, 5, seed=2, trace=False)
    b = run_gpu(raw, 1000, 16, 8, 5, seed=2, trace=False, device_points=True)
    np.testing.assert_array_equal(a.perm, b.perm)
    np.testing.assert_array_equal(a.final_centers, b.final_centers)


def test_errors_and_state():
    raw = synth.mixture(1000, 4, 3, seed=80)
    with B.Job(raw) as j:
        with pytest.raises(B.PsclError) as e:
            B.pscl_subcluster(j.h, 100, 4, 2, 0)
        assert e.value.code == B.PSCL_ESTATE
        B.pscl_scale_features(j.h)
        with pytest.raises(B.PsclError) as e:
            B.pscl_cluster(j.h, 4, 2, 0)
        assert e.value.code == B.PSCL_ESTATE
        B.pscl_subcluster(j.h, 100, 4, 2, 0)
        S, P = j.sizes()
        assert (S, P) == (10, 40)
        with pytest.raises(B.PsclError) as e:
            B.pscl_cluster(j.h, 41, 2, 0)
        assert e.value.code == B.PSCL_EINVAL
        with pytest.raises(B.PsclError) as e:
            B.pscl_subcluster(j.h, 0, 4, 2, 0)
        assert e.value.code == B.PSCL_EINVAL
    ctx = B.pscl_ctx_create(0, 1 << 20)
    try:
        with pytest.raises(B.PsclError) as e:
            B.pscl_job_create(ctx, synth.mixture(100000, 16, 3, seed=1))
        assert e.value.code == B.PSCL_ENOMEM
        assert B.pscl_ctx_bytes_in_use(ctx) == 0
    finally:
        B.pscl_ctx_destroy(ctx)


def test_nonfinite_input_is_reported():
    raw = synth.mixture(1000, 4, 3, seed=81)
    raw[17, 2] = np.nan
    with B.Job(raw) as j:
        B.pscl_scale_features(j.h)
        with pytest.raises(B.PsclError) as e:
            j.scaled()
        assert e.value.code == B.PSCL_EINVAL


@pytest.mark.parametrize("n,d,N,lk,fk,T", [
    (1, 3, 1, 1, 1, 3),                 # a single point: constant attributes, one subcluster
    (50, 1, 10, 3, 2, 5),               # one attribute (the any-d kernels)
    (300, 4, 1, 1, 5, 3),               # N = 1: every point its own subcluster and center
    (500, 8, 100, 5, 25, 0),            # no Lloyd iteration: the seeded initial centers
    (400, 6, 80, 4, 20, 4),             # final k = every pooled center
])
def test_degenerate_shapes_match_oracle(n, d, N, lk, fk, T):
    raw = synth.mixture(n, d, 3, seed=90 + n)
    g = run_gpu(raw, N, lk, fk, T, seed=3)
    o = run_oracle(raw, N, lk, fk, T, seed=3, gpu=g)
    compare(g, o)
