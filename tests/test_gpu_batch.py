"""Uneven batches of independent instances against the oracle, instance by instance."""
import numpy as np
import pytest

from paper_1412_1947_gb300 import binding as B
from paper_1412_1947_gb300 import synth
from tests.parity import compare_batch, run_gpu_batch

pytestmark = pytest.mark.gpu


def make_batch(count, d, lo, hi, seed, kdiv=64):
    sizes = synth.uneven_sizes(count, lo, hi, seed)
    parts = [synth.mixture(int(m), d, max(2, int(m) // 200), seed=seed * 31 + i) for i, m in enumerate(sizes)]
    ks = [max(2, int(m) // kdiv) for m in sizes]
    return parts, ks


@pytest.mark.parametrize("d", [32, 16, 5])
def test_batch_matches_oracle(d):
    parts, ks = make_batch(24, d, 40, 3000, seed=700 + d)
    g = run_gpu_batch(parts, ks, 8, seed=5)
    r = compare_batch(g, parts, ks, 8, seed=5)
    print(r)


def test_batch_edge_instances():
    # single-point instances, k above the size (k_eff = size), k = 1, one instance much
    # larger than a work unit
    rng = np.random.default_rng(3)
    parts = [rng.normal(size=(1, 8)).astype(np.float32), rng.normal(size=(3, 8)).astype(np.float32),
             rng.normal(size=(5000, 8)).astype(np.float32), rng.normal(size=(33, 8)).astype(np.float32)]
    ks = [4, 7, 1, 33]
    g = run_gpu_batch(parts, ks, 5, seed=9)
    compare_batch(g, parts, ks, 5, seed=9)


def test_batch_tuning_choices_do_not_change_results():
    parts, ks = make_batch(16, 32, 100, 5000, seed=811)
    ref = run_gpu_batch(parts, ks, 6, seed=2, trace=False)
    for ur, rpt in [(32, 0), (128, 1), (1024, 0), (512, 1)]:
        g = run_gpu_batch(parts, ks, 6, seed=2, trace=False, unit_rows=ur, rows_per_thread=rpt)
        np.testing.assert_array_equal(g.centers, ref.centers)
        np.testing.assert_array_equal(g.labels, ref.labels)
        np.testing.assert_array_equal(g.sse, ref.sse)
    g = run_gpu_batch(parts, ks, 6, seed=2, trace=False, tune=True)
    np.testing.assert_array_equal(g.centers, ref.centers)


def test_batch_graph_replay_device_input_and_plain_form():
    parts, ks = make_batch(12, 16, 64, 2000, seed=901)
    a = run_gpu_batch(parts, ks, 5, seed=4, trace=False, graph=False)
    b = run_gpu_batch(parts, ks, 5, seed=4, trace=False, graph=True, device_points=True)
    np.testing.assert_array_equal(a.centers, b.centers)
    np.testing.assert_array_equal(a.sse, b.sse)
    raw = np.concatenate(parts)
    with B.Batch(raw, [len(p) for p in parts], ks) as bt:
        bt.option(B.PSCL_OPT_PLAIN_LLOYD)
        bt.run(5, 4)
        c, lab, sse = bt.result()
        np.testing.assert_array_equal(c, a.centers)
        np.testing.assert_array_equal(sse, a.sse)
        # new points of the same shape through pscl_batch_load
        bt.load(np.ascontiguousarray(raw[::-1]))
        bt.option(B.PSCL_OPT_PLAIN_LLOYD, 0)
        bt.run(5, 4)
        bt.load(raw)
        bt.run(5, 4)
        c2, _, sse2 = bt.result()
        np.testing.assert_array_equal(c2, a.centers)


@pytest.mark.parametrize("name,prec", [("tf32", B.PSCL_PREC_TF32), ("bf16x3", B.PSCL_PREC_BF16X3)])
def test_batch_tensor_cores_equal_float32(name, prec):
    parts, ks = make_batch(20, 32, 200, 6000, seed=1200)
    ref = run_gpu_batch(parts, ks, 6, seed=8, trace=False)
    g = run_gpu_batch(parts, ks, 6, seed=8, trace=False, prec=prec)
    np.testing.assert_array_equal(g.centers, ref.centers)
    np.testing.assert_array_equal(g.labels, ref.labels)


def test_autotuner_remembers_its_choice():
    parts, ks = make_batch(10, 16, 200, 4000, seed=1300)
    raw = np.concatenate(parts)
    with B.Batch(raw, [len(p) for p in parts], ks) as b:
        u, r, cached = b.tune(2)
        assert u in (128, 256, 512, 1024) and r in (0, 1) and not cached
    with B.Batch(raw, [len(p) for p in parts], ks) as b:
        u2, r2, cached2 = b.tune(2)
        assert cached2 and (u2, r2) == (u, r)
