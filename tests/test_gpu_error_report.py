"""Error report at the precision workload's full size: 2^24 points, d = 64, 1024 blobs,
subclusters of 65536 (256 of them), 256 local centers, final k = 1024, 25 iterations.

Every precision mode runs the whole job; the tensor-core modes must give the float32 mode's
labels, centers and SSE bit for bit (near ties are re-decided in float32).  The float32 run
is then checked against the oracle on a seeded sample, since the oracle cannot take the
whole job in test time:
  * the local Lloyd of sampled subclusters (the first, the last and two drawn at random),
    replayed on the run's label trace (the oracle follows the GPU's label only where its
    own float64 choice is a near tie within 1e-5; any other disagreement fails);
  * the final Lloyd on the pooled local centers, replayed the same way;
  * the SSE: the float64 sum over all 2^24 points of the distance to the nearest final
    center (the oracle's assignment, run over 16 chunks in parallel processes).
The peel's selection at full size is pinned by test_gpu_full_size.  The table printed here
is the report (Algorithm 1 steps 3-5)."""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1412_1947_gb300 import binding as B
from paper_1412_1947_gb300 import synth
from tests.parity import CENTER_TOL, SSE_TOL, TIE_TOL, run_gpu

pytestmark = pytest.mark.gpu

MODES = [("tf32", B.PSCL_PREC_TF32), ("bf16", B.PSCL_PREC_BF16), ("tf32x3", B.PSCL_PREC_TF32X3),
         ("bf16x3", B.PSCL_PREC_BF16X3), ("tc", B.PSCL_PREC_TC)]
SEED = 21
SSE_CHUNKS = 16


def _center_err(got, ref):
    return float(np.max(np.abs(got - ref)) / max(1.0, float(np.max(np.abs(ref)))))


def _local_job(path, rows_idx, s, k, iters, trace):
    x = np.load(path, mmap_mode="r")
    rows = np.ascontiguousarray(x[rows_idx], np.float32)
    init = rows[oracle.init_indices(SEED, 0, s, len(rows), k)].astype(np.float64)
    c, _, _, _, forced, bad = oracle.lloyd(rows, init, iters, force=trace, tie_tol=TIE_TOL)
    return c, forced, bad


def _final_job(pooled, k, iters, trace):
    init = pooled[oracle.init_indices(SEED, 1, 0, len(pooled), k)].astype(np.float64)
    c, _, _, _, forced, bad = oracle.lloyd(pooled, init, iters, force=trace, tie_tol=TIE_TOL)
    return c, forced, bad


def _sse_job(path, lo, hi, centers):
    x = np.load(path, mmap_mode="r")
    _, best, _ = oracle.assign(np.ascontiguousarray(x[lo:hi], np.float32), centers)
    return math.fsum(best)


def test_error_report_at_full_size(tmp_path):
    import concurrent.futures as cf
    import multiprocessing as mp
    w = synth.LARGE
    raw = w.points()
    ref = run_gpu(raw, w.N, w.local_k, w.final_k, w.iters, seed=SEED, device_points=True)
    rows = [("fp32", ref.rechecked, ref.assigned)]
    for name, prec in MODES:
        g = run_gpu(raw, w.N, w.local_k, w.final_k, w.iters, seed=SEED, trace=False, device_points=True, prec=prec)
        np.testing.assert_array_equal(g.perm, ref.perm)
        np.testing.assert_array_equal(g.local_centers, ref.local_centers)
        np.testing.assert_array_equal(g.final_centers, ref.final_centers)
        np.testing.assert_array_equal(g.labels, ref.labels)
        assert g.sse == ref.sse
        rows.append((name, g.rechecked, g.assigned))
        del g
    del raw
    path = os.path.join(str(tmp_path), "scaled.npy")
    np.save(path, ref.scaled)
    n, N, k, T = w.n, w.N, w.local_k, w.iters
    S = len(ref.seg_off) - 1
    rng = np.random.default_rng(7)
    segs = sorted({0, S - 1} | set(int(v) for v in rng.choice(np.arange(1, S - 1), 2, replace=False)))
    fc = ref.final_centers.astype(np.float64)
    bounds = np.linspace(0, n, SSE_CHUNKS + 1).astype(np.int64)
    with cf.ProcessPoolExecutor(max_workers=min(os.cpu_count() or 1, SSE_CHUNKS + len(segs) + 1),
                                mp_context=mp.get_context("spawn")) as ex:
        fin = ex.submit(_final_job, ref.local_centers.astype(np.float32), w.final_k, T, ref.trace_final)
        loc = {s: ex.submit(_local_job, path, ref.perm[ref.seg_off[s]:ref.seg_off[s + 1]], s, k, T,
                            np.ascontiguousarray(ref.trace_local[:, ref.seg_off[s]:ref.seg_off[s + 1]]))
               for s in segs}
        sse_parts = [ex.submit(_sse_job, path, int(bounds[i]), int(bounds[i + 1]), fc) for i in range(SSE_CHUNKS)]
        loc = {s: f.result() for s, f in loc.items()}
        fin = fin.result()
        sse_or = math.fsum(f.result() for f in sse_parts)
    local_err = max(_center_err(ref.local_centers[s * k:(s + 1) * k], c) for s, (c, _, _) in loc.items())
    local_forced = sum(v[1] for v in loc.values())
    local_bad = sum(v[2] for v in loc.values())
    final_err = _center_err(ref.final_centers, fin[0])
    sse_rel = abs(ref.sse - sse_or) / sse_or
    print(f"\nerror report, n={n} d={w.d} N={N} local_k={k} final_k={w.final_k} iters={T}; "
          f"sampled subclusters {segs}")
    print("mode     rechecked/assigned (tensor-core near ties re-decided in float32)")
    for name, rc, asg in rows:
        print(f"{name:8s} {rc:>10d}/{asg:<10d}")
    print("every mode: labels, centers and SSE equal to fp32's; against the float64 oracle:")
    print(f"  local center err (sampled) {local_err:.2e}, exempt near ties {local_forced}, other disagreements "
          f"{local_bad}")
    print(f"  final center err {final_err:.2e}, exempt near ties {fin[1]}, other disagreements {fin[2]}")
    print(f"  SSE {ref.sse:.10e} vs float64 {sse_or:.10e}: relative {sse_rel:.2e}")
    assert local_bad == 0 and fin[2] == 0
    assert local_err <= CENTER_TOL and final_err <= CENTER_TOL
    assert sse_rel <= SSE_TOL
