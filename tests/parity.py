"""Running the CUDA library and the oracle on the same seeded input and comparing them.

Tolerances (the figures the method is held to):
  * scaled points and the partition into subclusters: bit-exact;
  * centers: |c_gpu - c_oracle|_inf <= 1e-4 * max(1, |c_oracle|_inf);
  * SSE: relative 1e-5;
  * labels: equal, except where the oracle's own choice is not unique within 1e-5: the
    oracle's distance to the CUDA path's choice is within 1e-5 * max(1, best) of its best.

Lloyd's trajectory is not unique at such near-ties, so the comparison replays it: the
oracle is given the CUDA path's label of every iteration and follows it only where its
own decision is such a near-tie; every other disagreement is counted as a failure.
"""
from dataclasses import dataclass

import numpy as np

import oracle
from paper_1412_1947_gb300 import binding as B

CENTER_TOL = 1e-4
SSE_TOL = 1e-5
TIE_TOL = 1e-5


@dataclass
class DeviceRun:
    scaled: np.ndarray
    perm: np.ndarray
    seg_off: np.ndarray
    local_centers: np.ndarray
    k_eff: np.ndarray
    counts: np.ndarray
    final_centers: np.ndarray
    labels: np.ndarray
    sse: float
    trace_local: np.ndarray | None
    trace_final: np.ndarray | None
    rechecked: int = 0
    assigned: int = 0


def run_gpu(raw, N, local_k, final_k, iters, seed, *, trace=True, plain=False, first_k=False,
            graph=False, prec=B.PSCL_PREC_FP32, runs=1, device_points=False, unequal_m=0,
            pool_weighted=False):
    pts = raw
    if device_points:
        import torch
        pts = torch.from_numpy(np.ascontiguousarray(raw, np.float32)).cuda()
    with B.Job(pts) as j:
        if trace:
            j.option(B.PSCL_OPT_TRACE_LABELS)
        if plain:
            j.option(B.PSCL_OPT_PLAIN_LLOYD)
        if first_k:
            j.option(B.PSCL_OPT_INIT_FIRST_K)
        if graph:
            j.option(B.PSCL_OPT_GRAPH)
        if pool_weighted:
            j.option(B.PSCL_OPT_POOL_WEIGHTED)
        for _ in range(runs):
            if unequal_m:
                j.steps_unequal(unequal_m, local_k, final_k, iters, seed, prec)
            elif graph:
                j.run(N, local_k, final_k, iters, seed, prec)
            else:
                j.steps(N, local_k, final_k, iters, seed, prec)
        perm, seg_off = j.partition()
        lc, ke, cnt = j.local_centers()
        fc, lab, sse = j.result()
        tl = j.trace(0, iters) if trace and iters else None
        tf = j.trace(1, iters) if trace and iters else None
        rc, asg = j.recheck_stats()
        return DeviceRun(j.scaled(), perm, seg_off, lc, ke, cnt, fc, lab, sse, tl, tf, rc, asg)


def run_oracle(raw, N, local_k, final_k, iters, seed, gpu: DeviceRun | None = None, first_k=False, unequal_m=0,
               pool_weighted=False):
    fl = ff = None
    if gpu is not None and gpu.trace_local is not None:
        fl, ff = gpu.trace_local, gpu.trace_final
    return oracle.two_level(raw, N, local_k, final_k, iters, seed, first_k=first_k,
                            force_local=fl, force_final=ff, tie_tol=TIE_TOL, unequal_m=unequal_m,
                            pool_weighted=pool_weighted)


def center_err(a, ref):
    ref = np.asarray(ref, np.float64)
    return float(np.abs(np.asarray(a, np.float64) - ref).max()) / max(1.0, float(np.abs(ref).max()))


def compare(g: DeviceRun, o, *, check_labels=True):
    """Assert parity; returns a dict of the measured differences."""
    assert np.array_equal(g.scaled, o.scaled), "scaled points differ"
    assert np.array_equal(g.seg_off, o.seg_off), "subcluster offsets differ"
    assert np.array_equal(g.perm, o.perm), "partition differs"
    assert np.array_equal(g.k_eff, o.local_k_eff)
    assert o.n_bad == 0, f"{o.n_bad} label disagreements outside the near-tie band"
    le = center_err(g.local_centers, o.local_centers)
    fe = center_err(g.final_centers, o.final_centers)
    assert le <= CENTER_TOL, f"local centers off by {le:.3e}"
    assert fe <= CENTER_TOL, f"final centers off by {fe:.3e}"
    rel = abs(g.sse - o.sse) / max(abs(o.sse), 1e-300)
    assert rel <= SSE_TOL, f"SSE {g.sse!r} vs oracle {o.sse!r} (rel {rel:.2e})"
    exempt = 0
    if check_labels:
        diff = np.flatnonzero(g.labels != o.labels)
        if len(diff):
            gap = o.second[diff] - o.best[diff]
            tie = gap <= TIE_TOL * np.maximum(1.0, o.best[diff])
            assert tie.all(), f"{int((~tie).sum())} final labels differ outside the near-tie band"
            exempt = len(diff)
    return {"local_center_err": le, "final_center_err": fe, "sse_rel": rel,
            "replayed_ties": int(o.n_forced), "label_ties": exempt}


# ---------------------------------------------------------------- uneven batches
@dataclass
class BatchRun:
    scaled: np.ndarray
    centers: np.ndarray          # sum(k_eff) x d
    labels: np.ndarray
    sse: np.ndarray              # per instance
    trace: np.ndarray | None     # iters x rows


def run_gpu_batch(parts, ks, iters, seed, *, trace=True, prec=B.PSCL_PREC_FP32, graph=True,
                  unit_rows=0, rows_per_thread=0, tune=False, device_points=False):
    raw = np.ascontiguousarray(np.concatenate(parts), np.float32)
    sizes = [len(p) for p in parts]
    pts = raw
    if device_points:
        import torch
        pts = torch.from_numpy(raw).cuda()
    with B.Batch(pts, sizes, ks) as b:
        b.option(B.PSCL_OPT_GRAPH, graph)
        if trace:
            b.option(B.PSCL_OPT_TRACE_LABELS)
        if unit_rows:
            b.option(B.PSCL_OPT_UNIT_ROWS, unit_rows)
        if rows_per_thread:
            b.option(B.PSCL_OPT_ROWS_PER_THREAD, rows_per_thread)
        if tune:
            b.tune(2, prec)
        b.run(iters, seed, prec)
        c, lab, sse = b.result()
        tr = b.trace() if trace and iters else None
        return BatchRun(b.scaled(), c, lab, sse, tr)


def compare_batch(g: BatchRun, parts, ks, iters, seed, only=None):
    """Each instance (or those listed in `only`) against the oracle: scaling, seeded init
    (stage 0, segment = index), Lloyd replayed on the CUDA path's labels, final nearest
    centers and SSE."""
    row = cen = 0
    worst = {"center_err": 0.0, "sse_rel": 0.0, "replayed_ties": 0, "label_ties": 0}
    keep = None if only is None else set(int(i) for i in only)
    for i, (p, k) in enumerate(zip(parts, ks)):
        m = len(p)
        ke = min(k, m)
        if keep is not None and i not in keep:
            row += m
            cen += ke
            continue
        xs, _, _ = oracle.scale(p)
        assert np.array_equal(g.scaled[row:row + m], xs), f"instance {i}: scaled points differ"
        init = xs[oracle.init_indices(seed, 0, i, m, ke)]
        force = None if g.trace is None else g.trace[:, row:row + m]
        c, _, _, _, nf, nb = oracle.lloyd(xs, init, iters, force=force, tie_tol=TIE_TOL)
        assert nb == 0, f"instance {i}: {nb} label disagreements outside the near-tie band"
        ce = center_err(g.centers[cen:cen + ke], c)
        assert ce <= CENTER_TOL, f"instance {i}: centers off by {ce:.3e}"
        lab, best, second = oracle.assign(xs, c)
        sse = float(best.sum())
        rel = abs(g.sse[i] - sse) / max(abs(sse), 1e-300)
        assert rel <= SSE_TOL, f"instance {i}: SSE {g.sse[i]!r} vs oracle {sse!r}"
        diff = np.flatnonzero(g.labels[row:row + m] != lab)
        if len(diff):
            tie = second[diff] - best[diff] <= TIE_TOL * np.maximum(1.0, best[diff])
            assert tie.all(), f"instance {i}: {int((~tie).sum())} final labels differ outside the near-tie band"
        worst["center_err"] = max(worst["center_err"], ce)
        worst["sse_rel"] = max(worst["sse_rel"], rel)
        worst["replayed_ties"] += nf
        worst["label_ties"] += len(diff)
        row += m
        cen += ke
    return worst
