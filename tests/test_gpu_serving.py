"""The job server: admission by device footprint, overlap of jobs on the device, and
results equal to the same jobs run alone."""
import math
import time

import numpy as np
import pytest

from paper_1412_1947_gb300 import binding as B
from paper_1412_1947_gb300 import synth

pytestmark = pytest.mark.gpu


def serving_params(n, final_k):
    """N = ceil(n / 64) and the local k of the serving recipe (pooled count >= 2 final_k)."""
    N = -(-n // 64)
    S = -(-n // N)
    local_k = min(N, max(8, -(-N // 256), -(-2 * final_k // S)))
    return N, local_k


def make_jobs(count, seed):
    rng = np.random.default_rng(seed)
    jobs = []
    for i in range(count):
        n = int(math.exp(rng.uniform(math.log(4000), math.log(60000))))
        d = int(rng.choice([8, 16, 32]))
        fk = int(math.exp(rng.uniform(math.log(4), math.log(64))))
        N, lk = serving_params(n, fk)
        pts = synth.mixture(n, d, max(2, fk), seed=seed * 100 + i)
        jobs.append(dict(points=pts, N=N, local_k=lk, final_k=fk, iters=6, seed=1000 + i))
    return jobs


def run_alone(job):
    with B.Job(job["points"]) as j:
        j.run(job["N"], job["local_k"], job["final_k"], job["iters"], job["seed"])
        return j.result()


@pytest.mark.parametrize("n,d,N,lk,fk,T,host", [(10000, 8, 157, 8, 8, 3, True), (50000, 32, 782, 12, 40, 2, False),
                                                 (4096, 4, 256, 16, 3, 20, False), (50000, 32, 782, 12, 300, 2, False),
                                                 (50000, 16, 782, 12, 512, 2, True)])
def test_footprint_is_the_allocated_bytes(n, d, N, lk, fk, T, host):
    import torch
    pts = synth.mixture(n, d, 5, seed=n)
    src = pts if host else torch.from_numpy(pts).cuda()
    ctx = B.pscl_ctx_create(0)
    try:
        j = B.Job(src, ctx=ctx)
        j.run(N, lk, fk, T, 1)
        j.result(labels=False)
        assert B.pscl_ctx_bytes_in_use(ctx) == B.pscl_job_footprint(ctx, n, d, N, lk, fk, T, on_device=not host)
        j.close()
        assert B.pscl_ctx_bytes_in_use(ctx) == 0
    finally:
        B.pscl_ctx_destroy(ctx)


def test_jobs_in_the_mix_equal_jobs_alone():
    import torch
    jobs = make_jobs(10, seed=41)
    alone = [run_alone(jb) for jb in jobs]
    dev = [torch.from_numpy(jb["points"]).cuda() for jb in jobs]
    with B.Server(slots=3) as s:
        tickets = [s.submit(x, jb["N"], jb["local_k"], jb["final_k"], jb["iters"], jb["seed"], want_labels=True)
                   for x, jb in zip(dev, jobs)]
        for t in tickets:
            s.wait(t)
        st = s.stats()
        for t, ref in zip(tickets, alone):
            c, lab, sse, times = s.fetch(t)
            np.testing.assert_array_equal(c, ref[0])
            np.testing.assert_array_equal(lab, ref[1])
            assert sse == ref[2]
            assert times[2] >= times[1] >= 0.0
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["max_running"] >= 2, st          # jobs were on the device together
    assert st["peak_bytes"] <= st["budget"]


def test_admission_keeps_to_the_budget():
    import torch
    jobs = make_jobs(6, seed=77)
    dev = [torch.from_numpy(jb["points"]).cuda() for jb in jobs]
    ctx = B.pscl_ctx_create(0)
    fps = [B.pscl_job_footprint(ctx, len(jb["points"]), jb["points"].shape[1], jb["N"], jb["local_k"],
                                jb["final_k"], jb["iters"]) for jb in jobs]
    budget = max(fps) + min(fps)             # at most two of them at a time, often one
    with B.Server(slots=4, hbm_budget_bytes=budget, ctx=ctx) as s:
        ts = [s.submit(x, jb["N"], jb["local_k"], jb["final_k"], jb["iters"], jb["seed"]) for x, jb in zip(dev, jobs)]
        for t in ts:
            s.wait(t)
        st = s.stats()
        for t, jb in zip(ts, jobs):
            c, _, sse, _ = s.fetch(t)
            ref = run_alone(jb)
            np.testing.assert_array_equal(c, ref[0])
        assert st["peak_bytes"] <= budget and st["completed"] == len(jobs)
        # a job larger than the whole budget can never start
        big = torch.from_numpy(synth.mixture(200000, 32, 8, seed=5)).cuda()
        with pytest.raises(B.PsclError) as e:
            s.submit(big, 3125, 8, 8, 3, 1)
        assert e.value.code == B.PSCL_ENOMEM
    B.pscl_ctx_destroy(ctx)


def test_wait_times_out_and_arrivals_overlap():
    import torch
    big = torch.from_numpy(synth.mixture(1 << 20, 16, 64, seed=9)).cuda()
    small = [torch.from_numpy(jb["points"]).cuda() for jb in make_jobs(4, seed=90)]
    with B.Server(slots=3) as s:
        t0 = s.submit(big, 16384, 16, 64, 25, 3)
        with pytest.raises(B.PsclError) as e:
            s.wait(t0, 1)
        assert e.value.code == B.PSCL_ETIMEOUT
        assert s.poll(t0) in (B.PSCL_JOB_QUEUED, B.PSCL_JOB_RUNNING)
        # jobs that arrive while the big one runs start and finish without waiting for it
        later = []
        for x in small:
            time.sleep(0.002)
            later.append(s.submit(x, 500, 8, 8, 3, 7))
        for t in later:
            s.wait(t)
        done_small = [s.poll(t) for t in later]
        s.wait(t0)
        assert all(v == B.PSCL_JOB_DONE for v in done_small)
        _, _, _, tb = s.fetch(t0)
        for t in later:
            _, _, _, ts = s.fetch(t)
            assert ts[0] < tb[2]               # admitted before the big job was done


def test_a_waiting_job_is_passed_over_only_by_jobs_that_start():
    # Backfill: a large job that does not fit while another large one runs lets the small
    # jobs behind it start.  It counts as passed over once per job that starts ahead of it,
    # not once per scheduler pass (which would reach the limit within a few ms and then
    # hold every later job back), so small jobs that arrive 5 ms later still start while
    # the first large job runs; results stay exact.
    import torch
    big = [torch.from_numpy(synth.mixture(1 << 21, 32, 64, seed=s)).cuda() for s in (11, 12)]
    smalls = make_jobs(3, seed=55)                 # as many as the slots left free
    dev = [torch.from_numpy(jb["points"]).cuda() for jb in smalls]
    ctx = B.pscl_ctx_create(0)
    fp_big = B.pscl_job_footprint(ctx, 1 << 21, 32, 8192, 64, 64, 40)
    fp_small = max(B.pscl_job_footprint(ctx, len(jb["points"]), jb["points"].shape[1], jb["N"], jb["local_k"],
                                        jb["final_k"], jb["iters"]) for jb in smalls)
    budget = 2 * fp_big - 1                        # the two large jobs never fit together
    assert fp_big + 3 * fp_small <= budget
    with B.Server(slots=4, hbm_budget_bytes=budget, ctx=ctx) as s:
        t0 = time.perf_counter()
        t_big = [s.submit(x, 8192, 64, 64, 40, 3) for x in big]
        sub_big1 = 1e3 * (time.perf_counter() - t0)
        time.sleep(0.005)                          # the second large job waits meanwhile
        ts, sub = [], []
        for x, jb in zip(dev, smalls):
            sub.append(1e3 * (time.perf_counter() - t0))
            ts.append(s.submit(x, jb["N"], jb["local_k"], jb["final_k"], jb["iters"], jb["seed"], want_labels=True))
        for t in t_big + ts:
            s.wait(t)
        _, _, _, tb0 = s.fetch(t_big[0])
        _, _, _, tb1 = s.fetch(t_big[1])
        for t, jb, sb in zip(ts, smalls, sub):
            c, lab, sse, tt = s.fetch(t)
            ref = run_alone(jb)
            np.testing.assert_array_equal(c, ref[0])
            np.testing.assert_array_equal(lab, ref[1])
            assert sse == ref[2]
            assert sb + tt[0] < tb0[2], (sb, tt, tb0)    # admitted before the first large job was done
        assert sub_big1 + tb1[0] + 0.1 >= tb0[2]         # the second large job waited for the first
    B.pscl_ctx_destroy(ctx)


def test_served_jobs_match_the_oracle():
    # a seeded sample of the serving recipe (n and final k log-uniform, d in {8, 32, 128},
    # half of the jobs stored in bfloat16, 25 iterations) served together; each job equals
    # the same job run alone, and that run (with its label traces) matches the oracle
    import torch
    from tests.parity import TIE_TOL, compare, run_gpu
    import oracle
    from tests.test_gpu_bf16 import to_bf16
    jobs = synth.serving_stream(12, seed=321, n_range=(1e4, 6e4), k_range=(8, 128))
    pts = []
    for jb in jobs:
        x = synth.mixture(jb["n"], jb["d"], jb["blobs"], seed=jb["seed"])
        pts.append(to_bf16(x) if jb["bf16"] else (x, x))
    dev = [torch.from_numpy(v).cuda().to(torch.bfloat16) if jb["bf16"] else torch.from_numpy(v).cuda()
           for (b, v), jb in zip(pts, jobs)]
    with B.Server(slots=4) as s:
        ts = [s.submit(x, jb["N"], jb["local_k"], jb["final_k"], jb["iters"], jb["seed"], want_labels=True)
              for x, jb in zip(dev, jobs)]
        for t in ts:
            s.wait(t)
        served = [s.fetch(t) for t in ts]
    assert sum(jb["bf16"] for jb in jobs) not in (0, len(jobs))
    for (bits, vals), jb, (c, lab, sse, _) in zip(pts, jobs, served):
        g = run_gpu(bits if jb["bf16"] else vals, jb["N"], jb["local_k"], jb["final_k"], jb["iters"], jb["seed"])
        np.testing.assert_array_equal(c, g.final_centers)
        np.testing.assert_array_equal(lab, g.labels)
        assert sse == g.sse
        o = oracle.two_level(vals, jb["N"], jb["local_k"], jb["final_k"], jb["iters"], jb["seed"],
                             bf16=jb["bf16"], force_local=g.trace_local, force_final=g.trace_final,
                             tie_tol=TIE_TOL)
        compare(g, o)
