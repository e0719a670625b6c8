"""The bounded device-side waits give up cleanly (the device-side peel loop's and the
tensor-core assignment's error paths).

Every grid-barrier wait of the peel polls at most PSCL_OPT_WAIT_LIMIT times; the test hook
PSCL_OPT_TEST_STALL makes the first barrier wait for one arrival more than the grid gives,
so that wait must run out.  Nothing faults: the CTA that gives up sets the abort flag, the
others leave at their next wait, the launch ends, and the host reads PSCL_ETIMEOUT.  The
context and the job stay usable: the next run gives the oracle's partition (Algorithm 1
steps 2-5)."""
import time

import numpy as np
import pytest

import oracle
from paper_1412_1947_gb300 import binding as B
from paper_1412_1947_gb300 import synth

pytestmark = pytest.mark.gpu


def _expect_timeout(job, N):
    t0 = time.perf_counter()
    with pytest.raises(B.PsclError) as e:
        job.steps(N, 8, 8, 2, 3)
        job.partition()
    assert e.value.code == B.PSCL_ETIMEOUT, str(e.value)
    return time.perf_counter() - t0


def test_peel_barrier_gives_up_and_the_context_stays_usable():
    raw = synth.mixture(20000, 8, 6, outlier_frac=0.01, seed=31)
    N = 1024
    ctx = B.pscl_ctx_create(0, 0, None)
    try:
        with B.Job(raw, ctx=ctx) as j:
            j.option(B.PSCL_OPT_TEST_STALL, 1).option(B.PSCL_OPT_WAIT_LIMIT, 1 << 12)
            assert _expect_timeout(j, N) < 30.0
            # the same job, the hook off: a clean run
            j.option(B.PSCL_OPT_TEST_STALL, 0).option(B.PSCL_OPT_WAIT_LIMIT, 0)
            j.steps(N, 8, 8, 2, 3)
            perm, off = j.partition()
            x = j.scaled()
        operm, ooff, _ = oracle.peel(x, N)
        np.testing.assert_array_equal(off, ooff)
        np.testing.assert_array_equal(perm, operm)
        # a fresh job on the same context
        with B.Job(raw, ctx=ctx) as j:
            j.steps(N, 8, 8, 2, 3)
            perm2, _ = j.partition()
        np.testing.assert_array_equal(perm2, operm)
    finally:
        B.pscl_ctx_destroy(ctx)


def test_tensor_core_wait_gives_up_and_the_context_stays_usable():
    # PSCL_OPT_TEST_STALL = 2: in every tensor-core assignment CTA one thread waits on an
    # mbarrier that nothing completes before any copy or MMA is issued; the wait runs out,
    # the CTA leaves through its abort path (TMEM freed), the host reads PSCL_ETIMEOUT, and
    # the next run on the same job equals the float32 direct path
    raw = synth.mixture(30000, 16, 6, outlier_frac=0.01, seed=33)
    N, lk, fk, T = 4096, 32, 16, 3
    ctx = B.pscl_ctx_create(0, 0, None)
    try:
        with B.Job(raw, ctx=ctx) as j:
            j.option(B.PSCL_OPT_TEST_STALL, 2).option(B.PSCL_OPT_WAIT_LIMIT, 1 << 12)
            t0 = time.perf_counter()
            with pytest.raises(B.PsclError) as e:
                j.steps(N, lk, fk, T, 3, B.PSCL_PREC_BF16X3)
                j.partition()
            assert e.value.code == B.PSCL_ETIMEOUT, str(e.value)
            assert time.perf_counter() - t0 < 30.0
            j.option(B.PSCL_OPT_TEST_STALL, 0).option(B.PSCL_OPT_WAIT_LIMIT, 0)
            j.steps(N, lk, fk, T, 3, B.PSCL_PREC_BF16X3)
            c_tc, l_tc, s_tc = j.result()
            assert j.recheck_stats()[1] > 0          # the tensor cores assigned rows
        with B.Job(raw, ctx=ctx) as j:
            j.steps(N, lk, fk, T, 3)
            c_fp, l_fp, s_fp = j.result()
        np.testing.assert_array_equal(c_tc, c_fp)
        np.testing.assert_array_equal(l_tc, l_fp)
        assert s_tc == s_fp
    finally:
        B.pscl_ctx_destroy(ctx)
