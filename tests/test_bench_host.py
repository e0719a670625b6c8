"""Host-side logic of bench.py that needs no GPU."""


def test_oracle_samples_pool_enough_centers():
    """The bench's CPU baseline runs the whole method on a sample of each workload: the
    sample must hold enough subclusters for their local centers to seed final_k."""
    import bench
    from paper_1412_1947_gb300 import synth
    for w in (synth.SMALL, synth.MEDIUM, synth.LARGE):
        ws = bench.oracle_sample(w, 1 << 17)
        subclusters = -(-ws.n // ws.N)
        assert subclusters * min(ws.local_k, ws.N) >= ws.final_k, w.name
        assert (ws.d, ws.N, ws.local_k, ws.final_k, ws.iters) == (w.d, w.N, w.local_k, w.final_k, w.iters)


def test_measured_peaks_are_read():
    """The rooflines divide by the machine's measured peaks when the file is there."""
    import bench
    p = bench.measured_peaks()
    assert p["kind"] in ("measured", "fallback")
    assert p["hbm_gbs"] > 1000 and p["bf16_tflops"] > 100 and p["bf16_tflops_sustained"] > 100
