"""Thin Python binding of the pscl C ABI (include/pscl.h).

Every function has the name of the C entry point it calls and only marshals arguments
(numpy arrays or torch CUDA tensors in, numpy arrays out); all work runs in the CUDA
library.  There is no other code path: if libpscl.so is missing or cannot be loaded,
``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpscl.so")

PSCL_OK, PSCL_EINVAL, PSCL_ESTATE, PSCL_ENOMEM, PSCL_EBUSY, PSCL_ETIMEOUT, PSCL_ECUDA = range(7)
PSCL_F32, PSCL_BF16 = 0, 1
PSCL_PREC_FP32, PSCL_PREC_TF32, PSCL_PREC_BF16, PSCL_PREC_TF32X3, PSCL_PREC_BF16X3 = 0, 1, 2, 3, 4
PSCL_PREC_TC = 5
PRECISIONS = {"fp32": PSCL_PREC_FP32, "tf32": PSCL_PREC_TF32, "bf16": PSCL_PREC_BF16,
              "tf32x3": PSCL_PREC_TF32X3, "bf16x3": PSCL_PREC_BF16X3, "tc": PSCL_PREC_TC}
PSCL_OPT_PLAIN_LLOYD, PSCL_OPT_TRACE_LABELS, PSCL_OPT_INIT_FIRST_K, PSCL_OPT_GRAPH = 1, 2, 3, 4
PSCL_OPT_KERNEL_TIMING, PSCL_OPT_UNIT_ROWS, PSCL_OPT_ROWS_PER_THREAD, PSCL_OPT_POOL_WEIGHTED = 5, 6, 7, 8
PSCL_OPT_PEEL_ROUNDS, PSCL_OPT_WAIT_LIMIT, PSCL_OPT_TEST_STALL, PSCL_OPT_PEEL_GRID = 9, 10, 11, 12

# entry point -> (restype, argtypes); the list is the C ABI of include/pscl.h
_P, _I, _I32, _I64, _U64, _SZ = C.c_void_p, C.c_int, C.c_int32, C.c_int64, C.c_uint64, C.c_size_t
SIGNATURES = {
    "pscl_ctx_create": (_I, [_P, _I, _SZ, _P]),
    "pscl_ctx_destroy": (_I, [_P]),
    "pscl_ctx_bytes_in_use": (_SZ, [_P]),
    "pscl_last_error": (C.c_char_p, []),
    "pscl_job_create": (_I, [_P, _P, _I, _I64, _I32, _I, _P]),
    "pscl_job_load": (_I, [_P, _P, _I]),
    "pscl_job_set_option": (_I, [_P, _I, _I64]),
    "pscl_job_destroy": (_I, [_P]),
    "pscl_scale_features": (_I, [_P]),
    "pscl_subcluster": (_I, [_P, _I64, _I32, _I32, _U64, _I]),
    "pscl_subcluster_unequal": (_I, [_P, _I32, _I32, _I32, _U64, _I]),
    "pscl_cluster": (_I, [_P, _I32, _I32, _U64, _I]),
    "pscl_run": (_I, [_P, _I64, _I32, _I32, _I32, _U64, _I]),
    "pscl_job_sync": (_I, [_P]),
    "pscl_get_scaled": (_I, [_P, _P]),
    "pscl_get_sizes": (_I, [_P, _P, _P]),
    "pscl_get_partition": (_I, [_P, _P, _P, _P]),
    "pscl_get_local_centers": (_I, [_P, _P, _P, _P]),
    "pscl_get_result": (_I, [_P, _P, _P, _P]),
    "pscl_get_label_trace": (_I, [_P, _I, _P]),
    "pscl_get_phase_ms": (_I, [_P, _P]),
    "pscl_get_kernel_times": (_I, [_P, _P, _P]),
    "pscl_get_recheck_stats": (_I, [_P, _P, _P]),
    "pscl_get_peel_stats": (_I, [_P, _P, _P, _P, _P]),
    "pscl_measure_grid_barrier": (_I, [_I, _P]),
    "pscl_measure_fp32_fma": (_I, [_I, _P]),
    "pscl_assign_sse_noalloc": (_I, [_P, _I64, _I32, _P, _I32, _P, _P, _P]),
    "pscl_job_footprint": (_I, [_P, _I64, _I32, _I64, _I32, _I32, _I32, _I, _I, _I, _P]),
    "pscl_server_create": (_I, [_P, _I32, _SZ, _P]),
    "pscl_submit": (_I, [_P, _P, _P]),
    "pscl_poll": (_I, [_P, _U64, _P]),
    "pscl_wait": (_I, [_P, _U64, _I64]),
    "pscl_fetch": (_I, [_P, _U64, _P, _P, _P, _P]),
    "pscl_server_stats": (_I, [_P, _P]),
    "pscl_server_destroy": (_I, [_P]),
    "pscl_batch_create": (_I, [_P, _P, _I, _I32, _I32, _P, _P, _P]),
    "pscl_batch_load": (_I, [_P, _P, _I]),
    "pscl_batch_set_option": (_I, [_P, _I, _I64]),
    "pscl_batch_tune": (_I, [_P, _I32, _I, _P, _P, _P]),
    "pscl_batch_run": (_I, [_P, _I32, _U64, _I]),
    "pscl_batch_sync": (_I, [_P]),
    "pscl_batch_get": (_I, [_P, _P, _P, _P]),
    "pscl_batch_get_scaled": (_I, [_P, _P]),
    "pscl_batch_get_label_trace": (_I, [_P, _P]),
    "pscl_batch_lloyd_ms": (_I, [_P, _P]),
    "pscl_batch_launches": (_I, [_P, _P]),
    "pscl_batch_destroy": (_I, [_P]),
}
PSCL_JOB_QUEUED, PSCL_JOB_RUNNING, PSCL_JOB_DONE, PSCL_JOB_FAILED = 0, 1, 2, 3


class JobDesc(C.Structure):
    """pscl_job_desc"""
    _fields_ = [("points", C.c_void_p), ("on_device", C.c_int32), ("dtype", C.c_int32), ("n", C.c_int64),
                ("d", C.c_int32), ("N", C.c_int64), ("local_k", C.c_int32), ("final_k", C.c_int32),
                ("iters", C.c_int32), ("seed", C.c_uint64), ("prec", C.c_int32), ("want_labels", C.c_int32)]


KERNELS = ["scale_minmax", "scale_apply", "peel", "gather", "lloyd_init", "lloyd_assign", "lloyd_finalize",
           "final_sse", "lloyd_sums"]

_lib = None


class PsclError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pscl error {code}: {msg}")
        self.code = code


def lib():
    """The loaded CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _chk(rc):
    if rc != PSCL_OK:
        raise PsclError(rc, lib().pscl_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()       # torch tensor


def _points(points):
    """(pointer, on_device, n, d, keep-alive) for a numpy array or a torch tensor:
    float32, or bfloat16 (torch.bfloat16, or numpy uint16 holding bfloat16 bits)."""
    if isinstance(points, np.ndarray):
        a = np.ascontiguousarray(points, dtype=np.uint16 if points.dtype == np.uint16 else np.float32)
        return a.ctypes.data, 0, a.shape[0], a.shape[1], a
    t = points
    if t.dtype.itemsize not in (2, 4) or not t.is_contiguous() or t.dim() != 2:
        raise ValueError("points must be a contiguous 2-D float32 or bfloat16 tensor")
    return t.data_ptr(), 1 if t.is_cuda else 0, t.shape[0], t.shape[1], t


def _dtype(points):
    """PSCL_BF16 for bfloat16 points (torch.bfloat16 or numpy uint16 bits), else PSCL_F32."""
    if isinstance(points, np.ndarray):
        return PSCL_BF16 if points.dtype == np.uint16 else PSCL_F32
    return PSCL_BF16 if points.dtype.itemsize == 2 else PSCL_F32


# ---------------------------------------------------------------- C entry points
def pscl_ctx_create(device=0, hbm_budget_bytes=0, stream=None):
    h = C.c_void_p()
    _chk(lib().pscl_ctx_create(C.byref(h), device, hbm_budget_bytes, stream))
    return h


def pscl_ctx_destroy(ctx):
    _chk(lib().pscl_ctx_destroy(ctx))


def pscl_ctx_bytes_in_use(ctx):
    return lib().pscl_ctx_bytes_in_use(ctx)


def pscl_job_create(ctx, points, dtype=None):
    p, dev, n, d, keep = _points(points)
    dtype = _dtype(points) if dtype is None else dtype
    h = C.c_void_p()
    _chk(lib().pscl_job_create(ctx, p, dtype, n, d, dev, C.byref(h)))
    return h, keep


def pscl_job_load(job, points):
    p, dev, _, _, keep = _points(points)
    _chk(lib().pscl_job_load(job, p, dev))
    return keep


def pscl_job_set_option(job, option, value):
    _chk(lib().pscl_job_set_option(job, option, int(value)))


def pscl_job_destroy(job):
    _chk(lib().pscl_job_destroy(job))


def pscl_scale_features(job):
    _chk(lib().pscl_scale_features(job))


def pscl_subcluster(job, N, local_k, iters, seed, prec=PSCL_PREC_FP32):
    _chk(lib().pscl_subcluster(job, N, local_k, iters, seed, prec))


def pscl_subcluster_unequal(job, m, local_k, iters, seed, prec=PSCL_PREC_FP32):
    _chk(lib().pscl_subcluster_unequal(job, m, local_k, iters, seed, prec))


def pscl_cluster(job, final_k, iters, seed, prec=PSCL_PREC_FP32):
    _chk(lib().pscl_cluster(job, final_k, iters, seed, prec))


def pscl_run(job, N, local_k, final_k, iters, seed, prec=PSCL_PREC_FP32):
    _chk(lib().pscl_run(job, N, local_k, final_k, iters, seed, prec))


def pscl_job_sync(job):
    _chk(lib().pscl_job_sync(job))


def pscl_get_sizes(job):
    s, p = C.c_int64(), C.c_int64()
    _chk(lib().pscl_get_sizes(job, C.byref(s), C.byref(p)))
    return s.value, p.value


def pscl_get_scaled(job, n, d):
    out = np.empty((n, d), np.float32)
    _chk(lib().pscl_get_scaled(job, _ptr(out)))
    return out


def pscl_get_partition(job, n):
    S, _ = pscl_get_sizes(job)
    perm = np.empty(n, np.int64)
    off = np.empty(S + 1, np.int64)
    ns = C.c_int64()
    _chk(lib().pscl_get_partition(job, _ptr(perm), _ptr(off), C.byref(ns)))
    return perm, off


def pscl_get_local_centers(job, d):
    S, P = pscl_get_sizes(job)
    c = np.empty((P, d), np.float32)
    ke = np.empty(S, np.int32)
    cnt = np.empty(P, np.int32)
    _chk(lib().pscl_get_local_centers(job, _ptr(c), _ptr(ke), _ptr(cnt)))
    return c, ke, cnt


def pscl_get_result(job, final_k, d, n=None):
    c = np.empty((final_k, d), np.float32)
    lab = None if n is None else np.empty(n, np.int32)
    sse = C.c_double()
    _chk(lib().pscl_get_result(job, _ptr(c), _ptr(lab), C.byref(sse)))
    return c, lab, sse.value


def pscl_get_label_trace(job, stage, length):
    out = np.empty(length, np.int32)
    _chk(lib().pscl_get_label_trace(job, stage, _ptr(out)))
    return out


def pscl_get_phase_ms(job):
    ms = np.empty(5, np.float32)
    _chk(lib().pscl_get_phase_ms(job, _ptr(ms)))
    return ms


def pscl_measure_fp32_fma(device=0):
    """Measured float32 FMA throughput of the device in TFLOP/s (2 flops per FMA)."""
    t = C.c_double()
    _chk(lib().pscl_measure_fp32_fma(device, C.byref(t)))
    return t.value


def pscl_get_recheck_stats(job):
    a, b = C.c_int64(), C.c_int64()
    _chk(lib().pscl_get_recheck_stats(job, C.byref(a), C.byref(b)))
    return a.value, b.value


def pscl_get_peel_stats(job):
    """(epochs, distance passes, passes that updated the keys, grid barriers) of the last peel."""
    a, b, c, e = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    _chk(lib().pscl_get_peel_stats(job, C.byref(a), C.byref(b), C.byref(c), C.byref(e)))
    return a.value, b.value, c.value, e.value


def pscl_measure_grid_barrier(device=0):
    """Microseconds per grid barrier of the peel's implementation, in its launch shape."""
    t = C.c_double()
    _chk(lib().pscl_measure_grid_barrier(device, C.byref(t)))
    return t.value


def pscl_get_kernel_times(job):
    """{kernel name: (launches, total ms)} of the last run."""
    n = np.empty(len(KERNELS), np.int64)
    ms = np.empty(len(KERNELS), np.float32)
    _chk(lib().pscl_get_kernel_times(job, _ptr(n), _ptr(ms)))
    return {k: (int(n[i]), float(ms[i])) for i, k in enumerate(KERNELS)}


def pscl_assign_sse_noalloc(points, centers, labels, sse, stream=None):
    """points (n x d float32), centers (k x d float32), labels (n int32) and sse (1 double)
    are CUDA tensors of the current device; nothing is allocated by the library."""
    n, d = points.shape
    k = centers.shape[0]
    _chk(lib().pscl_assign_sse_noalloc(points.data_ptr(), n, d, centers.data_ptr(), k,
                                       labels.data_ptr(), sse.data_ptr(), stream))


def pscl_job_footprint(ctx, n, d, N, local_k, final_k, iters, on_device=True, trace=False, dtype=PSCL_F32):
    b = C.c_size_t()
    _chk(lib().pscl_job_footprint(ctx, n, d, N, local_k, final_k, iters, dtype, int(on_device), int(trace),
                                  C.byref(b)))
    return b.value


def pscl_server_create(ctx, slots, hbm_budget_bytes=0):
    h = C.c_void_p()
    _chk(lib().pscl_server_create(ctx, slots, hbm_budget_bytes, C.byref(h)))
    return h


def pscl_submit(server, points, N, local_k, final_k, iters, seed, prec=PSCL_PREC_FP32, want_labels=False):
    """Queues a job; returns (ticket, keep-alive of the points)."""
    p, dev, n, d, keep = _points(points)
    desc = JobDesc(p, dev, _dtype(points), n, d, N, local_k, final_k, iters, seed, prec, int(want_labels))
    t = C.c_uint64()
    _chk(lib().pscl_submit(server, C.byref(desc), C.byref(t)))
    return t.value, keep


def pscl_poll(server, ticket):
    st = C.c_int32()
    _chk(lib().pscl_poll(server, ticket, C.byref(st)))
    return st.value


def pscl_wait(server, ticket, timeout_us=-1):
    _chk(lib().pscl_wait(server, ticket, timeout_us))


def pscl_fetch(server, ticket, final_k, d, n=None):
    c = np.empty((final_k, d), np.float32)
    lab = None if n is None else np.empty(n, np.int32)
    sse = C.c_double()
    times = np.empty(3, np.float64)
    _chk(lib().pscl_fetch(server, ticket, _ptr(c), _ptr(lab), C.byref(sse), _ptr(times)))
    return c, lab, sse.value, times


def pscl_server_stats(server):
    out = np.empty(8, np.int64)
    _chk(lib().pscl_server_stats(server, _ptr(out)))
    keys = ["completed", "failed", "queued", "running", "bytes_in_use", "peak_bytes", "max_running", "budget"]
    return dict(zip(keys, (int(v) for v in out)))


def pscl_server_destroy(server):
    _chk(lib().pscl_server_destroy(server))


def pscl_batch_create(ctx, points, sizes, k):
    """points: rows x d (numpy float32, or a torch CUDA tensor), sizes / k per instance."""
    p, dev, rows, d, keep = _points(points)
    sz = np.ascontiguousarray(sizes, np.int64)
    kk = np.ascontiguousarray(k, np.int32)
    if sz.shape != kk.shape or int(sz.sum()) != rows:
        raise ValueError("sizes and k need one entry per instance and sizes must add up to the rows")
    h = C.c_void_p()
    _chk(lib().pscl_batch_create(ctx, p, dev, d, len(sz), _ptr(sz), _ptr(kk), C.byref(h)))
    return h, keep


def pscl_batch_load(b, points):
    p, dev, _, _, keep = _points(points)
    _chk(lib().pscl_batch_load(b, p, dev))
    return keep


def pscl_batch_set_option(b, option, value):
    _chk(lib().pscl_batch_set_option(b, option, int(value)))


def pscl_batch_tune(b, iters, prec=PSCL_PREC_FP32):
    u, r, c = C.c_int64(), C.c_int32(), C.c_int32()
    _chk(lib().pscl_batch_tune(b, iters, prec, C.byref(u), C.byref(r), C.byref(c)))
    return u.value, r.value, bool(c.value)


def pscl_batch_run(b, iters, seed, prec=PSCL_PREC_FP32):
    _chk(lib().pscl_batch_run(b, iters, seed, prec))


def pscl_batch_sync(b):
    _chk(lib().pscl_batch_sync(b))


def pscl_batch_get(b, P, rows, n_inst, d, labels=True):
    c = np.empty((P, d), np.float32)
    lab = np.empty(rows, np.int32) if labels else None
    sse = np.empty(n_inst, np.float64)
    _chk(lib().pscl_batch_get(b, _ptr(c), _ptr(lab), _ptr(sse)))
    return c, lab, sse


def pscl_batch_get_scaled(b, rows, d):
    out = np.empty((rows, d), np.float32)
    _chk(lib().pscl_batch_get_scaled(b, _ptr(out)))
    return out


def pscl_batch_get_label_trace(b, iters, rows):
    out = np.empty(iters * rows, np.int32)
    _chk(lib().pscl_batch_get_label_trace(b, _ptr(out)))
    return out.reshape(iters, rows)


def pscl_batch_lloyd_ms(b):
    ms = C.c_float()
    _chk(lib().pscl_batch_lloyd_ms(b, C.byref(ms)))
    return ms.value


def pscl_batch_launches(b):
    n = C.c_int64()
    _chk(lib().pscl_batch_launches(b, C.byref(n)))
    return n.value


def pscl_batch_destroy(b):
    _chk(lib().pscl_batch_destroy(b))


# ---------------------------------------------------------------- convenience
class Server:
    """Continuous-batching job server (a light owner of the handles)."""

    def __init__(self, slots=4, hbm_budget_bytes=0, device=0, ctx=None):
        self._own_ctx = ctx is None
        self.ctx = pscl_ctx_create(device) if ctx is None else ctx
        self.h = pscl_server_create(self.ctx, slots, hbm_budget_bytes)
        self._jobs = {}

    def submit(self, points, N, local_k, final_k, iters, seed, prec=PSCL_PREC_FP32, want_labels=False):
        t, keep = pscl_submit(self.h, points, N, local_k, final_k, iters, seed, prec, want_labels)
        self._jobs[t] = (keep, final_k, int(points.shape[1]), int(points.shape[0]) if want_labels else None)
        return t

    def poll(self, ticket):
        return pscl_poll(self.h, ticket)

    def wait(self, ticket, timeout_us=-1):
        pscl_wait(self.h, ticket, timeout_us)

    def fetch(self, ticket):
        _, fk, d, n = self._jobs.pop(ticket)
        return pscl_fetch(self.h, ticket, fk, d, n)

    def stats(self):
        return pscl_server_stats(self.h)

    def footprint(self, n, d, N, local_k, final_k, iters, on_device=True):
        return pscl_job_footprint(self.ctx, n, d, N, local_k, final_k, iters, on_device)

    def close(self):
        if self.h is not None:
            pscl_server_destroy(self.h)
            self.h = None
        if self._own_ctx and self.ctx is not None:
            pscl_ctx_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Independent clustering instances of uneven sizes (a light owner of the handles)."""

    def __init__(self, points, sizes, k, device=0, hbm_budget_bytes=0, stream=None, ctx=None):
        self._own_ctx = ctx is None
        self.ctx = pscl_ctx_create(device, hbm_budget_bytes, stream) if ctx is None else ctx
        self.h, self._keep = pscl_batch_create(self.ctx, points, sizes, k)
        self.sizes = np.asarray(sizes, np.int64)
        self.k = np.minimum(np.asarray(k, np.int64), self.sizes)
        self.rows, self.d = int(points.shape[0]), int(points.shape[1])
        self.iters = 0

    def option(self, opt, value=1):
        pscl_batch_set_option(self.h, opt, value)
        return self

    def load(self, points):
        self._keep = pscl_batch_load(self.h, points)

    def tune(self, iters=3, prec=PSCL_PREC_FP32):
        return pscl_batch_tune(self.h, iters, prec)

    def run(self, iters, seed, prec=PSCL_PREC_FP32):
        pscl_batch_run(self.h, iters, seed, prec)
        self.iters = iters

    def sync(self):
        pscl_batch_sync(self.h)

    def result(self, labels=True):
        return pscl_batch_get(self.h, int(self.k.sum()), self.rows, len(self.sizes), self.d, labels)

    def scaled(self):
        return pscl_batch_get_scaled(self.h, self.rows, self.d)

    def trace(self):
        return pscl_batch_get_label_trace(self.h, self.iters, self.rows)

    def lloyd_ms(self):
        return pscl_batch_lloyd_ms(self.h)

    def launches(self):
        return pscl_batch_launches(self.h)

    def close(self):
        if self.h is not None:
            pscl_batch_destroy(self.h)
            self.h = None
        if self._own_ctx and self.ctx is not None:
            pscl_ctx_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Job:
    """One clustering problem on one device (a light owner of the C handles)."""

    def __init__(self, points, device=0, hbm_budget_bytes=0, stream=None, ctx=None):
        self._own_ctx = ctx is None
        self.ctx = pscl_ctx_create(device, hbm_budget_bytes, stream) if ctx is None else ctx
        self.h, self._keep = pscl_job_create(self.ctx, points)
        self.n, self.d = int(points.shape[0]), int(points.shape[1])
        self.final_k = None

    def option(self, opt, value=1):
        pscl_job_set_option(self.h, opt, value)
        return self

    def load(self, points):
        self._keep = pscl_job_load(self.h, points)

    def run(self, N, local_k, final_k, iters, seed, prec=PSCL_PREC_FP32):
        pscl_run(self.h, N, local_k, final_k, iters, seed, prec)
        self.final_k = final_k

    def steps(self, N, local_k, final_k, iters, seed, prec=PSCL_PREC_FP32):
        pscl_scale_features(self.h)
        pscl_subcluster(self.h, N, local_k, iters, seed, prec)
        pscl_cluster(self.h, final_k, iters, seed, prec)
        self.final_k = final_k

    def steps_unequal(self, m, local_k, final_k, iters, seed, prec=PSCL_PREC_FP32):
        """Algorithm 2 in place of the peel: m landmarks along the segment from L to H."""
        pscl_scale_features(self.h)
        pscl_subcluster_unequal(self.h, m, local_k, iters, seed, prec)
        pscl_cluster(self.h, final_k, iters, seed, prec)
        self.final_k = final_k

    def scaled(self):
        return pscl_get_scaled(self.h, self.n, self.d)

    def partition(self):
        return pscl_get_partition(self.h, self.n)

    def local_centers(self):
        return pscl_get_local_centers(self.h, self.d)

    def result(self, labels=True):
        return pscl_get_result(self.h, self.final_k, self.d, self.n if labels else None)

    def sizes(self):
        return pscl_get_sizes(self.h)

    def trace(self, stage, iters):
        S, P = self.sizes()
        return pscl_get_label_trace(self.h, stage, iters * (self.n if stage == 0 else P)).reshape(iters, -1)

    def phase_ms(self):
        return pscl_get_phase_ms(self.h)

    def kernel_times(self):
        return pscl_get_kernel_times(self.h)

    def recheck_stats(self):
        return pscl_get_recheck_stats(self.h)

    def peel_stats(self):
        return pscl_get_peel_stats(self.h)

    def close(self):
        if self.h is not None:
            pscl_job_destroy(self.h)
            self.h = None
        if self._own_ctx and self.ctx is not None:
            pscl_ctx_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
