"""Python access to the plain C oracle (``pscl_oracle.c``).

TEST INFRASTRUCTURE: imported only by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py``.  The product library never imports it.
The oracle is compiled from its single C file with gcc at -O2 -ffp-contract=off (and
OpenMP, which it uses only to run independent subclusters side by side).
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pscl_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (skipped when up to date)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c99", "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        L.or_splitmix64_next.restype = C.c_uint64
        L.or_splitmix64_next.argtypes = [P]
        L.or_init_state.restype = C.c_uint64
        L.or_init_state.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32]
        L.or_init_indices.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int64, C.c_int32, P]
        L.or_scale.argtypes = [P, C.c_int64, C.c_int32, P, P, P]
        L.or_group_unequal.argtypes = [P, C.c_int64, C.c_int32, C.c_int32, P, P, P, P, P]
        L.or_scale_storage.argtypes = [P, C.c_int64, C.c_int32, P, P, P, C.c_int]
        L.or_peel.argtypes = [P, C.c_int64, C.c_int32, C.c_int64, P, P, P, P]
        L.or_peel_select.argtypes = [P, C.c_int64, C.c_int32, C.c_int64, P, P, P, P]
        L.or_assign.argtypes = [P, C.c_int64, C.c_int32, P, C.c_int32, P, P, P]
        L.or_lloyd.argtypes = [P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P,
                               C.c_double, P, P]
        L.or_lloyd_w.argtypes = [P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, P, P, P, P, P, P,
                                 C.c_double, P, P]
        L.or_lloyd_seeded.argtypes = [P, C.c_int64, C.c_int32, C.c_int32, C.c_int32, C.c_uint64,
                                      C.c_uint32, C.c_uint32, C.c_int, P, P, P, P]
        L.or_two_level.argtypes = [P]
        for f in ("or_init_indices", "or_scale", "or_peel", "or_peel_select", "or_assign", "or_lloyd",
                  "or_lloyd_w", "or_lloyd_seeded", "or_two_level"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with status {rc}")


def splitmix64(state: int, count: int) -> list[int]:
    s = C.c_uint64(state)
    return [lib().or_splitmix64_next(C.byref(s)) for _ in range(count)]


def init_indices(seed: int, stage: int, segment: int, m: int, k: int) -> np.ndarray:
    out = np.empty(k, np.int64)
    _check(lib().or_init_indices(seed, stage, segment, m, k, _p(out)), "init_indices")
    return out


def scale(raw: np.ndarray, bf16: bool = False):
    """Min-max scaling; bf16 rounds the scaled values to bfloat16 (kept in float32)."""
    raw = np.ascontiguousarray(raw, np.float32)
    n, d = raw.shape
    out = np.empty_like(raw)
    mn = np.empty(d, np.float64)
    mx = np.empty(d, np.float64)
    _check(lib().or_scale_storage(_p(raw), n, d, _p(out), _p(mn), _p(mx), int(bf16)), "scale")
    return out, mn, mx


def peel(x: np.ndarray, N: int, select: bool = False):
    """Returns (perm[n], seg_off[S+1], landmarks[S, d]).  select=True uses the O(n_r)
    per-round selection form (same result, for large inputs)."""
    x = np.ascontiguousarray(x, np.float32)
    n, d = x.shape
    S_max = -(-n // N)
    perm = np.empty(n, np.int64)
    seg_off = np.empty(S_max + 1, np.int64)
    lm = np.empty((S_max, d), np.float32)
    S = C.c_int64(0)
    f = lib().or_peel_select if select else lib().or_peel
    _check(f(_p(x), n, d, N, _p(perm), _p(seg_off), C.byref(S), _p(lm)), "peel")
    S = S.value
    return perm, seg_off[:S + 1].copy(), lm[:S].copy()


def group_unequal(x: np.ndarray, m: int):
    """Algorithm 2's grouping: returns (perm[n], seg_off[S+1], landmarks[m, d], group[n])."""
    x = np.ascontiguousarray(x, np.float32)
    n, d = x.shape
    perm = np.empty(n, np.int64)
    seg_off = np.empty(m + 1, np.int64)
    lm = np.empty((m, d), np.float32)
    g = np.empty(n, np.int32)
    S = C.c_int64(0)
    _check(lib().or_group_unequal(_p(x), n, d, m, _p(perm), _p(seg_off), C.byref(S), _p(lm), _p(g)),
           "group_unequal")
    return perm, seg_off[:S.value + 1].copy(), lm, g


def assign(pts: np.ndarray, centers: np.ndarray):
    pts = np.ascontiguousarray(pts, np.float32)
    c = np.ascontiguousarray(centers, np.float64)
    m, d = pts.shape
    k = c.shape[0]
    lab = np.empty(m, np.int32)
    b = np.empty(m, np.float64)
    s = np.empty(m, np.float64)
    _check(lib().or_assign(_p(pts), m, d, _p(c), k, _p(lab), _p(b), _p(s)), "assign")
    return lab, b, s


def lloyd(pts: np.ndarray, init_centers: np.ndarray, iters: int, force=None, tie_tol=0.0, weights=None):
    """Lloyd from given initial centers.  Returns (centers, labels, sse_hist, counts, n_forced, n_bad).
    weights: optional non-negative integer weight per point (weighted means, weighted SSE)."""
    pts = np.ascontiguousarray(pts, np.float32)
    c = np.array(init_centers, np.float64, order="C", copy=True)
    m, d = pts.shape
    k = c.shape[0]
    lab = np.empty(m, np.int32)
    hist = np.empty(max(iters, 1), np.float64)
    cnt = np.empty(k, np.int64)
    nf = C.c_int64(0)
    nb = C.c_int64(0)
    frc = None if force is None else np.ascontiguousarray(force, np.int32)
    w = None if weights is None else np.ascontiguousarray(weights, np.int64)
    _check(lib().or_lloyd_w(_p(pts), m, d, k, iters, _p(c), _p(lab), _p(hist), _p(cnt), _p(w), _p(frc),
                            tie_tol, C.byref(nf), C.byref(nb)), "lloyd")
    return c, lab, hist[:iters], cnt, nf.value, nb.value


def standard_kmeans(x: np.ndarray, init_centers: np.ndarray, iters: int):
    """One-level ("standard") k-means, Lloyd's algorithm as Section I describes it: every
    point goes to the center at the smallest squared Euclidean distance (the lowest index
    among equal distances), then every center moves to the mean of its points (a center
    with none stays).  The method reduces to it with one subcluster and one local center
    per point.  Written apart from the C oracle's Lloyd, in vectorised float64 numpy, so
    that the two-level oracle can be pinned against something other than itself.
    Returns (centers, labels, SSE after each iteration's update)."""
    pts = np.asarray(x, np.float64)
    c = np.array(init_centers, np.float64, copy=True)
    lab = np.zeros(len(pts), np.int64)
    hist = []
    for _ in range(iters):
        d2 = ((pts[:, None, :] - c[None, :, :]) ** 2).sum(axis=2)
        lab = d2.argmin(axis=1)
        for j in range(len(c)):
            members = pts[lab == j]
            if len(members):
                c[j] = members.mean(axis=0)
        hist.append(float(((pts - c[lab]) ** 2).sum()))
    return c, lab, np.array(hist)


def lloyd_seeded(pts: np.ndarray, k: int, iters: int, seed: int, stage: int = 0, segment: int = 0,
                 first_k: bool = False):
    pts = np.ascontiguousarray(pts, np.float32)
    m, d = pts.shape
    ke = min(k, m)
    c = np.empty((ke, d), np.float64)
    lab = np.empty(m, np.int32)
    hist = np.empty(max(iters, 1), np.float64)
    cnt = np.empty(ke, np.int64)
    _check(lib().or_lloyd_seeded(_p(pts), m, d, k, iters, seed, stage, segment, int(first_k),
                                 _p(c), _p(lab), _p(hist), _p(cnt)), "lloyd_seeded")
    return c, lab, hist[:iters], cnt


class _Args(C.Structure):
    _fields_ = [
        ("raw", C.c_void_p), ("n", C.c_int64), ("N", C.c_int64), ("d", C.c_int32),
        ("local_k", C.c_int32), ("final_k", C.c_int32), ("iters", C.c_int32),
        ("seed", C.c_uint64), ("first_k", C.c_int32), ("n_threads", C.c_int32),
        ("select_peel", C.c_int32), ("unequal_m", C.c_int32), ("storage_bf16", C.c_int32),
        ("pool_weighted", C.c_int32),
        ("force_local", C.c_void_p), ("force_final", C.c_void_p), ("tie_tol", C.c_double),
        ("scaled", C.c_void_p), ("perm", C.c_void_p), ("seg_off", C.c_void_p),
        ("landmarks", C.c_void_p), ("local_centers", C.c_void_p), ("local_k_eff", C.c_void_p),
        ("local_labels", C.c_void_p), ("local_sse", C.c_void_p), ("final_centers", C.c_void_p),
        ("final_sse_hist", C.c_void_p), ("final_labels_pooled", C.c_void_p),
        ("labels", C.c_void_p), ("best", C.c_void_p), ("second", C.c_void_p),
        ("sse", C.c_double), ("n_seg", C.c_int64), ("n_pooled", C.c_int64),
        ("n_forced", C.c_int64), ("n_bad", C.c_int64),
    ]


@dataclass
class TwoLevel:
    scaled: np.ndarray
    perm: np.ndarray
    seg_off: np.ndarray
    landmarks: np.ndarray
    local_centers: np.ndarray     # P x d (float64)
    local_k_eff: np.ndarray       # S
    local_labels: np.ndarray      # n, subcluster-packed order
    local_sse: np.ndarray         # S x iters
    final_centers: np.ndarray     # final_k x d (float64)
    final_sse_hist: np.ndarray    # iters
    final_labels_pooled: np.ndarray
    labels: np.ndarray            # n
    best: np.ndarray
    second: np.ndarray
    sse: float
    n_forced: int
    n_bad: int


def pooled_count(n: int, N: int, local_k: int) -> tuple[int, int]:
    """(S, P): number of subclusters and of pooled local centers."""
    S = -(-n // N)
    full = n // N
    P = full * min(local_k, N)
    if n % N:
        P += min(local_k, n % N)
    return S, P


def two_level(raw: np.ndarray, N: int, local_k: int, final_k: int, iters: int, seed: int,
              first_k: bool = False, threads: int = 0, force_local=None, force_final=None,
              select_peel: bool = False, unequal_m: int = 0, bf16: bool = False,
              tie_tol: float = 0.0, pool_weighted: bool = False) -> TwoLevel:
    """unequal_m > 0: Algorithm 2 with that many landmarks instead of the peel (N unused).
    pool_weighted: the pooled Lloyd weighs each local center by its cluster's size."""
    raw = np.ascontiguousarray(raw, np.float32)
    n, d = raw.shape
    if unequal_m > 0:
        N = 1
        S, P = unequal_m, min(n, unequal_m * local_k)      # upper bounds, trimmed below
    else:
        S, P = pooled_count(n, N, local_k)
    o = dict(
        scaled=np.empty((n, d), np.float32), perm=np.empty(n, np.int64),
        seg_off=np.empty(S + 1, np.int64), landmarks=np.empty((S, d), np.float32),
        local_centers=np.empty((P, d), np.float64), local_k_eff=np.empty(S, np.int32),
        local_labels=np.empty(n, np.int32), local_sse=np.empty((S, max(iters, 1)), np.float64),
        final_centers=np.empty((final_k, d), np.float64),
        final_sse_hist=np.empty(max(iters, 1), np.float64),
        final_labels_pooled=np.empty(P, np.int32), labels=np.empty(n, np.int32),
        best=np.empty(n, np.float64), second=np.empty(n, np.float64))
    fl = None if force_local is None else np.ascontiguousarray(force_local, np.int32)
    ff = None if force_final is None else np.ascontiguousarray(force_final, np.int32)
    a = _Args()
    a.raw = raw.ctypes.data
    a.n, a.N, a.d = n, N, d
    a.local_k, a.final_k, a.iters, a.seed = local_k, final_k, iters, seed
    a.first_k, a.n_threads = int(first_k), int(threads)
    a.select_peel = int(select_peel)
    a.unequal_m = int(unequal_m)
    a.storage_bf16 = int(bf16)
    a.pool_weighted = int(pool_weighted)
    a.force_local = None if fl is None else fl.ctypes.data
    a.force_final = None if ff is None else ff.ctypes.data
    a.tie_tol = tie_tol
    for k, v in o.items():
        setattr(a, k, v.ctypes.data)
    _check(lib().or_two_level(C.byref(a)), "two_level")
    if unequal_m > 0:
        S, P = a.n_seg, a.n_pooled
        o["seg_off"] = o["seg_off"][:S + 1]
        o["local_centers"] = o["local_centers"][:P]
        o["local_k_eff"] = o["local_k_eff"][:S]
        o["local_sse"] = o["local_sse"][:S]
        o["final_labels_pooled"] = o["final_labels_pooled"][:P]
    elif a.n_seg != S or a.n_pooled != P:
        raise RuntimeError("oracle subcluster count disagrees with the closed form")
    o["local_sse"] = o["local_sse"][:, :iters]
    o["final_sse_hist"] = o["final_sse_hist"][:iters]
    return TwoLevel(sse=a.sse, n_forced=a.n_forced, n_bad=a.n_bad, **o)
