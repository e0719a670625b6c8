"""Seeded synthetic inputs shared by the CUDA path, its tests, the bench and the oracle.

This module draws random numbers and nothing else: it holds none of the clustering
arithmetic (no scaling, no distances, no means), so that the oracle and the CUDA
library can both be fed from it without sharing any of the method.

The paper times its method on 2-D synthetic blobs with 500 points per cluster (§VI,
Table 2) that are not published; the workloads below stand in for them with the same
structure (isotropic Gaussian blobs, optionally uniform outliers) at the sizes the
benchmarks use:

* ``mixture``       -- n points, equal-probability choice among ``blobs`` isotropic
  Gaussians whose means are uniform in [0, 10]^d; a per-blob sigma is either fixed or
  uniform in ``sigma_range``; an ``outlier_frac`` share of the points is uniform in
  [-3*sigma_max, 10 + 3*sigma_max]^d.  Drawn in float64 and rounded once to float32.
* ``uneven_sizes``  -- instance sizes floor(exp(U[ln lo, ln hi])) (log-uniform).
* ``blob_points``   -- exactly ``per_blob`` points from each of ``blobs`` isotropic
  Gaussians (means uniform in [0, 10]^d, sigma uniform in ``sigma_range``), in a random
  order: the shape of the paper's timing data (2-D, 500 points per cluster, Table 2).

Every generator takes an explicit integer seed; numpy's PCG64 is the bit source.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 0x14121947


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def mixture(n: int, d: int, blobs: int, *, sigma: float | None = None,
            sigma_range: tuple[float, float] = (0.2, 1.0), outlier_frac: float = 0.0,
            seed: int = BASE_SEED, dtype=np.float32, chunk: int = 1 << 20) -> np.ndarray:
    """n x d row-major points from a seeded isotropic Gaussian mixture (+ uniform outliers)."""
    g = rng(seed)
    means = g.uniform(0.0, 10.0, size=(blobs, d))
    if sigma is not None:
        sig = np.full(blobs, float(sigma))
    else:
        sig = g.uniform(sigma_range[0], sigma_range[1], size=blobs)
    n_out = int(round(outlier_frac * n))
    n_in = n - n_out
    out = np.empty((n, d), dtype=dtype)
    done = 0
    while done < n_in:
        m = min(chunk, n_in - done)
        which = g.integers(0, blobs, size=m)
        z = g.standard_normal(size=(m, d))
        out[done:done + m] = means[which] + z * sig[which][:, None]
        done += m
    if n_out:
        smax = float(sig.max())
        lo, hi = -3.0 * smax, 10.0 + 3.0 * smax
        u = g.uniform(lo, hi, size=(n_out, d))
        out[n_in:] = u
        # interleave the outliers with the blob points so that neither end of the
        # index range is special (the peel breaks ties by index)
        perm = g.permutation(n)
        out = out[perm]
    return out


def blob_points(blobs: int, per_blob: int, d: int, *, sigma_range: tuple[float, float] = (0.2, 1.0),
                seed: int = BASE_SEED, dtype=np.float32) -> np.ndarray:
    """blobs * per_blob x d points, exactly per_blob from each blob, shuffled."""
    g = rng(seed)
    means = g.uniform(0.0, 10.0, size=(blobs, d))
    sig = g.uniform(sigma_range[0], sigma_range[1], size=blobs)
    which = np.repeat(np.arange(blobs), per_blob)
    z = g.standard_normal(size=(blobs * per_blob, d))
    pts = (means[which] + z * sig[which][:, None]).astype(dtype)
    return pts[g.permutation(blobs * per_blob)]


def uneven_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    g = rng(seed)
    return np.floor(np.exp(g.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


@dataclass(frozen=True)
class Workload:
    """One two-level clustering problem: points plus the method's parameters."""
    name: str
    n: int
    d: int
    blobs: int
    N: int            # subcluster size (Algorithm 1)
    local_k: int      # local centers per subcluster
    final_k: int      # centers of the final clustering
    iters: int        # Lloyd iterations, local and final
    sigma: float | None = None
    outlier_frac: float = 0.0
    seed: int = BASE_SEED

    def points(self) -> np.ndarray:
        return mixture(self.n, self.d, self.blobs, sigma=self.sigma,
                       outlier_frac=self.outlier_frac, seed=self.seed)


# The plain-method workload of the small configuration: 4096 points, d=4, 3 blobs with
# sigma 0.5, subclusters of 256, 16 local centers, 20 Lloyd iterations, final k=3.
SMALL = Workload("n4096_d4_N256_k16_f3", n=4096, d=4, blobs=3, N=256, local_k=16,
                 final_k=3, iters=20, sigma=0.5, seed=BASE_SEED + 0)

# The headline workload: 2^20 points, d=16, 64 blobs (sigma ~ U[0.2,1]) plus 1% uniform
# outliers; subclusters of 4096 (256 of them), 64 local centers, 25 iterations, final k=64.
MEDIUM = Workload("n1048576_d16_N4096_k64_f64", n=1 << 20, d=16, blobs=64, N=4096,
                  local_k=64, final_k=64, iters=25, outlier_frac=0.01, seed=BASE_SEED + 1)

# The precision workload: 2^24 points, d=64, 1024 blobs; N=65536, 256 local centers,
# final k=1024, 25 iterations.
LARGE = Workload("n16777216_d64_N65536_k256_f1024", n=1 << 24, d=64, blobs=1024, N=65536,
                 local_k=256, final_k=1024, iters=25, seed=BASE_SEED + 3)


def scaled_down(w: Workload, n: int, *, N: int | None = None, local_k: int | None = None,
                final_k: int | None = None, iters: int | None = None, seed: int | None = None) -> Workload:
    """The same recipe at a size the oracle finishes quickly (for parity tests)."""
    return Workload(w.name + f"_n{n}", n=n, d=w.d, blobs=w.blobs, N=N or w.N,
                    local_k=local_k or w.local_k, final_k=final_k or w.final_k,
                    iters=iters or w.iters, sigma=w.sigma, outlier_frac=w.outlier_frac,
                    seed=w.seed if seed is None else seed)


def uneven_batch(count: int = 2048, d: int = 32, lo: int = 256, hi: int = 65536,
                 seed: int = BASE_SEED + 2):
    """Independent Lloyd instances with log-uniform sizes; each instance is its own
    mixture with k = max(8, size // 256) blobs.  Returns (list of arrays, list of k)."""
    sizes = uneven_sizes(count, lo, hi, seed)
    pts, ks = [], []
    for i, m in enumerate(sizes):
        k = max(8, int(m) // 256)
        pts.append(mixture(int(m), d, k, seed=seed * 7919 + i + 1))
        ks.append(k)
    return pts, ks


def mixture_device(n: int, d: int, blobs: int, seed: int, device, sigma_range=(0.2, 1.0)):
    """The mixture recipe drawn on a CUDA device with a seeded torch generator (the job
    server's workload, where a host upload per job would dominate).  Not bit-identical to
    mixture() with the same seed: a different bit source."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    means = torch.rand((blobs, d), generator=g, device=device, dtype=torch.float64) * 10.0
    sig = sigma_range[0] + (sigma_range[1] - sigma_range[0]) * torch.rand(blobs, generator=g, device=device,
                                                                         dtype=torch.float64)
    which = torch.randint(0, blobs, (n,), generator=g, device=device)
    out = torch.empty((n, d), device=device, dtype=torch.float32)
    step = max(1, (1 << 24) // d)            # rows per chunk: float64 temporaries stay ~130 MB
    for r0 in range(0, n, step):
        r1 = min(n, r0 + step)
        z = torch.randn((r1 - r0, d), generator=g, device=device, dtype=torch.float64)
        w = which[r0:r1]
        out[r0:r1] = (means[w] + z * sig[w][:, None]).to(torch.float32)
    return out


def serving_stream(count: int, seed: int, n_range=(1e4, 1e6), dims=(8, 32, 128), k_range=(8, 1024)):
    """Job shapes of the serving workload: n and final k log-uniform, d uniform on dims,
    N = ceil(n / 64), local k = min(N, max(8, ceil(N / 256), ceil(2 final_k / S))) so that
    the pooled local centers number at least 2 final_k; 25 iterations; storage bfloat16 or
    float32 with probability 1/2 each."""
    g = rng(seed)
    jobs = []
    for i in range(count):
        n = int(math.exp(g.uniform(math.log(n_range[0]), math.log(n_range[1]))))
        d = int(g.choice(dims))
        fk = int(math.exp(g.uniform(math.log(k_range[0]), math.log(k_range[1]))))
        N = -(-n // 64)
        S = -(-n // N)
        lk = min(N, max(8, -(-N // 256), -(-2 * fk // S)))
        fk = min(fk, S * lk)
        bf16 = bool(g.random() < 0.5)
        jobs.append({"n": n, "d": d, "N": N, "local_k": lk, "final_k": fk, "iters": 25, "seed": seed * 7 + i,
                     "blobs": max(2, fk), "bf16": bf16})
    return jobs
