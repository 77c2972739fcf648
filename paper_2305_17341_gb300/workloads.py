"""Seeded synthetic inputs shaped like the paper's workloads.

Only input generation lives here (NumPy PCG64 streams); no part of the
homomorphic method.  Both the tests' oracle side and the CUDA side draw from
these functions, so the same bytes reach both.

The paper's datasets (MNIST, Fashion-MNIST, Yale; Sec. 7.2.3) are not
available; the low-rank-plus-noise matrices below stand in for them with the
paper's shapes (s samples x 256 pixel features in [0, 1]).
"""
import numpy as np


def matmul_pair(n, seed):
    """A, B: n x n, entries i.i.d. uniform[-1, 1] (products of Sec. 4, Table 3)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, (n, n)), rng.uniform(-1.0, 1.0, (n, n))


def lowrank_dataset(s, t, seed, decay=0.8, noise=0.01):
    """X = U diag(decay^i) V^T + noise * N(0, 1), U, V random orthogonal (QR of
    Gaussian matrices, sign-fixed), globally min-max scaled to [0, 1]."""
    rng = np.random.default_rng(seed)
    k = min(s, t)
    U, Ru = np.linalg.qr(rng.standard_normal((s, k)))
    U = U * np.sign(np.diag(Ru))
    V, Rv = np.linalg.qr(rng.standard_normal((t, k)))
    V = V * np.sign(np.diag(Rv))
    X = (U * decay ** np.arange(k)) @ V.T + noise * rng.standard_normal((s, t))
    X = (X - X.min()) / (X.max() - X.min())
    return X


def mixed_matmul_jobs(count, seed, dims=(16, 32, 64, 128), logNs=(15, 16), levels=(3, 20)):
    """Jobs of a mixed batch: (n, logN, level, A, B) with n, logN, level drawn
    uniformly; entries uniform[-1, 1]."""
    rng = np.random.default_rng(seed)
    jobs = []
    for _ in range(count):
        n = int(rng.choice(dims))
        logN = int(rng.choice(logNs))
        level = int(rng.integers(levels[0], levels[1] + 1))
        A = rng.uniform(-1.0, 1.0, (n, n))
        B = rng.uniform(-1.0, 1.0, (n, n))
        jobs.append((n, logN, level, A, B))
    return jobs


def poisson_arrivals(rate, duration, seed):
    """Arrival times (s) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            return out
        out.append(t)


def served_job_mix(rate, duration, seed, weights=(("xtx_block", 0.55), ("matmul", 0.25), ("covariance", 0.12),
                                                  ("covariance_large", 0.03), ("pca", 0.05)), max_xtx=None):
    """A served workload: Poisson arrivals, each labelled with a job kind drawn
    from `weights`.  With max_xtx, at most that many arrivals are row blocks
    ("xtx_block") of the streamed dataset; later draws of that kind become
    "covariance".  Returns [(t, kind)] in arrival order."""
    ts = poisson_arrivals(rate, duration, seed)
    rng = np.random.default_rng(seed + 1)
    kinds = [k for k, _ in weights]
    p = np.array([w for _, w in weights], dtype=float)
    p /= p.sum()
    out, nx = [], 0
    for t in ts:
        kind = kinds[int(rng.choice(len(kinds), p=p))]
        if kind == "xtx_block" and max_xtx is not None:
            if nx >= max_xtx:
                kind = "covariance"
            else:
                nx += 1
        out.append((t, kind))
    return out


# The served configuration's mix: one 60000 x 256 dataset streamed as its
# 469 row blocks of 128 x 256 (the last zero-padded), 256 x 256 and
# 4096 x 256 covariances and top-k PCA jobs; at 4 jobs/s over 120 s the
# expected number of row-block arrivals (0.97 x 480) is about the dataset's
# 469 blocks.
SERVED_STREAM_WEIGHTS = (("xtx_block", 0.97), ("covariance", 0.015), ("covariance_large", 0.005), ("pca", 0.01))
