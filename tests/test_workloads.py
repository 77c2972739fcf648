"""Seeded input generators: determinism, shapes and the arrival process."""
import numpy as np

from paper_2305_17341_gb300 import workloads


def test_generators_are_seeded():
    a = workloads.lowrank_dataset(64, 32, 3)
    assert np.array_equal(a, workloads.lowrank_dataset(64, 32, 3))
    assert a.shape == (64, 32) and a.min() == 0.0 and a.max() == 1.0
    A, B = workloads.matmul_pair(16, 1)
    assert A.shape == B.shape == (16, 16) and np.abs(A).max() <= 1.0


def test_lowrank_spectrum_decays():
    X = workloads.lowrank_dataset(256, 64, 2)
    Xc = X - X.mean(0)
    w = np.linalg.eigvalsh(Xc.T @ Xc)[::-1]
    # singular values follow 0.8^i above the noise floor: ratio of eigenvalues ~ 0.64
    r = w[1:6] / w[:5]
    assert np.all((r > 0.4) & (r < 0.9))


def test_poisson_arrivals_rate_and_order():
    ts = workloads.poisson_arrivals(4.0, 500.0, 5)
    assert all(0 < x < 500 for x in ts) and ts == sorted(ts)
    assert abs(len(ts) / 500.0 - 4.0) < 0.3          # 2000 expected, sd ~ 45
    gaps = np.diff([0.0] + ts)
    assert abs(gaps.mean() - 0.25) < 0.02


def test_served_mix_kinds():
    mix = workloads.served_job_mix(4.0, 300.0, 9)
    kinds = [k for _, k in mix]
    assert set(kinds) <= {"xtx_block", "matmul", "covariance", "covariance_large", "pca"}
    frac = kinds.count("xtx_block") / len(kinds)
    assert 0.45 < frac < 0.65
    assert mix == workloads.served_job_mix(4.0, 300.0, 9)


def test_mixed_jobs_ranges():
    jobs = workloads.mixed_matmul_jobs(96, 4)
    assert len(jobs) == 96
    for n, logN, level, A, B in jobs:
        assert n in (16, 32, 64, 128) and logN in (15, 16) and 3 <= level <= 20
        assert A.shape == (n, n)
