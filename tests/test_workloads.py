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


def test_multsum_tuner_picks_are_read_from_the_log():
    """bench.py reports, per (level, items, rotations), the fastest plan of
    the MultSum tuner's log lines, and the fused C^k kernel's separately."""
    import bench
    log = "\n".join([
        "multsum level 20 B 8 G 15 chunk 8 BI 8 stream 0 ms 2.5000",
        "multsum level 20 B 8 G 15 chunk 4 BI 116 stream 0 ms 2.1000",
        "multsum level 18 B 8 G 1 chunk 1 BI 184 stream 0 ms 0.3000",
        "multsum level 18 B 8 G 1 chunk 1 BI 4 stream 1 ms 0.4000",
        "multsum_ck level 19 B 8 G 15 chunk 4 BI 8 ms 7.1000",
        "multsum_ck level 19 B 8 G 15 chunk 8 BI 0 ms 7.5000",
        "ntt forward logN 16 rows 1024 ctas_per_sm 3 ms 0.7469",
    ])
    assert bench.multsum_picks(log) == [
        "level 18 B 8 G 1: 1 keys per launch, variant 84, 0.3000 ms",
        "level 20 B 8 G 15: 4 keys per launch, variant 16, 2.1000 ms",
        "C^k fused, level 19 B 8 G 15: 4 keys per launch, 8 items per CTA, 7.1000 ms",
    ]
