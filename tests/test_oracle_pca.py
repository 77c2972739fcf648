"""Pins of the oracle's covariance and PowerMethod circuits: the paper's
printed Lazy Normalization figures, its theorems (Taylor lower bound,
monotone Newton convergence, no amplification after EigenShift), and the
decrypted circuits against FP64."""
import os

import numpy as np
import pytest

from oracle.pca import PCA, lazy_normalization_schedule, newton_inv_sqrt, taylor_inv_sqrt


def test_lazy_normalization_reproduces_printed_averages():
    path = os.path.join(os.path.dirname(__file__), "golden", "lazy_normalization.txt")
    rows = 0
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        lP, avg = line.split()
        counts = lazy_normalization_schedule(int(lP), S=0.5, e=1e-5, Bp=1e-3, B2=2.0 ** 16)
        assert round(sum(counts) / len(counts), 1) == float(avg)
        rows += 1
    assert rows == 2


def test_taylor_init_is_a_lower_bound():
    # Sec. 6.1.2: T(x) <= 1/sqrt(x) on (0, B^2]
    B2 = 2.0 ** 16
    x = np.concatenate([np.logspace(-7, 0, 2000), np.linspace(1, B2, 20000)])
    assert np.all(taylor_inv_sqrt(x, B2 / 2 + 1) <= 1 / np.sqrt(x))


def test_newton_monotone_from_below():
    # Thm itr_invsqrt: y_{i-1} <= y_i <= 1/sqrt(x) when 0 < y_0 <= 1/sqrt(x)
    rng = np.random.default_rng(1)
    for x in rng.uniform(1e-4, 1e4, 200):
        y = rng.uniform(0, 1) / np.sqrt(x)
        for _ in range(40):
            y2 = newton_inv_sqrt(x, y, 1)
            assert y - 1e-15 <= y2 <= 1 / np.sqrt(x) * (1 + 1e-12)
            y = y2
        assert abs(y * np.sqrt(x) - 1) < 1e-9


def test_eigen_shift_does_not_amplify():
    # Thm EigShiftnoBig: lambda = <S v, v> <= lambda_1 for unit v, so the
    # shifted matrix amplifies no vector more than S does
    rng = np.random.default_rng(2)
    A = rng.standard_normal((20, 20))
    S = A @ A.T
    lam1 = np.linalg.eigvalsh(S)[-1]
    for _ in range(50):
        v = rng.standard_normal(20)
        v /= np.linalg.norm(v)
        lam = v @ S @ v
        assert lam <= lam1 + 1e-9
        S2 = S - lam * np.outer(v, v)
        assert np.linalg.eigvalsh(S2)[-1] <= lam1 + 1e-9


def _small(levels, seed=3):
    from oracle.ckks import CKKS, Params
    P = Params(11, [60] + [40] * levels, [60])
    return P, CKKS(P, seed)


def _rot_keys(he, P, n, n1, extra=()):
    from oracle.hmm import matmul_rot_steps, transpose_rot_steps
    steps = set(matmul_rot_steps(n, n1, n1, P.S)) | set(transpose_rot_steps(n, n1, P.S))
    i = 1
    while i < n * n:
        steps.add(i % (n * n))
        steps.add((-i) % (n * n))
        i <<= 1
    for s in steps | set(extra):
        if s:
            he.gen_rotation_key(s)
    he.gen_relin_key()


def test_aggregate_axes():
    from oracle.hmm import tile
    P, he = _small(4)
    n = 16
    _rot_keys(he, P, n, 4)
    M = np.random.default_rng(5).uniform(-1, 1, (n, n))
    ct = he.encrypt_slots(tile(M.ravel(), n, P.S), P.L, obj=3, period=n * n)
    pca = PCA(he)
    r0 = he.decrypt_slots(pca.aggregate(ct, 0, n)).real[: n * n].reshape(n, n)
    assert np.abs(r0 - M.sum(0)[None, :]).max() < 1e-5        # every row = column sums
    r1 = he.decrypt_slots(pca.aggregate(ct, 1, n)).real[: n * n].reshape(n, n)
    assert np.abs(r1 - M.sum(1)[:, None]).max() < 1e-5        # every column = row sums


@pytest.mark.parametrize("dcd", [0, 8])
def test_covariance_decrypts_to_fp64(dcd):
    """HCovMtrx, with undecomposed block products and with the Diagonal
    Convergence Decomposition at n' = 8 (Sec. 7 decomposes the covariance's
    products), against FP64."""
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    P, he = _small(7)
    n, n1 = 16, 4
    _rot_keys(he, P, n, n1)
    X = lowrank_dataset(32, 32, 2)
    blocks = []
    obj = 100
    for l in range(2):
        row = []
        for j in range(2):
            z = np.zeros(P.S)
            z[: n * n] = X[l * n:(l + 1) * n, j * n:(j + 1) * n].ravel()
            row.append(he.encrypt_slots(z, P.L, obj=obj))
            obj += 1
        blocks.append(row)
    C = PCA(he).covariance(blocks, 32, n, n1, n1, dcd_z=dcd, dcd_t=dcd)
    Xc = X - X.mean(0)
    ref = Xc.T @ Xc / 32
    for a in range(2):
        for b in range(2):
            d = he.decrypt_slots(C[a][b]).real[: n * n].reshape(n, n)
            assert np.abs(d - ref[a * n:(a + 1) * n, b * n:(b + 1) * n]).max() < 1e-4


def test_power_method_matches_plaintext_replay():
    from oracle.hmm import tile
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    P, he = _small(12)
    n, k = 16, 2
    t = n * k
    _rot_keys(he, P, n, 4)
    X = lowrank_dataset(64, t, 2)
    Xc = X - X.mean(0)
    Cov = Xc.T @ Xc / 64
    Cs = Cov * (1.5 / np.linalg.eigvalsh(Cov)[-1])
    C = [[he.encrypt_slots(tile(Cs[a * n:(a + 1) * n, b * n:(b + 1) * n].ravel(), n, P.S), P.L,
                            obj=10 + a * k + b, period=n * n) for b in range(k)] for a in range(k)]
    v0 = np.random.default_rng(7).standard_normal(t)
    v0 /= np.linalg.norm(v0)
    V0 = [he.encrypt_slots(tile(np.tile(v0[j * n:(j + 1) * n], n), n, P.S), P.L, obj=1000 + j, period=n * n)
          for j in range(k)]
    l_P = 3
    counts = lazy_normalization_schedule(l_P)
    pca = PCA(he)
    lam, V, axis, VT = pca.power_method(C, V0, 0, n, l_P, counts, 2.0 ** 16)
    assert pca.refreshes > 0
    vec = []
    for j in range(k):
        d = he.decrypt_slots(V[j]).real[: n * n].reshape(n, n)
        vec.append(d[0] if axis == 0 else d[:, 0])
    vec = np.concatenate(vec)
    v = v0.copy()
    x0 = 2.0 ** 15 + 1
    for it in range(l_P):
        y = Cs @ v
        x = y @ y
        v = y * newton_inv_sqrt(x, taylor_inv_sqrt(x, x0), counts[it])
    assert np.abs(vec - v).max() < 1e-4
    assert abs(he.decrypt_slots(lam).real[0] - (Cs @ v) @ v) < 1e-4


def test_composite_newton_is_two_steps_in_five_levels():
    """The composite of Sec. 7 (two InvSRT iterations in one) decrypts to two
    plain Newton steps, spends five levels where two steps spend six, lands at
    scale Delta, and an odd count ends with one ordinary step."""
    P, he = _small(14)
    he.gen_relin_key()
    rng = np.random.default_rng(5)
    x = rng.uniform(0.5, 2.0, P.S)
    y0 = 0.8 / np.sqrt(x)
    cx = he.encrypt_slots(x, P.L, obj=1)
    cy = he.encrypt_slots(y0, P.L, obj=2)
    pca = PCA(he, compose_newton=True)
    _, y2 = pca.newton2(cx, cy)
    assert cy.level - y2.level == 5
    assert abs(y2.scale / P.delta - 1) < 1e-9
    want = newton_inv_sqrt(x, y0, 2)
    assert np.abs(he.decrypt_slots(y2).real - want).max() < 1e-6
    single = PCA(he).newton(cx, cy, 2)
    assert cy.level - single.level == 6
    y3 = pca.newton(cx, cy, 3)
    assert cy.level - y3.level == 8 and pca.refreshes == 0
    assert np.abs(he.decrypt_slots(y3).real - newton_inv_sqrt(x, y0, 3)).max() < 1e-6


def test_power_method_with_composite_newton_matches_plaintext_replay():
    from oracle.hmm import tile
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    P, he = _small(15)
    n, k = 16, 2
    t = n * k
    _rot_keys(he, P, n, 4)
    X = lowrank_dataset(64, t, 2)
    Xc = X - X.mean(0)
    Cov = Xc.T @ Xc / 64
    Cs = Cov * (1.5 / np.linalg.eigvalsh(Cov)[-1])
    C = [[he.encrypt_slots(tile(Cs[a * n:(a + 1) * n, b * n:(b + 1) * n].ravel(), n, P.S), P.L,
                            obj=10 + a * k + b, period=n * n) for b in range(k)] for a in range(k)]
    v0 = np.random.default_rng(7).standard_normal(t)
    v0 /= np.linalg.norm(v0)
    V0 = [he.encrypt_slots(tile(np.tile(v0[j * n:(j + 1) * n], n), n, P.S), P.L, obj=1000 + j, period=n * n)
          for j in range(k)]
    l_P = 3
    counts = lazy_normalization_schedule(l_P)
    plain, comp = PCA(he), PCA(he, compose_newton=True)
    plain.power_method(C, V0, 0, n, l_P, counts, 2.0 ** 16)
    lam, V, axis, VT = comp.power_method(C, V0, 0, n, l_P, counts, 2.0 ** 16)
    assert comp.refreshes < plain.refreshes
    vec = []
    for j in range(k):
        d = he.decrypt_slots(V[j]).real[: n * n].reshape(n, n)
        vec.append(d[0] if axis == 0 else d[:, 0])
    vec = np.concatenate(vec)
    v = v0.copy()
    x0 = 2.0 ** 15 + 1
    for it in range(l_P):
        y = Cs @ v
        x = y @ y
        v = y * newton_inv_sqrt(x, taylor_inv_sqrt(x, x0), counts[it])
    assert np.abs(vec - v).max() < 1e-4
    assert abs(he.decrypt_slots(lam).real[0] - (Cs @ v) @ v) < 1e-4


@pytest.mark.parametrize("axis", [0, 1])
def test_packed_refresh_restores_every_segment(axis):
    """App. C: the k segments of a replicated vector refreshed as one
    ciphertext come back replicated along the same axis with the same
    values, at level L - 1, for one refresh instead of k."""
    from oracle.hmm import tile
    P, he = _small(6)
    n, k = 16, 3
    _rot_keys(he, P, n, 4)
    rng = np.random.default_rng(11 + axis)
    vs = [rng.uniform(-1, 1, n) for _ in range(k)]
    V = []
    for j, v in enumerate(vs):
        blk = np.tile(v, (n, 1)) if axis == 0 else np.tile(v[:, None], (1, n))
        ct = he.encrypt_slots(tile(blk.ravel(), n, P.S), P.L, obj=40 + j, period=n * n)
        V.append(he.drop(ct, 1))
    pca = PCA(he, pack_refresh=True)
    out = pca.packed_refresh(V, axis, n)
    assert pca.refreshes == 1
    for j, (ct, v) in enumerate(zip(out, vs)):
        assert ct.level == P.L - 1
        d = he.decrypt_slots(ct).real[: n * n].reshape(n, n)
        want = np.tile(v, (n, 1)) if axis == 0 else np.tile(v[:, None], (1, n))
        assert np.abs(d - want).max() < 1e-6, j


def test_power_method_with_packed_refresh_matches_plaintext_replay():
    from oracle.hmm import tile
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    P, he = _small(13)
    n, k = 16, 2
    t = n * k
    _rot_keys(he, P, n, 4)
    X = lowrank_dataset(64, t, 2)
    Xc = X - X.mean(0)
    Cov = Xc.T @ Xc / 64
    Cs = Cov * (1.5 / np.linalg.eigvalsh(Cov)[-1])
    C = [[he.encrypt_slots(tile(Cs[a * n:(a + 1) * n, b * n:(b + 1) * n].ravel(), n, P.S), P.L,
                            obj=10 + a * k + b, period=n * n) for b in range(k)] for a in range(k)]
    v0 = np.random.default_rng(7).standard_normal(t)
    v0 /= np.linalg.norm(v0)
    V0 = [he.encrypt_slots(tile(np.tile(v0[j * n:(j + 1) * n], n), n, P.S), P.L, obj=1000 + j, period=n * n)
          for j in range(k)]
    l_P = 4
    counts = lazy_normalization_schedule(l_P)
    plain, packed = PCA(he), PCA(he, pack_refresh=True)
    plain.power_method(C, V0, 0, n, l_P, counts, 2.0 ** 16)
    lam, V, axis, VT = packed.power_method(C, V0, 0, n, l_P, counts, 2.0 ** 16)
    assert packed.refreshes < plain.refreshes
    vec = []
    for j in range(k):
        d = he.decrypt_slots(V[j]).real[: n * n].reshape(n, n)
        vec.append(d[0] if axis == 0 else d[:, 0])
    vec = np.concatenate(vec)
    v = v0.copy()
    x0 = 2.0 ** 15 + 1
    for it in range(l_P):
        y = Cs @ v
        x = y @ y
        v = y * newton_inv_sqrt(x, taylor_inv_sqrt(x, x0), counts[it])
    assert np.abs(vec - v).max() < 1e-4
    assert abs(he.decrypt_slots(lam).real[0] - (Cs @ v) @ v) < 1e-4


def test_covariance_three_column_blocks_decrypts_to_fp64():
    """HCovMtrx with k = 3 column blocks (t = 3n features, ragged rows):
    six block products per row block, three mirrored by G, against FP64."""
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    P, he = _small(7)
    n, n1 = 16, 4
    _rot_keys(he, P, n, n1)
    X = lowrank_dataset(20, 48, 6)           # 2 row blocks, the second zero-padded
    k, nrb = 3, 2
    Xp = np.zeros((nrb * n, k * n))
    Xp[:20] = X
    blocks = []
    for l in range(nrb):
        row = []
        for j in range(k):
            z = np.zeros(P.S)
            z[: n * n] = Xp[l * n:(l + 1) * n, j * n:(j + 1) * n].ravel()
            row.append(he.encrypt_slots(z, P.L, obj=200 + l * k + j))
        blocks.append(row)
    C = PCA(he).covariance(blocks, 20, n, n1, n1)
    Xc = X - X.mean(0)
    ref = Xc.T @ Xc / 20
    for a in range(k):
        for b in range(k):
            d = he.decrypt_slots(C[a][b]).real[: n * n].reshape(n, n)
            assert np.abs(d - ref[a * n:(a + 1) * n, b * n:(b + 1) * n]).max() < 1e-4, (a, b)
