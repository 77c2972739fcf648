"""CUDA covariance / PowerMethod path against the oracle (bit-exact residues)
and against FP64 (decrypted values)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LOGN, QBITS, PBITS = 12, [60] + [40] * 12, [60]


@pytest.fixture(scope="module")
def env():
    import paper_2305_17341_gb300 as pk
    from oracle.ckks import CKKS, Params
    from oracle.hmm import matmul_rot_steps, transpose_rot_steps
    pk.build()
    ctx = pk.he_ctx_create(pk.make_params(LOGN, QBITS, PBITS), 13)
    P = Params(LOGN, QBITS, PBITS)
    he = CKKS(P, 13)
    n, n1 = 16, 4
    steps = set(matmul_rot_steps(n, n1, n1, P.S)) | set(transpose_rot_steps(n, n1, P.S))
    i = 1
    while i < n * n:
        steps |= {i % (n * n), (-i) % (n * n)}
        i <<= 1
    steps.discard(0)
    pk.he_keygen(ctx, sorted(steps), want_relin=True)
    for s in steps:
        he.gen_rotation_key(s)
    he.gen_relin_key()
    yield pk, ctx, P, he, n, n1
    pk.he_ctx_destroy(ctx)


def res(ct):
    return np.stack([ct.c0, ct.c1])


def test_aggregate_and_refresh_bit_exact(env):
    from oracle.hmm import tile
    from oracle.pca import PCA
    pk, ctx, P, he, n, n1 = env
    M = np.random.default_rng(3).uniform(-1, 1, (n, n))
    z = tile(M.ravel(), n, P.S)
    o = he.encrypt_slots(z, 5, obj=21, period=n * n)
    g = pk.he_ct_import(ctx, res(o), 5, o.scale, n * n)
    pca = PCA(he)
    for axis in (0, 1):
        ga = pk.he_aggregate(ctx, g, axis, n)
        oa = pca.aggregate(o, axis, n)
        assert np.array_equal(pk.he_ct_export(ctx, ga), res(oa))
        pk.he_ct_free(ga)
    rs = pk.he_refresh_state(7, 0)
    gr = pk.he_refresh(ctx, g, rs)
    orr = he.refresh(o, 8)
    assert (rs.next_obj, rs.count) == (8, 1)
    assert np.array_equal(pk.he_ct_export(ctx, gr), res(orr))
    assert pk.he_ct_info(gr)[0] == P.L
    for h in (g, gr):
        pk.he_ct_free(h)


def _dataset_blocks(pk, ctx, P, he, X, n):
    s, t = X.shape
    nrb, k = -(-s // n), -(-t // n)
    Xp = np.zeros((nrb * n, k * n))
    Xp[:s, :t] = X
    g, o = [], []
    for l in range(nrb):
        row = []
        for j in range(k):
            blk = Xp[l * n:(l + 1) * n, j * n:(j + 1) * n]
            z = np.zeros(P.S)
            z[: n * n] = blk.ravel()
            row.append(he.encrypt_slots(z, P.L, obj=300 + l * k + j))
            g.append(pk.he_encrypt_matrix(ctx, blk, P.L, 300 + l * k + j))
        o.append(row)
    return g, o, nrb, k


def test_covariance_bit_exact_and_fp64(env):
    from oracle.pca import PCA
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    pk, ctx, P, he, n, n1 = env
    X = lowrank_dataset(40, 32, 2)          # ragged: 40 rows -> 3 row blocks, last zero-padded
    g, o, nrb, k = _dataset_blocks(pk, ctx, P, he, X, n)
    C = pk.he_covariance(ctx, g, nrb, k, n, X.shape[0], False, n1, n1)
    Co = PCA(he).covariance(o, X.shape[0], n, n1, n1)
    Xc = X - X.mean(0)
    ref = Xc.T @ Xc / X.shape[0]
    for a in range(k):
        for b in range(k):
            assert np.array_equal(pk.he_ct_export(ctx, C[a * k + b]), res(Co[a][b])), (a, b)
            d = pk.he_decrypt_matrix(ctx, C[a * k + b], n, n)
            assert np.abs(d - ref[a * n:(a + 1) * n, b * n:(b + 1) * n]).max() < 1e-4
    for h in C + g:
        pk.he_ct_free(h)


def test_power_method_and_eigen_shift_bit_exact(env):
    from oracle.hmm import tile
    from oracle.pca import PCA, lazy_normalization_schedule
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    pk, ctx, P, he, n, n1 = env
    k = 2
    t = n * k
    X = lowrank_dataset(64, t, 4)
    Xc = X - X.mean(0)
    Cov = Xc.T @ Xc / 64
    Cs = Cov * (1.5 / np.linalg.eigvalsh(Cov)[-1])
    Co, Cg = [], []
    for a in range(k):
        row = []
        for b in range(k):
            z = tile(Cs[a * n:(a + 1) * n, b * n:(b + 1) * n].ravel(), n, P.S)
            ct = he.encrypt_slots(z, P.L, obj=500 + a * k + b, period=n * n)
            row.append(ct)
            Cg.append(pk.he_ct_import(ctx, res(ct), P.L, ct.scale, n * n))
        Co.append(row)
    v0 = np.random.default_rng(7).standard_normal(t)
    v0 /= np.linalg.norm(v0)
    V0o = [he.encrypt_slots(tile(np.tile(v0[j * n:(j + 1) * n], n), n, P.S), P.L, obj=900 + j, period=n * n)
           for j in range(k)]
    V0g = [pk.he_ct_import(ctx, res(v), P.L, v.scale, n * n) for v in V0o]
    l_P = 3
    counts = lazy_normalization_schedule(l_P)
    pca = PCA(he)
    pca.refresh_obj = 1 << 20
    lam_o, V_o, ax_o, VT_o = pca.power_method(Co, V0o, 0, n, l_P, counts, 2.0 ** 16)
    rs = pk.he_refresh_state(1 << 20, 0)
    lam_g, V_g, VT_g, ax_g = pk.he_power_method(ctx, Cg, k, n, V0g, 0, l_P, counts, 2.0 ** 16, rs)
    assert ax_g == ax_o and rs.count == pca.refreshes
    assert np.array_equal(pk.he_ct_export(ctx, lam_g), res(lam_o))
    for j in range(k):
        assert np.array_equal(pk.he_ct_export(ctx, V_g[j]), res(V_o[j]))
        assert np.array_equal(pk.he_ct_export(ctx, VT_g[j]), res(VT_o[j]))
    S_o = pca.eigen_shift(Co, lam_o, V_o, ax_o, VT_o, n)
    S_g = pk.he_eigen_shift(ctx, Cg, k, n, lam_g, V_g, ax_g, VT_g, rs)
    assert rs.count == pca.refreshes
    for a in range(k):
        for b in range(k):
            assert np.array_equal(pk.he_ct_export(ctx, S_g[a * k + b]), res(S_o[a][b]))
    for h in S_g + V_g + VT_g + V0g + [lam_g]:
        pk.he_ct_free(h)


def test_full_size_covariance_256():
    """Config 2: 256x256 low-rank dataset, 128x128 blocks at N=2^16, chain
    60 + 20x40, p 2x60: decrypted covariance within 1e-4 of FP64."""
    import paper_2305_17341_gb300 as pk
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    pk.build()
    ctx = pk.he_ctx_create(pk.he_params_default(2), 77)
    try:
        n, n1 = 128, 16
        S = 1 << 15
        steps = set(pk.he_rot_steps_for_matmul(n, n1, n1, S)) | set(pk.he_rot_steps_for_transpose(n, n1, S))
        i = n
        while i < n * n:
            steps.add(i)
            i <<= 1
        pk.he_keygen(ctx, sorted(steps), want_relin=True)
        X = lowrank_dataset(256, 256, 2)
        blocks = [pk.he_encrypt_matrix(ctx, X[l * n:(l + 1) * n, j * n:(j + 1) * n], 20, 10 + 2 * l + j)
                  for l in range(2) for j in range(2)]
        C = pk.he_covariance(ctx, blocks, 2, 2, n, 256, False, n1, n1)
        Xc = X - X.mean(0)
        ref = Xc.T @ Xc / 256
        for a in range(2):
            for b in range(2):
                d = pk.he_decrypt_matrix(ctx, C[a * 2 + b], n, n)
                assert np.abs(d - ref[a * n:(a + 1) * n, b * n:(b + 1) * n]).max() < 1e-4
        for h in C + blocks:
            pk.he_ct_free(h)
    finally:
        pk.he_ctx_destroy(ctx)


def test_pca_two_components_bit_exact(env):
    """he_pca (l_E = 2) equals the oracle's PowerMethod, EigenShift, PowerMethod."""
    from oracle.hmm import tile
    from oracle.pca import PCA, lazy_normalization_schedule
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    pk, ctx, P, he, n, n1 = env
    k = 2
    t = n * k
    X = lowrank_dataset(64, t, 6)
    Xc = X - X.mean(0)
    Cs = (Xc.T @ Xc / 64) * t
    Co, Cg = [], []
    for a in range(k):
        row = []
        for b in range(k):
            ct = he.encrypt_slots(tile(Cs[a * n:(a + 1) * n, b * n:(b + 1) * n].ravel(), n, P.S), P.L,
                                  obj=700 + a * k + b, period=n * n)
            row.append(ct)
            Cg.append(pk.he_ct_import(ctx, res(ct), P.L, ct.scale, n * n))
        Co.append(row)
    rng = np.random.default_rng(9)
    V0o, V0g = [], []
    for m in range(2):
        v0 = rng.standard_normal(t)
        v0 /= np.linalg.norm(v0)
        vs = [he.encrypt_slots(tile(np.tile(v0[j * n:(j + 1) * n], n), n, P.S), P.L, obj=800 + 10 * m + j,
                               period=n * n) for j in range(k)]
        V0o.append(vs)
        V0g += [pk.he_ct_import(ctx, res(v), P.L, v.scale, n * n) for v in vs]
    l_P = 2
    counts = lazy_normalization_schedule(l_P)
    pca = PCA(he)
    C = Co
    want = []
    for m in range(2):
        lam, V, ax, VT = pca.power_method(C, V0o[m], 0, n, l_P, counts, 2.0 ** 16)
        want.append((lam, V, ax))
        if m == 0:
            C = pca.eigen_shift(C, lam, V, ax, VT, n)
    rs = pk.he_refresh_state(1 << 20, 0)
    lams, Vs, axes = pk.he_pca(ctx, Cg, k, n, 2, V0g, 0, l_P, counts, 2.0 ** 16, rs)
    assert rs.count == pca.refreshes
    for m in range(2):
        assert axes[m] == want[m][2]
        assert np.array_equal(pk.he_ct_export(ctx, lams[m]), res(want[m][0]))
        for j in range(k):
            assert np.array_equal(pk.he_ct_export(ctx, Vs[m][j]), res(want[m][1][j]))
    for h in lams + [x for v in Vs for x in v] + Cg + V0g:
        pk.he_ct_free(h)


@pytest.mark.parametrize("compose,pack", [(True, False), (False, True), (True, True)])
def test_power_method_composed_newton_bit_exact(env, compose, pack):
    """HPowerMethod with pairs of Newton steps as five-level composites
    (Sec. 7) and / or the packed eigenvector refresh (App. C): residues,
    refresh count and axis equal the oracle's same schedule."""
    from oracle.hmm import tile
    from oracle.pca import PCA, lazy_normalization_schedule
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    pk, ctx, P, he, n, n1 = env
    k = 2
    t = n * k
    X = lowrank_dataset(64, t, 6)
    Xc = X - X.mean(0)
    Cov = Xc.T @ Xc / 64
    Cs = Cov * (1.5 / np.linalg.eigvalsh(Cov)[-1])
    Co, Cg = [], []
    for a in range(k):
        row = []
        for b in range(k):
            z = tile(Cs[a * n:(a + 1) * n, b * n:(b + 1) * n].ravel(), n, P.S)
            ct = he.encrypt_slots(z, P.L, obj=600 + a * k + b, period=n * n)
            row.append(ct)
            Cg.append(pk.he_ct_import(ctx, res(ct), P.L, ct.scale, n * n))
        Co.append(row)
    v0 = np.random.default_rng(8).standard_normal(t)
    v0 /= np.linalg.norm(v0)
    V0o = [he.encrypt_slots(tile(np.tile(v0[j * n:(j + 1) * n], n), n, P.S), P.L, obj=950 + j, period=n * n)
           for j in range(k)]
    V0g = [pk.he_ct_import(ctx, res(v), P.L, v.scale, n * n) for v in V0o]
    l_P = 3
    counts = lazy_normalization_schedule(l_P)
    pca = PCA(he, compose_newton=compose, pack_refresh=pack)
    pca.refresh_obj = 1 << 21
    lam_o, V_o, ax_o, VT_o = pca.power_method(Co, V0o, 0, n, l_P, counts, 2.0 ** 16)
    rs = pk.he_refresh_state(1 << 21, 0)
    pk.he_ctx_set_newton_composition(ctx, compose)
    pk.he_ctx_set_packed_refresh(ctx, pack)
    try:
        lam_g, V_g, VT_g, ax_g = pk.he_power_method(ctx, Cg, k, n, V0g, 0, l_P, counts, 2.0 ** 16, rs)
    finally:
        pk.he_ctx_set_newton_composition(ctx, False)
        pk.he_ctx_set_packed_refresh(ctx, False)
    assert ax_g == ax_o and rs.count == pca.refreshes
    assert np.array_equal(pk.he_ct_export(ctx, lam_g), res(lam_o))
    for j in range(k):
        assert np.array_equal(pk.he_ct_export(ctx, V_g[j]), res(V_o[j]))
        assert np.array_equal(pk.he_ct_export(ctx, VT_g[j]), res(VT_o[j]))
    for h in V_g + VT_g + V0g + Cg + [lam_g]:
        pk.he_ct_free(h)


def test_covariance_decomposed_bit_exact(env):
    """HCovMtrx with its block products decomposed (Sec. 7 runs the
    covariance with the Diagonal Convergence Decomposition): residues equal
    the oracle's same schedule, decrypted blocks match FP64."""
    from oracle.pca import PCA
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    pk, ctx, P, he, n, n1 = env
    X = lowrank_dataset(32, 32, 3)
    g, o, nrb, k = _dataset_blocks(pk, ctx, P, he, X, n)
    C = pk.he_covariance(ctx, g, nrb, k, n, X.shape[0], False, n1, n1, dcd_z=8, dcd_t=8)
    Co = PCA(he).covariance(o, X.shape[0], n, n1, n1, dcd_z=8, dcd_t=8)
    Xc = X - X.mean(0)
    ref = Xc.T @ Xc / X.shape[0]
    for a in range(k):
        for b in range(k):
            assert np.array_equal(pk.he_ct_export(ctx, C[a * k + b]), res(Co[a][b])), (a, b)
            d = pk.he_decrypt_matrix(ctx, C[a * k + b], n, n)
            assert np.abs(d - ref[a * n:(a + 1) * n, b * n:(b + 1) * n]).max() < 1e-4
    lv_plain = PCA(he).covariance(o, X.shape[0], n, n1, n1)[0][0].level
    assert Co[0][0].level == lv_plain - 1      # product depth 2 + ceil(15/8) = 4 instead of 3
    for h in C + g:
        pk.he_ct_free(h)


def test_pca_cosine_vs_eigh_with_clear_eigen_gap(env):
    """Accuracy of the encrypted PCA against numpy.linalg.eigh: a 32-feature
    dataset whose singular values halve from one component to the next
    (eigen-gap 0.25), two components by he_pca with l_P = 10: each
    eigenvector has |cos| >= 0.999 with eigh's and its eigenvalue is within
    1 % of eigh's.  The same schedule run in FP64 (the oracle's TaylorInit and
    Newton steps) agrees with the encrypted vectors to 1e-4, so what remains
    against eigh is the method's convergence, not the encryption."""
    from oracle.hmm import tile
    from oracle.pca import lazy_normalization_schedule, newton_inv_sqrt, taylor_inv_sqrt
    pk, ctx, P, he, n, n1 = env
    k, s = 2, 96
    t = n * k
    rng = np.random.default_rng(31)
    U0, _ = np.linalg.qr(rng.standard_normal((s, t)))
    V0m, _ = np.linalg.qr(rng.standard_normal((t, t)))
    X = (U0 * 0.5 ** np.arange(t)) @ V0m.T
    Xc = X - X.mean(0)
    Cov = Xc.T @ Xc / s
    # scaled so that the second eigenvalue is 1: the contraction S = 0.5 that
    # Lazy Normalization's Newton counts assume stays below every eigenvalue
    # the PowerMethod targets, so each deflated run ends at unit length
    Cs = Cov * (1.0 / np.linalg.eigvalsh(Cov)[-2])
    w, E = np.linalg.eigh(Cs)
    w, E = w[::-1], E[:, ::-1]
    assert w[1] / w[0] < 0.3 and w[2] / w[1] < 0.3
    def enc_tiled(z, obj):
        """Encrypts slots already tiled with period n^2 and marks that period."""
        g = pk.he_encrypt_slots(ctx, z, P.L, obj)
        h = pk.he_ct_import(ctx, pk.he_ct_export(ctx, g), P.L, pk.he_ct_info(g)[1], n * n)
        pk.he_ct_free(g)
        return h

    Cg = []
    for a in range(k):
        for b in range(k):
            Cg.append(enc_tiled(tile(Cs[a * n:(a + 1) * n, b * n:(b + 1) * n].ravel(), n, P.S), 1500 + a * k + b))
    l_E, l_P = 2, 10
    counts = lazy_normalization_schedule(l_P)
    V0g, v0s = [], []
    for m in range(l_E):
        v0 = rng.standard_normal(t)
        v0 /= np.linalg.norm(v0)
        v0s.append(v0)
        for j in range(k):
            V0g.append(enc_tiled(tile(np.tile(v0[j * n:(j + 1) * n], n), n, P.S), 1600 + m * k + j))
    rs = pk.he_refresh_state(1 << 22, 0)
    lams, Vs, axes = pk.he_pca(ctx, Cg, k, n, l_E, V0g, 0, l_P, counts, 2.0 ** 16, rs)
    C64 = Cs.copy()
    x0 = 2.0 ** 15 + 1
    for m in range(l_E):
        parts = []
        for j in range(k):
            d = pk.he_decrypt_matrix(ctx, Vs[m][j], n, n)
            parts.append(d[0] if axes[m] == 0 else d[:, 0])
        v = np.concatenate(parts)
        cos = abs(v @ E[:, m]) / np.linalg.norm(v)
        lam = pk.he_decrypt_slots(ctx, lams[m], 1)[0]
        assert cos >= 0.999, (m, cos)
        assert abs(lam - w[m]) < 0.01 * w[m], (m, lam, w[m])
        # the same schedule in FP64
        f = v0s[m].copy()
        for it in range(l_P):
            y = C64 @ f
            x = y @ y
            f = y * newton_inv_sqrt(x, taylor_inv_sqrt(x, x0), counts[it])
        lam64 = (C64 @ f) @ f
        assert np.abs(v - f).max() < 1e-4, m
        C64 = C64 - lam64 * np.outer(f, f)
    for h in lams + [x for vv in Vs for x in vv] + Cg + V0g:
        pk.he_ct_free(h)


def test_covariance_parts_over_row_block_shares_equal_whole(env):
    """he_covariance_partial on two shares of the row blocks (2 + 1 of a
    ragged 40 x 32 dataset), the parts added residue by residue mod q (what
    the all-reduce of the sharded covariance does), imported, and
    he_covariance_finish: the covariance blocks equal he_covariance's word
    for word.  The sharding module run on a one-rank process group gives the
    same words."""
    import socket

    import torch.distributed as dist

    from paper_2305_17341_gb300 import sharding
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    pk, ctx, P, he, n, n1 = env
    X = lowrank_dataset(40, 32, 2)
    g, _, nrb, k = _dataset_blocks(pk, ctx, P, he, X, n)
    s = X.shape[0]
    whole = pk.he_covariance(ctx, g, nrb, k, n, s, False, n1, n1)
    want = [pk.he_ct_export(ctx, h) for h in whole]
    q, _ = pk.he_ctx_primes(ctx)
    parts = [pk.he_covariance_partial(ctx, g[lo * k:hi * k], hi - lo, k, n, s, False, n1, n1)
             for lo, hi in ((0, 2), (2, 3))]

    def add(hs):
        lv, sc, per = pk.he_ct_info(hs[0])
        r = sum(pk.he_ct_export(ctx, h).astype(object) for h in hs)
        r = np.array(r % np.array(q[: lv + 1], dtype=object)[:, None], dtype=np.uint64)
        return pk.he_ct_import(ctx, r, lv, sc, per)

    upper = [add([p[0][u] for p in parts]) for u in range(k * (k + 1) // 2)]
    colsum = [add([p[1][j] for p in parts]) for j in range(k)]
    C = pk.he_covariance_finish(ctx, upper, colsum, k, n, s, False, n1, n1, pk.he_ct_info(g[0])[0])
    for i in range(k * k):
        assert np.array_equal(pk.he_ct_export(ctx, C[i]), want[i]), i
    sock = socket.socket()
    sock.bind(("127.0.0.1", 0))
    port = sock.getsockname()[1]
    sock.close()
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=0, world_size=1)
    try:
        C1 = sharding.covariance_sharded(ctx, g, nrb, k, n, s, False, n1, n1)
    finally:
        dist.destroy_process_group()
    for i in range(k * k):
        assert np.array_equal(pk.he_ct_export(ctx, C1[i]), want[i]), i
    for h in C + C1 + whole + upper + colsum + g + [x for p in parts for hs in p for x in hs]:
        pk.he_ct_free(h)
