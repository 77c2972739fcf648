"""Parity with the oracle under two special primes (alpha = 2).

Every benchmarked configuration switches keys with digits of two q's and
rounds the ModDown over P = p_0 p_1 (App. A KeySwitch with hybrid digits).
Here the CUDA path is compared with the oracle element by element on that
gadget: products under the paper's DMatrixMult (Sec. 4.3), with one
relinearisation per product and with the Diagonal Convergence Decomposition
(Sec. 4.2), HCovMtrx (Sec. 5.2) and a two-component PCA (Sec. 6.2), all at
N = 2^14 on the register-blocked NTT path the benchmark runs, with a chain
whose top level ends in a digit of one prime; and one 128 x 128 product with
the benchmark's schedule (n1 = 16) at N = 2^15, where n^2 = N/2 so the
product needs no replication.  Residues are compared in coefficient form;
decrypted values against FP64 within 1e-4 per entry."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-4
LOGN, QBITS, PBITS = 14, [60] + [40] * 12, [60, 60]
# MultSum launch variants: -1 the tuner's pick, 0 the thread-per-word
# kernel (16, 20: with L2 prefetch; 32, 36, 48: more CTAs per SM; 64, 65: the
# rotations split over warps; 80, 84, 96, 97: two coefficients per thread),
# 8, 9, 10 the bulk-copy kernel with three tile shapes
VARIANTS = (-1, 0, 16, 20, 32, 36, 48, 64, 65, 80, 84, 96, 97, 8, 9, 10)
# NTT variants: one-tile CTAs (2, 3 or, as 5, 4 per SM), persistent bulk-copy passes (4),
# one pass per limb by 8-CTA clusters (6; N = 2^16 only, here as 3)
NTT_VARIANTS = (2, 3, 5, 4, 6)


def res(ct):
    return np.stack([ct.c0, ct.c1])


@pytest.fixture(scope="module")
def a2():
    import paper_2305_17341_gb300 as pk
    from oracle.ckks import CKKS, Params
    from oracle.hmm import matmul_rot_steps, transpose_rot_steps
    pk.build()
    P = Params(LOGN, QBITS, PBITS)
    assert P.alpha == 2 and (P.L + 1) % 2 == 1      # the top level ends in a one-prime digit
    ctx = pk.he_ctx_create(pk.make_params(LOGN, QBITS, PBITS), 17)
    he = CKKS(P, 17)
    n, n1 = 16, 4
    steps = set(matmul_rot_steps(n, n1, n1, P.S)) | set(transpose_rot_steps(n, n1, P.S))
    steps |= set(matmul_rot_steps(n, n1, n1, P.S, 8, 8))
    i = 1
    while i < n * n:
        steps |= {i % (n * n), (-i) % (n * n)}
        i <<= 1
    steps.discard(0)
    steps = sorted(steps)
    pk.he_keygen(ctx, steps, want_relin=True)
    for s in steps:
        he.gen_rotation_key(s)
    he.gen_relin_key()
    yield pk, ctx, P, he, n, n1
    pk.he_ctx_destroy(ctx)


def _encrypted_pair(pk, ctx, P, he, n, seed):
    rng = np.random.default_rng(seed)
    A, B = rng.uniform(-1, 1, (n, n)), rng.uniform(-1, 1, (n, n))
    out = []
    for M, obj in ((A, 2 * seed), (B, 2 * seed + 1)):
        z = np.zeros(P.S)
        z[: n * n] = M.ravel()
        o = he.encrypt_slots(z, P.L, obj=obj)
        g = pk.he_encrypt_matrix(ctx, M, P.L, obj)
        assert np.array_equal(pk.he_ct_export(ctx, g), res(o))
        out.append((o, g))
    return A, B, out


def test_alpha2_primes_and_key_switch_shape(a2):
    pk, ctx, P, he, n, n1 = a2
    q, p = pk.he_ctx_primes(ctx)
    assert q == P.q and p == P.p
    info = pk.he_ctx_info(ctx)
    assert (info["alpha"], info["dnum"]) == (2, 7)


@pytest.mark.parametrize("sched", ["dmatrixmult", "relin_once", "dcd8"])
def test_alpha2_product_bit_exact_every_multsum_variant(a2, sched):
    """16 x 16 product at level 12 (digits {q0,q1} .. {q12}): residues and
    MultSum / Decompose / ModDown counts equal the oracle's under every
    MultSum launch variant and every NTT variant; the product decrypts to
    A.B."""
    from oracle.hmm import HMM
    pk, ctx, P, he, n, n1 = a2
    kw = {"dmatrixmult": {}, "relin_once": {"relin_once": True}, "dcd8": {"dcd_z": 8, "dcd_t": 8}}[sched]
    A, B, ((oa, ga), (ob, gb)) = _encrypted_pair(pk, ctx, P, he, n, 60 + len(sched))
    he.cnt.reset()
    oc = HMM(he).hmatmul(oa, ob, n, n1, n1, **kw)
    want = res(oc)
    try:
        for v, nv, chunk in ([(v, -1, None) for v in VARIANTS] + [(-1, nv, 0) for nv in NTT_VARIANTS] +
                             [(-1, 3, 5)]):
            pk.he_ctx_set_multsum_variant(ctx, v)
            pk.he_ctx_set_ntt_variant(ctx, nv)
            if chunk is not None:
                pk.he_ctx_set_ntt_chunk(ctx, chunk)
            pk.he_counters(ctx, reset=True)
            gc = pk.he_hmatmul(ctx, ga, gb, n, n1, n1, **kw)
            cnt = pk.he_counters(ctx)
            assert (cnt["MS"], cnt["Dp"], cnt["MD"]) == (he.cnt.MS, he.cnt.Dp, he.cnt.MD), v
            got = pk.he_ct_export(ctx, gc)
            assert np.array_equal(got, want), "variants %d/%d: %d of %d words differ" % (
                v, nv, (got != want).sum(), got.size)
            lv, sc, per = pk.he_ct_info(gc)
            assert (lv, per) == (oc.level, n * n) and sc == oc.scale
            assert np.abs(pk.he_decrypt_matrix(ctx, gc, n, n) - A @ B).max() < TOL
            pk.he_ct_free(gc)
    finally:
        pk.he_ctx_set_multsum_variant(ctx, -1)
        pk.he_ctx_set_ntt_variant(ctx, -1)
        pk.he_ctx_set_ntt_chunk(ctx, 0)
    for h in (ga, gb):
        pk.he_ct_free(h)


def test_alpha2_fused_ck_forms_bit_exact(a2):
    """n1 = 8 (7 C^k babies per giant: launches of 4 and 3 rotations): the
    product under the tuner, the thread-per-word fused C^k kernel (variant
    0) and its rotations-split-over-warps form (variant 96, the 4-rotation
    launches) equals the oracle word for word."""
    from oracle.hmm import HMM, matmul_rot_steps
    pk, ctx, P, he, n, _ = a2
    n1 = 8
    steps = sorted(set(matmul_rot_steps(n, n1, n1, P.S)))
    pk.he_keygen(ctx, steps, want_relin=True)
    for st in steps:
        he.gen_rotation_key(st)
    A, B, ((oa, ga), (ob, gb)) = _encrypted_pair(pk, ctx, P, he, n, 91)
    want = res(HMM(he).hmatmul(oa, ob, n, n1, n1))
    try:
        for v in (-1, 0, 96):
            pk.he_ctx_set_multsum_variant(ctx, v)
            gc = pk.he_hmatmul(ctx, ga, gb, n, n1, n1)
            got = pk.he_ct_export(ctx, gc)
            assert np.array_equal(got, want), "variant %d: %d of %d words differ" % (v, (got != want).sum(), got.size)
            assert np.abs(pk.he_decrypt_matrix(ctx, gc, n, n) - A @ B).max() < TOL
            pk.he_ct_free(gc)
    finally:
        pk.he_ctx_set_multsum_variant(ctx, -1)
    for h in (ga, gb):
        pk.he_ct_free(h)


def test_alpha2_batched_products_at_two_levels(a2):
    """Three products in one he_hmatmul_batch call, two at level 12 and one
    at level 9 (a two-prime last digit): each equals the oracle."""
    from oracle.hmm import HMM
    pk, ctx, P, he, n, n1 = a2
    H = HMM(he)
    jobs, want, refs, hs = [], [], [], []
    for i, level in enumerate((P.L, 9, P.L)):
        A, B, ((oa, ga), (ob, gb)) = _encrypted_pair(pk, ctx, P, he, n, 90 + i)
        if level != P.L:
            oa, ob = he.drop(oa, level), he.drop(ob, level)
            pk.he_ct_free(ga)
            pk.he_ct_free(gb)
            ga = pk.he_ct_import(ctx, res(oa), level, oa.scale, P.S)
            gb = pk.he_ct_import(ctx, res(ob), level, ob.scale, P.S)
        jobs.append((ga, gb, n, n1, n1))
        want.append(res(H.hmatmul(oa, ob, n, n1, n1)))
        refs.append(A @ B)
        hs += [ga, gb]
    outs = pk.he_hmatmul_batch(jobs)
    for o, w, ref in zip(outs, want, refs):
        assert np.array_equal(pk.he_ct_export(ctx, o), w)
        assert np.abs(pk.he_decrypt_matrix(ctx, o, n, n) - ref).max() < TOL
    for h in outs + hs:
        pk.he_ct_free(h)


def test_alpha2_covariance_bit_exact_and_fp64(a2):
    """HCovMtrx of a ragged 24 x 32 dataset (2 row blocks, the second
    zero-padded; 2 feature blocks): residues equal the oracle's, decrypted
    blocks within 1e-4 of FP64 Xc^T Xc / s."""
    from oracle.pca import PCA
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    pk, ctx, P, he, n, n1 = a2
    X = lowrank_dataset(24, 32, 3)
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
    C = pk.he_covariance(ctx, g, nrb, k, n, s, False, n1, n1)
    Co = PCA(he).covariance(o, s, n, n1, n1)
    Xc = X - X.mean(0)
    ref = Xc.T @ Xc / s
    for a in range(k):
        for b in range(k):
            assert np.array_equal(pk.he_ct_export(ctx, C[a * k + b]), res(Co[a][b])), (a, b)
            d = pk.he_decrypt_matrix(ctx, C[a * k + b], n, n)
            assert np.abs(d - ref[a * n:(a + 1) * n, b * n:(b + 1) * n]).max() < TOL
    for h in C + g:
        pk.he_ct_free(h)


def test_alpha2_pca_two_components_bit_exact(a2):
    """he_pca with two components (PowerMethod, EigenShift, PowerMethod;
    Sec. 6.2): eigenvalue and eigenvector residues, axes and the refresh
    count equal the oracle's."""
    from oracle.hmm import tile
    from oracle.pca import PCA, lazy_normalization_schedule
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    pk, ctx, P, he, n, n1 = a2
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


def test_alpha2_128x128_benchmark_schedule_bit_exact():
    """The benchmark's product shape and schedule -- 128 x 128, n1 = 16 for
    Z and T, per-product relinearisation -- at N = 2^15 (n^2 = N/2: one
    matrix fills the slots, no replication), q 60 + 4 x 40, p 2 x 60: residues
    and operation counts equal the oracle's (562 MultSums, 176 Decomposes,
    421 ModDowns: the schedule's 564 / 178 / 423 at N = 2^16 less the two
    replication rotations, one per operand), the product decrypts to A.B."""
    import paper_2305_17341_gb300 as pk
    from oracle.ckks import CKKS, Params
    from oracle.hmm import HMM, matmul_rot_steps
    pk.build()
    qbits, pbits = [60] + [40] * 4, [60, 60]
    P = Params(15, qbits, pbits)
    he = CKKS(P, 23)
    ctx = pk.he_ctx_create(pk.make_params(15, qbits, pbits), 23)
    try:
        n, n1 = 128, 16
        steps = matmul_rot_steps(n, n1, n1, P.S)
        assert sorted(steps) == sorted(pk.he_rot_steps_for_matmul(n, n1, n1, P.S))
        pk.he_keygen(ctx, steps, want_relin=True)
        for s in steps:
            he.gen_rotation_key(s)
        he.gen_relin_key()
        A, B, ((oa, ga), (ob, gb)) = _encrypted_pair(pk, ctx, P, he, n, 5)
        he.cnt.reset()
        oc = HMM(he).hmatmul(oa, ob, n, n1, n1)
        assert (he.cnt.MS, he.cnt.Dp, he.cnt.MD) == (562, 176, 421)
        # the tuner's launches, then the fused C^k kernel pinned to its
        # eight-rotation split form (variant 97: the 15 babies of a giant as
        # launches of 8, 4 and 3 rotations)
        for v in (-1, 97):
            pk.he_ctx_set_multsum_variant(ctx, v)
            pk.he_counters(ctx, reset=True)
            gc = pk.he_hmatmul(ctx, ga, gb, n, n1, n1)
            cnt = pk.he_counters(ctx)
            assert (cnt["MS"], cnt["Dp"], cnt["MD"]) == (562, 176, 421)
            got, want = pk.he_ct_export(ctx, gc), res(oc)
            assert np.array_equal(got, want), "variant %d: %d of %d words differ" % (v, (got != want).sum(), got.size)
            assert pk.he_ct_info(gc)[0] == 1
            assert np.abs(pk.he_decrypt_matrix(ctx, gc, n, n) - A @ B).max() < TOL
            pk.he_ct_free(gc)
        for h in (ga, gb):
            pk.he_ct_free(h)
    finally:
        pk.he_ctx_destroy(ctx)
