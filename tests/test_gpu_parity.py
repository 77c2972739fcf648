"""Parity of the CUDA path (through the C ABI) with the oracle.

Ciphertext residues are compared element by element in coefficient form
(bit-exact); decrypted values against FP64 within 1e-4 per matrix entry.
Sizes: N = 2^14 (config 1 chain) for full residue parity; N = 2^16 with the
128x128 chain for the launch configuration the bench times (sampled parity
of a rotation, property checks of the full product)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def lib():
    import paper_2305_17341_gb300 as pk
    pk.build()
    return pk


@pytest.fixture(scope="module")
def c1(lib):
    """Config 1 chain: logN 14, q 60+3x40, p 60, seed 101, on both sides."""
    from oracle.ckks import CKKS, Params
    prm = lib.he_params_default(1)
    ctx = lib.he_ctx_create(prm, 101)
    P = Params(14, [60, 40, 40, 40], [60])
    he = CKKS(P, 101)
    yield lib, ctx, P, he
    lib.he_ctx_destroy(ctx)


def residues(he, ct):
    return np.stack([ct.c0, ct.c1])


def test_primes_match_oracle(c1):
    lib, ctx, P, he = c1
    q, p = lib.he_ctx_primes(ctx)
    assert q == P.q and p == P.p


def test_secret_key_matches(c1):
    lib, ctx, P, he = c1
    assert np.array_equal(lib.he_sk_export(ctx), he.s_int)


def test_encrypt_bit_exact_every_level(c1):
    lib, ctx, P, he = c1
    rng = np.random.default_rng(11)
    z = rng.uniform(-1, 1, P.S)
    for level in range(P.L + 1):
        g = lib.he_encrypt_slots(ctx, z, level, 1000 + level)
        o = he.encrypt_slots(z, level, obj=1000 + level)
        got = lib.he_ct_export(ctx, g)
        assert np.array_equal(got, residues(he, o)), "level %d" % level
        assert np.abs(lib.he_decrypt_slots(ctx, g, P.S) - z).max() < 1e-6
        lib.he_ct_free(g)


def test_encrypt_ragged_slot_count(c1):
    lib, ctx, P, he = c1
    z = np.random.default_rng(12).uniform(-1, 1, 1000)     # 1000 of 8192 slots, rest zero
    full = np.zeros(P.S)
    full[:1000] = z
    g = lib.he_encrypt_slots(ctx, z, P.L, 7)
    o = he.encrypt_slots(full, P.L, obj=7)
    assert np.array_equal(lib.he_ct_export(ctx, g), residues(he, o))
    lib.he_ct_free(g)


def test_import_export_roundtrip(c1):
    lib, ctx, P, he = c1
    o = he.encrypt_slots(np.random.default_rng(3).uniform(-1, 1, P.S), 2, obj=5)
    r = residues(he, o)
    g = lib.he_ct_import(ctx, r, 2, o.scale, P.S)
    assert np.array_equal(lib.he_ct_export(ctx, g), r)
    lib.he_ct_free(g)


@pytest.mark.parametrize("step", [1, 7, 4095, 8191])
def test_rotation_bit_exact(c1, step):
    lib, ctx, P, he = c1
    lib.he_keygen(ctx, [step], want_relin=False)
    he.gen_rotation_key(step)
    z = np.random.default_rng(step).uniform(-1, 1, P.S)
    for level in (P.L, 1):
        o = he.drop(he.encrypt_slots(z, P.L, obj=50 + step), level)
        g = lib.he_ct_import(ctx, residues(he, o), level, o.scale, P.S)
        gr = lib.he_rotate(ctx, g, step)
        orr = he.rotate(o, step)
        assert np.array_equal(lib.he_ct_export(ctx, gr), residues(he, orr))
        assert np.abs(lib.he_decrypt_slots(ctx, gr, P.S) - np.roll(z, -step)).max() < 1e-5
        lib.he_ct_free(g)
        lib.he_ct_free(gr)


def test_mult_relin_rescale_bit_exact(c1):
    lib, ctx, P, he = c1
    lib.he_keygen(ctx, [], want_relin=True)
    he.gen_relin_key()
    rng = np.random.default_rng(21)
    x, y = rng.uniform(-1, 1, P.S), rng.uniform(-1, 1, P.S)
    a, b = he.encrypt_slots(x, P.L, obj=61), he.encrypt_slots(y, P.L, obj=62)
    ga = lib.he_ct_import(ctx, residues(he, a), P.L, a.scale, P.S)
    gb = lib.he_ct_import(ctx, residues(he, b), P.L, b.scale, P.S)
    gm = lib.he_mult(ctx, ga, gb)
    om = he.mult_relin(a, b)
    assert np.array_equal(lib.he_ct_export(ctx, gm), residues(he, om))
    gr = lib.he_rescale(ctx, gm)
    orr = he.rescale(om)
    assert np.array_equal(lib.he_ct_export(ctx, gr), residues(he, orr))
    assert lib.he_ct_info(gr)[1] == orr.scale
    assert np.abs(lib.he_decrypt_slots(ctx, gr, P.S) - x * y).max() < 1e-6
    for h in (ga, gb, gm, gr):
        lib.he_ct_free(h)


def _matrix_pair(P, he, lib, ctx, n, seed, level=None):
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, (n, n))
    B = rng.uniform(-1, 1, (n, n))
    level = P.L if level is None else level
    za = np.zeros(P.S); za[: n * n] = A.ravel()
    zb = np.zeros(P.S); zb[: n * n] = B.ravel()
    oa, ob = he.encrypt_slots(za, level, obj=seed * 2), he.encrypt_slots(zb, level, obj=seed * 2 + 1)
    ga = lib.he_encrypt_matrix(ctx, A, level, seed * 2)
    gb = lib.he_encrypt_matrix(ctx, B, level, seed * 2 + 1)
    return A, B, oa, ob, ga, gb


def test_transpose_bit_exact(c1):
    from oracle.hmm import HMM, transpose_rot_steps
    lib, ctx, P, he = c1
    n, n1 = 32, 8
    steps = transpose_rot_steps(n, n1, P.S)
    lib.he_keygen(ctx, steps, want_relin=False)
    for s in steps:
        he.gen_rotation_key(s)
    A, _, oa, _, ga, gb = _matrix_pair(P, he, lib, ctx, n, 31)
    gt = lib.he_transpose(ctx, ga, n, n1, 1.0)
    ot = HMM(he).transpose(oa, n, n1)
    assert np.array_equal(lib.he_ct_export(ctx, gt), residues(he, ot))
    out = lib.he_decrypt_matrix(ctx, gt, n, n)
    assert np.abs(out - A.T).max() < TOL
    for h in (ga, gb, gt):
        lib.he_ct_free(h)


@pytest.mark.parametrize("relin_once", [False, True])
def test_hmatmul_config1_bit_exact(c1, relin_once):
    """Config 1: 32x32 product at N=2^14, q 60+3x40, p 60 -- residues
    bit-exact to the oracle, decrypted product within 1e-4 of FP64 A.B; with
    the per-product relinearisation of DMatrixMult and with one
    relinearisation of the summed tensors."""
    from oracle.hmm import HMM, matmul_rot_steps
    lib, ctx, P, he = c1
    n, n1 = 32, 8
    steps = matmul_rot_steps(n, n1, n1, P.S)
    lib.he_keygen(ctx, steps, want_relin=True)
    for s in steps:
        he.gen_rotation_key(s)
    he.gen_relin_key()
    A, B, oa, ob, ga, gb = _matrix_pair(P, he, lib, ctx, n, 41)
    assert np.array_equal(lib.he_ct_export(ctx, ga), residues(he, oa))
    lib.he_counters(ctx, reset=True)
    gc = lib.he_hmatmul(ctx, ga, gb, n, n1, n1, relin_once=relin_once)
    cnt = lib.he_counters(ctx)
    he.cnt.reset()
    oc = HMM(he).hmatmul(oa, ob, n, n1, n1, relin_once=relin_once)
    assert (cnt["MS"], cnt["Dp"], cnt["MD"]) == (he.cnt.MS, he.cnt.Dp, he.cnt.MD)
    got = lib.he_ct_export(ctx, gc)
    want = residues(he, oc)
    assert got.shape == want.shape
    assert np.array_equal(got, want), "mismatching residues: %d of %d" % ((got != want).sum(), got.size)
    lv, sc, per = lib.he_ct_info(gc)
    assert (lv, per) == (0, n * n) and sc == oc.scale
    out = lib.he_decrypt_matrix(ctx, gc, n, n)
    assert np.abs(out - A @ B).max() < TOL
    for h in (ga, gb, gc):
        lib.he_ct_free(h)


def test_hmatmul_batch_equals_single(c1):
    lib, ctx, P, he = c1
    n, n1 = 32, 8
    from oracle.hmm import matmul_rot_steps
    lib.he_keygen(ctx, matmul_rot_steps(n, n1, n1, P.S), want_relin=True)
    pairs = [_matrix_pair(P, he, lib, ctx, n, 70 + i) for i in range(3)]
    singles = [lib.he_hmatmul(ctx, p[4], p[5], n, n1, n1) for p in pairs]
    batch = lib.he_hmatmul_batch([(p[4], p[5], n, n1, n1) for p in pairs])
    for s, b, p in zip(singles, batch, pairs):
        assert np.array_equal(lib.he_ct_export(ctx, s), lib.he_ct_export(ctx, b))
        assert np.abs(lib.he_decrypt_matrix(ctx, b, n, n) - p[0] @ p[1]).max() < TOL
    for h in singles + batch + [x for p in pairs for x in p[4:6]]:
        lib.he_ct_free(h)


def test_hmatmul_batch_shared_operands(c1):
    """Products of one batch that share operands (Sec. 5.2, covariance
    Optimizations 1 and 2): every product bit-exact to its single
    he_hmatmul, and the shared sigma/tau, C^k and R^k run once per operand --
    4 products of 2 distinct A and 2 distinct B cost the key switches of 2
    products plus the relinearisations (one MS, Dp and MD per k) of 2 more."""
    lib, ctx, P, he = c1
    n, n1 = 32, 8
    from oracle.hmm import matmul_rot_steps
    lib.he_keygen(ctx, matmul_rot_steps(n, n1, n1, P.S), want_relin=True)
    (A0, B0, _, _, a0, b0), (A1, B1, _, _, a1, b1) = [_matrix_pair(P, he, lib, ctx, n, 110 + i) for i in range(2)]
    pairs = [(a0, b0, A0, B0), (a0, b1, A0, B1), (a1, b0, A1, B0), (a0, b0, A0, B0)]
    lib.he_counters(ctx, reset=True)
    two = lib.he_hmatmul_batch([(a0, b0, n, n1, n1), (a1, b1, n, n1, n1)])
    c2 = lib.he_counters(ctx, reset=True)
    shared = lib.he_hmatmul_batch([(x, y, n, n1, n1) for x, y, _, _ in pairs])
    c4 = lib.he_counters(ctx, reset=True)
    for key in ("MS", "Dp", "MD"):
        assert c4[key] - c2[key] == 2 * n, (key, c2, c4)
    for o, (x, y, X, Y) in zip(shared, pairs):
        s = lib.he_hmatmul(ctx, x, y, n, n1, n1)
        assert np.array_equal(lib.he_ct_export(ctx, s), lib.he_ct_export(ctx, o))
        assert np.abs(lib.he_decrypt_matrix(ctx, o, n, n) - X @ Y).max() < TOL
        lib.he_ct_free(s)
    for h in two + shared + [a0, b0, a1, b1]:
        lib.he_ct_free(h)


def test_hmatmul_levels_and_errors(c1):
    lib, ctx, P, he = c1
    n, n1 = 32, 8
    _, _, _, _, ga, gb = _matrix_pair(P, he, lib, ctx, n, 90, level=2)
    with pytest.raises(lib.HeError) as e:
        lib.he_hmatmul(ctx, ga, gb, n, n1, n1)
    assert e.value.code == -3
    with pytest.raises(lib.HeError):
        lib.he_hmatmul(ctx, ga, gb, n, 3, n1)
    lib.he_ct_free(ga)
    lib.he_ct_free(gb)


# ------------------------------------------------ full size: 128x128, N=2^16

@pytest.fixture(scope="module")
def c2(lib):
    prm = lib.he_params_default(2)
    ctx = lib.he_ctx_create(prm, 202)
    yield lib, ctx
    lib.he_ctx_destroy(ctx)


def test_full_size_rotation_sampled_parity(c2):
    """One hoisted rotation at N=2^16, level 20, 23 primes: bit-exact to the oracle."""
    from oracle.ckks import CKKS, Params
    lib, ctx = c2
    P = Params(16, [60] + [40] * 20, [60, 60])
    he = CKKS(P, 202)
    step = 16
    lib.he_keygen(ctx, [step], want_relin=False)
    he.gen_rotation_key(step)
    z = np.random.default_rng(5).uniform(-1, 1, P.S)
    o = he.encrypt_slots(z, P.L, obj=3)
    g = lib.he_encrypt_slots(ctx, z, P.L, 3)
    assert np.array_equal(lib.he_ct_export(ctx, g), residues(he, o))
    gr = lib.he_rotate(ctx, g, step)
    assert np.array_equal(lib.he_ct_export(ctx, gr), residues(he, he.rotate(o, step)))
    lib.he_ct_free(g)
    lib.he_ct_free(gr)


def test_full_size_hmatmul_properties(c2):
    """128x128 at N=2^16 (the benchmarked configuration): decrypted product
    within 1e-4 of FP64 for a batch of 2, and batch == single bit-exact."""
    lib, ctx = c2
    n, n1 = 128, 16
    lib.he_keygen(ctx, lib.he_rot_steps_for_matmul(n, n1, n1, 1 << 15), want_relin=True)
    rng = np.random.default_rng(9)
    mats = [(rng.uniform(-1, 1, (n, n)), rng.uniform(-1, 1, (n, n))) for _ in range(2)]
    cts = [(lib.he_encrypt_matrix(ctx, A, 20, 10 + 2 * i), lib.he_encrypt_matrix(ctx, B, 20, 11 + 2 * i))
           for i, (A, B) in enumerate(mats)]
    batch = lib.he_hmatmul_batch([(a, b, n, n1, n1) for a, b in cts])
    single = lib.he_hmatmul(ctx, cts[0][0], cts[0][1], n, n1, n1)
    assert np.array_equal(lib.he_ct_export(ctx, single), lib.he_ct_export(ctx, batch[0]))
    for (A, B), o in zip(mats, batch):
        err = np.abs(lib.he_decrypt_matrix(ctx, o, n, n) - A @ B).max()
        assert err < TOL, err
        assert lib.he_ct_info(o)[0] == 17
    for h in batch + [single] + [x for c in cts for x in c]:
        lib.he_ct_free(h)


@pytest.mark.parametrize("logN,qbits,pbits", [(12, [60, 40, 40], [60]), (16, [60] + [40] * 20, [60, 60])])
def test_ntt_negacyclic_product_and_roundtrip(lib, logN, qbits, pbits):
    """he_ntt (generic smem path at 2^12, register-blocked two-pass path at
    2^16): NTT, pointwise product, inverse NTT equals the oracle's
    negacyclic product in Z_q[X]/(X^N + 1); inverse(forward(x)) = x; every
    output in [0, q).  Rows cycle through the primes of Q_l P."""
    import torch
    from oracle import _c
    ctx = lib.he_ctx_create(lib.make_params(logN, qbits, pbits), 5)
    try:
        q, p = lib.he_ctx_primes(ctx)
        level = len(qbits) - 1
        primes = list(q) + list(p)
        pick = [0, 1, len(primes) - 1]                      # q0, a 40-bit q, the last special prime
        N = 1 << logN
        rng = np.random.default_rng(logN)
        a = np.stack([rng.integers(0, primes[i], N, dtype=np.uint64) for i in range(len(primes))])
        b = np.stack([rng.integers(0, primes[i], N, dtype=np.uint64) for i in range(len(primes))])
        da = torch.from_numpy(a.view(np.int64).copy()).cuda()
        db = torch.from_numpy(b.view(np.int64).copy()).cuda()
        lib.he_ntt(ctx, da.data_ptr(), len(primes), level)
        lib.he_ntt(ctx, db.data_ptr(), len(primes), level)
        fa = da.cpu().numpy().view(np.uint64)
        fb = db.cpu().numpy().view(np.uint64)
        for i in range(len(primes)):
            assert int(fa[i].max()) < primes[i] and int(fb[i].max()) < primes[i]
        prod = np.stack([np.array([(int(x) * int(y)) % primes[i] if i in pick else 0
                                   for x, y in zip(fa[i], fb[i])], dtype=np.uint64) for i in range(len(primes))])
        dp = torch.from_numpy(prod.view(np.int64).copy()).cuda()
        lib.he_ntt(ctx, dp.data_ptr(), len(primes), level, inverse=True)
        got = dp.cpu().numpy().view(np.uint64)
        for i in pick:
            assert np.array_equal(got[i], _c.polymul(primes[i], a[i], b[i])), "prime %d" % i
        lib.he_ntt(ctx, da.data_ptr(), len(primes), level, inverse=True)
        assert np.array_equal(da.cpu().numpy().view(np.uint64), a)
    finally:
        lib.he_ctx_destroy(ctx)


def test_hmatmul_batch_relin_once_equals_single(c1):
    """Batched products with one relinearisation each equal the single calls."""
    lib, ctx, P, he = c1
    n, n1 = 32, 8
    from oracle.hmm import matmul_rot_steps
    lib.he_keygen(ctx, matmul_rot_steps(n, n1, n1, P.S), want_relin=True)
    pairs = [_matrix_pair(P, he, lib, ctx, n, 80 + i) for i in range(3)]
    singles = [lib.he_hmatmul(ctx, p[4], p[5], n, n1, n1, relin_once=True) for p in pairs]
    batch = lib.he_hmatmul_batch([(p[4], p[5], n, n1, n1, True) for p in pairs])
    for s, b, p in zip(singles, batch, pairs):
        assert np.array_equal(lib.he_ct_export(ctx, s), lib.he_ct_export(ctx, b))
        assert np.abs(lib.he_decrypt_matrix(ctx, b, n, n) - p[0] @ p[1]).max() < TOL
    for h in singles + batch + [x for p in pairs for x in p[4:6]]:
        lib.he_ct_free(h)



def test_rotate_hoisted_batch_bit_exact(c1):
    """he_rotate_hoisted: three ciphertexts (two levels) x three steps, one
    Decompose per ciphertext, each output equal to the oracle's hoisted
    rotation and to he_rotate."""
    lib, ctx, P, he = c1
    steps = [1, 7, P.S - 3]
    lib.he_keygen(ctx, steps, want_relin=False)
    for s in steps:
        he.gen_rotation_key(s)
    rng = np.random.default_rng(99)
    os_, gs = [], []
    for i, level in enumerate((P.L, 2, P.L)):
        o = he.drop(he.encrypt_slots(rng.uniform(-1, 1, P.S), P.L, obj=400 + i), level)
        os_.append(o)
        gs.append(lib.he_ct_import(ctx, residues(he, o), level, o.scale, P.S))
    outs = lib.he_rotate_hoisted(ctx, gs, steps)
    for i, o in enumerate(os_):
        dg = he.modup(o.c1, o.level)
        for j, s in enumerate(steps):
            want = he.rotate_hoisted(o, dg, s)
            assert np.array_equal(lib.he_ct_export(ctx, outs[i][j]), residues(he, want)), (i, s)
            single = lib.he_rotate(ctx, gs[i], s)
            assert np.array_equal(lib.he_ct_export(ctx, single), lib.he_ct_export(ctx, outs[i][j]))
            lib.he_ct_free(single)
    for h in gs + [x for row in outs for x in row]:
        lib.he_ct_free(h)


def test_autotuned_launches_compute_the_same_words(c1):
    """The MultSum variants the autotuner chooses among (items per CTA, load
    caching) give identical residues: a product with the tuner on equals the
    same product with the fixed default launch."""
    lib, ctx, P, he = c1
    n, n1 = 32, 8
    from oracle.hmm import matmul_rot_steps
    lib.he_keygen(ctx, matmul_rot_steps(n, n1, n1, P.S), want_relin=True)
    pairs = [_matrix_pair(P, he, lib, ctx, n, 120 + i) for i in range(3)]
    jobs = [(p[4], p[5], n, n1, n1) for p in pairs]
    tuned = lib.he_hmatmul_batch(jobs)
    lib.he_ctx_set_autotune(ctx, False)
    try:
        fixed = lib.he_hmatmul_batch(jobs)
    finally:
        lib.he_ctx_set_autotune(ctx, True)
    for a, b in zip(tuned, fixed):
        assert np.array_equal(lib.he_ct_export(ctx, a), lib.he_ct_export(ctx, b))
    for h in tuned + fixed + [x for p in pairs for x in p[4:6]]:
        lib.he_ct_free(h)


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_linear_transform_bit_exact(c1, kind):
    """sigma (Z), tau (T) and G alone through he_linear_transform, bit-exact
    to the oracle's double-hoisted BSGS transforms; the decrypted sigma/tau
    match the index maps of eq. 5 / eq. 6 and G the transpose."""
    from oracle.hmm import HMM, matmul_rot_steps, transpose_rot_steps
    lib, ctx, P, he = c1
    n, n1 = 32, 8
    steps = sorted(set(matmul_rot_steps(n, n1, n1, P.S)) | set(transpose_rot_steps(n, n1, P.S)))
    lib.he_keygen(ctx, steps, want_relin=False)
    for s in steps:
        he.gen_rotation_key(s)
    A, B, oa, ob, ga, gb = _matrix_pair(P, he, lib, ctx, n, 140 + kind)
    H = HMM(he)
    r = H.replicate(oa, n)
    want = H.sigma(r, n, n1) if kind == 0 else H.tau(r, n, n1) if kind == 1 else H.transpose(oa, n, n1)
    got = lib.he_linear_transform(ctx, ga, kind, n, n1)
    assert np.array_equal(lib.he_ct_export(ctx, got), residues(he, want))
    out = lib.he_decrypt_matrix(ctx, got, n, n)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ref = A[i, (i + j) % n] if kind == 0 else A[(i + j) % n, j] if kind == 1 else A.T
    assert np.abs(out - ref).max() < TOL
    for h in (ga, gb, got):
        lib.he_ct_free(h)


@pytest.mark.parametrize("n,n1z,n1t", [(32, 1, 1), (32, 32, 32), (32, 1, 32), (32, 32, 1), (2, 1, 2), (2, 2, 1)])
def test_hmatmul_degenerate_schedules_bit_exact(c1, n, n1z, n1t):
    """Edge schedules of the double-hoisted BSGS (eq. 3', Table 1): n1 = 1
    (no baby steps, n giants), n1 = n (one giant), mixed, and the smallest
    matrix (n = 2, replicated 2048 times over the slots): residues and
    key-switch counts equal the oracle's, the product decrypts to A.B."""
    from oracle.hmm import HMM, matmul_rot_steps
    lib, ctx, P, he = c1
    steps = matmul_rot_steps(n, n1z, n1t, P.S)
    lib.he_keygen(ctx, steps, want_relin=True)
    for s in steps:
        he.gen_rotation_key(s)
    he.gen_relin_key()
    A, B, oa, ob, ga, gb = _matrix_pair(P, he, lib, ctx, n, 140 + n + n1z + 3 * n1t)
    lib.he_counters(ctx, reset=True)
    gc = lib.he_hmatmul(ctx, ga, gb, n, n1z, n1t)
    cnt = lib.he_counters(ctx)
    he.cnt.reset()
    oc = HMM(he).hmatmul(oa, ob, n, n1z, n1t)
    assert (cnt["MS"], cnt["Dp"], cnt["MD"]) == (he.cnt.MS, he.cnt.Dp, he.cnt.MD)
    assert np.array_equal(lib.he_ct_export(ctx, gc), residues(he, oc))
    assert np.abs(lib.he_decrypt_matrix(ctx, gc, n, n) - A @ B).max() < TOL
    for h in (ga, gb, gc):
        lib.he_ct_free(h)


@pytest.mark.parametrize("logN", [14, 15, 16])
def test_ntt_variants_compute_the_same_words(lib, logN):
    """Every NTT variant (one-tile CTAs at 2, 3 or 4 per SM, all rows at once
    or in chunks of rows; persistent passes fed by bulk copies: row tiles as
    contiguous copies, column tiles as 2-D tensor-map boxes; one pass per
    limb by an 8-CTA cluster at N = 2^16, as 3 below) gives the same
    forward words on a ragged number of
    rows cycling through q_0..q_L, p_0, p_1 (the 60-bit rows take the
    reducing butterflies), and the inverse returns the input."""
    import torch
    ctx = lib.he_ctx_create(lib.make_params(logN, [60] + [40] * 6, [60, 60]), 6)
    try:
        q, p = lib.he_ctx_primes(ctx)
        primes = list(q) + list(p)
        N, R, level = 1 << logN, 37, 6
        rng = np.random.default_rng(logN + 100)
        a = np.stack([rng.integers(0, primes[r % len(primes)], N, dtype=np.uint64) for r in range(R)])
        outs = {}
        # (variant, rows per launch pair): 7-row chunks leave a ragged last chunk of 2
        for v, chunk in ((2, 0), (3, 0), (5, 0), (4, 0), (6, 0), (3, 7), (5, 7), (6, 7)):
            lib.he_ctx_set_ntt_variant(ctx, v)
            lib.he_ctx_set_ntt_chunk(ctx, chunk)
            d = torch.from_numpy(a.view(np.int64).copy()).cuda()
            torch.cuda.synchronize()
            lib.he_ntt(ctx, d.data_ptr(), R, level)
            outs[(v, chunk)] = d.cpu().numpy().view(np.uint64).copy()
            lib.he_ntt(ctx, d.data_ptr(), R, level, inverse=True)
            assert np.array_equal(d.cpu().numpy().view(np.uint64), a), (v, chunk)
        for key, o in outs.items():
            assert np.array_equal(o, outs[(2, 0)]), key
        for r in range(R):
            assert int(outs[(4, 0)][r].max()) < primes[r % len(primes)]
            assert int(outs[(6, 0)][r].max()) < primes[r % len(primes)]
    finally:
        lib.he_ctx_set_ntt_chunk(ctx, 0)
        lib.he_ctx_set_ntt_variant(ctx, -1)
        lib.he_ctx_destroy(ctx)


def test_full_size_product_same_words_under_every_ntt_variant(c2):
    """The benchmarked shape (128x128, N = 2^16, level 20, two special
    primes): the product's residues are the same whether the forward NTTs
    run as two passes of one-tile CTAs, as persistent bulk-copy passes or in
    one pass per limb by 8-CTA clusters exchanging through distributed
    shared memory (Decompose with its skipped rows, the fused ModDown and
    Rescale epilogues)."""
    lib, ctx = c2
    n, n1 = 128, 16
    lib.he_keygen(ctx, lib.he_rot_steps_for_matmul(n, n1, n1, 1 << 15), want_relin=True)
    rng = np.random.default_rng(19)
    A, B = rng.uniform(-1, 1, (n, n)), rng.uniform(-1, 1, (n, n))
    a, b = lib.he_encrypt_matrix(ctx, A, 20, 90), lib.he_encrypt_matrix(ctx, B, 20, 91)
    outs = {}
    try:
        for v in (3, 6, 4):
            lib.he_ctx_set_ntt_variant(ctx, v)
            o = lib.he_hmatmul(ctx, a, b, n, n1, n1)
            outs[v] = lib.he_ct_export(ctx, o)
            if v == 6:
                assert np.abs(lib.he_decrypt_matrix(ctx, o, n, n) - A @ B).max() < TOL
            lib.he_ct_free(o)
    finally:
        lib.he_ctx_set_ntt_variant(ctx, -1)
    assert np.array_equal(outs[6], outs[3]) and np.array_equal(outs[4], outs[3])
    lib.he_ct_free(a)
    lib.he_ct_free(b)
