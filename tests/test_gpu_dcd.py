"""Diagonal Convergence Decomposition on the GPU (Sec. 4.2): decomposed
sigma / tau alone and inside the matrix product, bit-exact to the oracle's
decomposition chains; batched, single and graph-replayed products agree."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LOGN, QBITS, PBITS = 12, [60] + [40] * 8, [60]


@pytest.fixture(scope="module")
def env():
    import paper_2305_17341_gb300 as pk
    from oracle.ckks import CKKS, Params
    from oracle.hmm import matmul_rot_steps
    pk.build()
    n, n1 = 16, 4
    P = Params(LOGN, QBITS, PBITS)
    ctx = pk.he_ctx_create(pk.make_params(LOGN, QBITS, PBITS), 41)
    he = CKKS(P, 41)
    steps = set()
    for dz, dt in ((8, 8), (4, 4), (8, 0), (0, 4)):
        steps |= set(matmul_rot_steps(n, n1, n1, P.S, dz, dt))
    steps = sorted(steps)
    pk.he_keygen(ctx, steps, want_relin=True)
    for s in steps:
        he.gen_rotation_key(s)
    he.gen_relin_key()
    yield pk, ctx, P, he, n, n1
    pk.he_ctx_destroy(ctx)


def _pair(pk, ctx, P, he, n, seed):
    rng = np.random.default_rng(seed)
    A, B = rng.uniform(-1, 1, (n, n)), rng.uniform(-1, 1, (n, n))
    out = []
    for M, obj in ((A, 2 * seed), (B, 2 * seed + 1)):
        z = np.zeros(P.S)
        z[: n * n] = M.ravel()
        o = he.encrypt_slots(z, P.L, obj=obj)
        g = pk.he_ct_import(ctx, np.stack([o.c0, o.c1]), P.L, o.scale, P.S)
        out.append((o, g))
    return A, B, out


def res(ct):
    return np.stack([ct.c0, ct.c1])


@pytest.mark.parametrize("n_prime", [4, 8])
def test_decomposed_sigma_tau_bit_exact(env, n_prime):
    from oracle.hmm import HMM
    pk, ctx, P, he, n, n1 = env
    A, B, ((oa, ga), (ob, gb)) = _pair(pk, ctx, P, he, n, 30 + n_prime)
    H = HMM(he)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for kind, want, ref in ((0, H.sigma_dcd(H.replicate(oa, n), n, n1, n_prime), A[i, (i + j) % n]),
                            (1, H.tau_dcd(H.replicate(oa, n), n, n1, n_prime), A[(i + j) % n, j])):
        got = pk.he_linear_transform(ctx, ga, kind, n, n1, n_prime)
        m = ((n - 1) if kind == 0 else (n - 2)) // n_prime + 1
        assert pk.he_ct_info(got)[0] == P.L - m
        assert np.array_equal(pk.he_ct_export(ctx, got), res(want)), kind
        assert np.abs(pk.he_decrypt_matrix(ctx, got, n, n) - ref).max() < 1e-4
        pk.he_ct_free(got)
    pk.he_ct_free(ga)
    pk.he_ct_free(gb)


@pytest.mark.parametrize("dz,dt", [(8, 8), (4, 4), (8, 0), (0, 4)])
def test_decomposed_product_bit_exact(env, dz, dt):
    from oracle.hmm import HMM
    pk, ctx, P, he, n, n1 = env
    A, B, ((oa, ga), (ob, gb)) = _pair(pk, ctx, P, he, n, 50 + dz + dt)
    pk.he_counters(ctx, reset=True)
    gc = pk.he_hmatmul(ctx, ga, gb, n, n1, n1, dcd_z=dz, dcd_t=dt)
    cnt = pk.he_counters(ctx)
    he.cnt.reset()
    oc = HMM(he).hmatmul(oa, ob, n, n1, n1, dcd_z=dz, dcd_t=dt)
    assert (cnt["MS"], cnt["Dp"], cnt["MD"]) == (he.cnt.MS, he.cnt.Dp, he.cnt.MD)
    depth = 2 + max((n - 1) // dz + 1 if dz else 1, (n - 2) // dt + 1 if dt else 1)
    lv, sc, per = pk.he_ct_info(gc)
    assert lv == P.L - depth == oc.level and sc == oc.scale
    assert np.array_equal(pk.he_ct_export(ctx, gc), res(oc))
    assert np.abs(pk.he_decrypt_matrix(ctx, gc, n, n) - A @ B).max() < 1e-4
    for h in (ga, gb, gc):
        pk.he_ct_free(h)


def test_decomposed_batch_graph_and_single_agree(env):
    pk, ctx, P, he, n, n1 = env
    pairs = [_pair(pk, ctx, P, he, n, 70 + i) for i in range(3)]
    jobs = [(p[2][0][1], p[2][1][1], n, n1, n1, False, 8, 8) for p in pairs]
    singles = [pk.he_hmatmul(ctx, j[0], j[1], n, n1, n1, dcd_z=8, dcd_t=8) for j in jobs]
    batch = pk.he_hmatmul_batch(jobs)
    plan = pk.he_mm_plan_create(jobs)
    try:
        replay = pk.he_mm_plan_run(plan)
    finally:
        pk.he_mm_plan_destroy(plan)
    for s, b, r in zip(singles, batch, replay):
        assert np.array_equal(pk.he_ct_export(ctx, s), pk.he_ct_export(ctx, b))
        assert np.array_equal(pk.he_ct_export(ctx, s), pk.he_ct_export(ctx, r))
    for h in singles + batch + replay + [x for p in pairs for x in (p[2][0][1], p[2][1][1])]:
        pk.he_ct_free(h)


@pytest.mark.parametrize("n_prime", [5, 15])
def test_decomposed_divisor_schedules_bit_exact(env, n_prime):
    """n1 = 1 with an n' dividing n - 1: Z's chain takes floor((n-1)/n') + 1
    factors so that its left factor stays inside its BSGS range [0, n');
    sigma, tau and the product are bit-exact to the oracle and decrypt
    correctly."""
    from oracle.hmm import HMM, matmul_rot_steps
    pk, ctx, P, he, n, _ = env
    n1 = 1
    steps = matmul_rot_steps(n, n1, n1, P.S, n_prime, n_prime)
    pk.he_keygen(ctx, steps, want_relin=True)
    for s in steps:
        he.gen_rotation_key(s)
    A, B, ((oa, ga), (ob, gb)) = _pair(pk, ctx, P, he, n, 60 + n_prime)
    H = HMM(he)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    for kind, want, ref in ((0, H.sigma_dcd(H.replicate(oa, n), n, n1, n_prime), A[i, (i + j) % n]),
                            (1, H.tau_dcd(H.replicate(oa, n), n, n1, n_prime), A[(i + j) % n, j])):
        got = pk.he_linear_transform(ctx, ga, kind, n, n1, n_prime)
        assert np.array_equal(pk.he_ct_export(ctx, got), res(want)), kind
        assert np.abs(pk.he_decrypt_matrix(ctx, got, n, n) - ref).max() < 1e-4
        pk.he_ct_free(got)
    gc = pk.he_hmatmul(ctx, ga, gb, n, n1, n1, dcd_z=n_prime, dcd_t=n_prime)
    oc = H.hmatmul(oa, ob, n, n1, n1, dcd_z=n_prime, dcd_t=n_prime)
    assert np.array_equal(pk.he_ct_export(ctx, gc), res(oc))
    assert np.abs(pk.he_decrypt_matrix(ctx, gc, n, n) - A @ B).max() < 1e-4
    for h in (ga, gb, gc):
        pk.he_ct_free(h)
