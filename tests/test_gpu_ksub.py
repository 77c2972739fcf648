"""Simple key substitution (Sec. 4.2, Table 2's SmpKeySub rows) on the GPU:
sigma and tau through he_linear_transform_ksub with only the keys of the
babies' head, bit-exact to the oracle's same schedule, with its MultSum /
Decompose / ModDown counts, decrypting to the index maps of eq. 5 / eq. 6.
Config 1 chain (N = 2^14, q 60 + 3x40, p 60), 32 x 32 matrices, n1 = 8."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_MAT, N1 = 32, 8


@pytest.fixture(scope="module")
def setup():
    import paper_2305_17341_gb300 as pk
    from oracle.ckks import CKKS, Params
    pk.build()
    ctx = pk.he_ctx_create(pk.he_params_default(1), 77)
    P = Params(14, [60, 40, 40, 40], [60])
    he = CKKS(P, 77)
    q, p = pk.he_ctx_primes(ctx)
    assert list(q) == P.q and list(p) == P.p
    steps = set()
    for kind in (0, 1):
        for head in (2, 3, 5, 8):
            steps |= set(pk.he_rot_steps_for_ksub(N_MAT, kind, N1, head, P.S))
    pk.he_keygen(ctx, sorted(steps), want_relin=False)
    for s in sorted(steps):
        he.gen_rotation_key(s)
    yield pk, ctx, P, he
    pk.he_ctx_destroy(ctx)


@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("head", [2, 3, 5, 8])
def test_key_substitution_bit_exact_to_oracle(setup, kind, head):
    from oracle.hmm import HMM, ksub_rot_steps
    pk, ctx, P, he = setup
    n = N_MAT
    n2 = n // N1
    # the transform's own keys are Table 2's MinRotKeys
    assert len(ksub_rot_steps(n, kind, N1, head)) == head + (2 * n2 if kind == 0 else n2) - 2
    rng = np.random.default_rng(100 + 10 * kind + head)
    A = rng.uniform(-1, 1, (n, n))
    za = np.zeros(P.S)
    za[: n * n] = A.ravel()
    obj = 500 + 10 * kind + head
    oa = he.encrypt_slots(za, P.L, obj=obj)
    ga = pk.he_encrypt_matrix(ctx, A, P.L, obj)
    H = HMM(he)
    r = H.replicate(oa, n)
    gr = pk.he_replicate(ctx, ga, n)
    assert np.array_equal(pk.he_ct_export(ctx, gr), np.stack([r.c0, r.c1]))
    he.cnt.reset()
    want = H.sigma(r, n, N1, head) if kind == 0 else H.tau(r, n, N1, head)
    pk.he_counters(ctx, reset=True)
    got = pk.he_linear_transform_ksub(ctx, gr, kind, n, N1, head)
    cnt = pk.he_counters(ctx)
    assert (cnt["MS"], cnt["Dp"], cnt["MD"]) == (he.cnt.MS, he.cnt.Dp, he.cnt.MD)
    assert np.array_equal(pk.he_ct_export(ctx, got), np.stack([want.c0, want.c1]))
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ref = A[i, (i + j) % n] if kind == 0 else A[(i + j) % n, j]
    assert np.abs(pk.he_decrypt_matrix(ctx, got, n, n) - ref).max() < 1e-4
    for h in (ga, gr, got):
        pk.he_ct_free(h)


def test_key_substitution_refuses_bad_arguments(setup):
    pk, ctx, P, he = setup
    ga = pk.he_encrypt_matrix(ctx, np.zeros((N_MAT, N_MAT)), P.L, 999)
    try:
        for kind, n1, head in ((2, 8, 2), (0, 6, 2), (0, 8, 1), (0, 8, 9)):
            with pytest.raises(pk.HeError):
                pk.he_linear_transform_ksub(ctx, ga, kind, N_MAT, n1, head)
    finally:
        pk.he_ct_free(ga)
