"""Captured batched products (he_mm_plan_*): every replay equals
he_hmatmul_batch on the same jobs, bit for bit, for a batch that mixes
levels (two groups) and replication states."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LOGN, QBITS, PBITS = 12, [60] + [40] * 8, [60]


@pytest.fixture(scope="module")
def env():
    import paper_2305_17341_gb300 as pk
    pk.build()
    ctx = pk.he_ctx_create(pk.make_params(LOGN, QBITS, PBITS), 33)
    n, n1 = 16, 4
    pk.he_keygen(ctx, pk.he_rot_steps_for_matmul(n, n1, n1, 1 << (LOGN - 1)), want_relin=True)
    yield pk, ctx, n, n1
    pk.he_ctx_destroy(ctx)


def test_plan_replays_equal_batch(env):
    from paper_2305_17341_gb300.workloads import matmul_pair
    pk, ctx, n, n1 = env
    L = len(QBITS) - 1
    cts, mats = [], []
    for i, lv in enumerate((L, L, L - 2, L)):
        A, B = matmul_pair(n, 90 + i)
        mats.append((A, B))
        cts.append((pk.he_encrypt_matrix(ctx, A, lv, 2 * i), pk.he_encrypt_matrix(ctx, B, lv, 2 * i + 1)))
    # one operand already replicated (period n^2): a third group
    rep = pk.he_replicate(ctx, cts[3][0], n)
    jobs = [(a, b, n, n1, n1) for a, b in cts[:3]] + [(rep, cts[3][1], n, n1, n1)]
    want = pk.he_hmatmul_batch(jobs)
    plan = pk.he_mm_plan_create(jobs)
    try:
        info = pk.he_mm_plan_info(plan)
        assert info["launches"] > 100 and info["bytes"] > 0
        for _ in range(2):
            pk.he_counters(ctx, reset=True)
            got = pk.he_mm_plan_run(plan)
            assert pk.he_counters(ctx)["launches"] == info["launches"]
            for g, w in zip(got, want):
                assert np.array_equal(pk.he_ct_export(ctx, g), pk.he_ct_export(ctx, w))
                assert pk.he_ct_info(g) == pk.he_ct_info(w)
            for (A, B), g in zip(mats, got):
                assert np.abs(pk.he_decrypt_matrix(ctx, g, n, n) - A @ B).max() < 1e-4
            for g in got:
                pk.he_ct_free(g)
    finally:
        pk.he_mm_plan_destroy(plan)
    for h in want + [rep] + [x for p in cts for x in p]:
        pk.he_ct_free(h)


def test_plan_refuses_missing_keys_and_operands_of_two_contexts(env):
    """A plan may hold jobs of several contexts (each group a branch), but
    not a job whose operands belong to two contexts, nor a job of a context
    without the product's rotation keys."""
    pk, ctx, n, n1 = env
    L = len(QBITS) - 1
    a = pk.he_encrypt_matrix(ctx, np.eye(n), L, 1)
    with pytest.raises(pk.HeError) as e:
        pk.he_mm_plan_create([(a, a, n, 8, 8)])
    assert e.value.code == pk.HE_ERR_KEY_MISSING
    other = pk.he_ctx_create(pk.make_params(LOGN, QBITS, PBITS), 34)
    try:
        b = pk.he_encrypt_matrix(other, np.eye(n), L, 1)
        with pytest.raises(pk.HeError) as e:
            pk.he_mm_plan_create([(a, b, n, n1, n1)])
        assert e.value.code == pk.HE_ERR_ARG
        with pytest.raises(pk.HeError) as e:
            pk.he_mm_plan_create([(a, a, n, n1, n1), (b, b, n, n1, n1)])
        assert e.value.code == pk.HE_ERR_KEY_MISSING
        pk.he_ct_free(b)
    finally:
        pk.he_ctx_destroy(other)
    pk.he_ct_free(a)
