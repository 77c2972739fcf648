"""Mixed batches (uneven block sizes, levels and ring degrees in one step).

The jobs of one captured plan are grouped by (context, level, block size,
schedule) and every group runs as a concurrent branch of one CUDA graph.
The outputs must be the words of the unbatched product, of the grouped
batch and -- for a sample at N = 2^15 with the 60 + 20 x 40 / 2 x 60 chain of
the mixed workload -- of the oracle; decrypted products within 1e-4 of
FP64 A.B."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-4
N1_FOR = {8: 2, 16: 4, 32: 8}


def res(ct):
    return np.stack([ct.c0, ct.c1])


def test_mixed_plan_equals_plain_batch_and_oracle():
    import paper_2305_17341_gb300 as pk
    from oracle.ckks import CKKS, Params
    from oracle.hmm import HMM, matmul_rot_steps
    pk.build()
    # the mixed workload's N = 2^15 context (chain of the 128x128 preset)
    qbits, pbits = [60] + [40] * 20, [60, 60]
    P = Params(15, qbits, pbits)
    ctx15 = pk.he_ctx_create(pk.he_params_default(4), 15)
    # a second context of another ring degree in the same plan
    ctx14 = pk.he_ctx_create(pk.he_params_default(1), 14)
    try:
        assert pk.he_ctx_primes(ctx15)[0] == P.q
        he = CKKS(P, 15)
        steps15 = sorted(set(matmul_rot_steps(16, 4, 4, P.S)) | set(matmul_rot_steps(32, 8, 8, P.S)))
        pk.he_keygen(ctx15, steps15, want_relin=True)
        steps14 = pk.he_rot_steps_for_matmul(8, 2, 2, 1 << 13)
        pk.he_keygen(ctx14, steps14, want_relin=True)
        rng = np.random.default_rng(44)
        # (context, n, level); two jobs share (n, level) so that one branch batches them
        spec = [(ctx15, 16, 3), (ctx15, 32, 5), (ctx15, 16, 4), (ctx15, 16, 3), (ctx14, 8, 3), (ctx15, 32, 3)]
        mats, cts = [], []
        for i, (ctx, n, level) in enumerate(spec):
            A, B = rng.uniform(-1, 1, (n, n)), rng.uniform(-1, 1, (n, n))
            mats.append((A, B))
            cts.append((pk.he_encrypt_matrix(ctx, A, level, 2 * i), pk.he_encrypt_matrix(ctx, B, level, 2 * i + 1)))
        jobs = [(a, b, n, N1_FOR[n], N1_FOR[n]) for (a, b), (_, n, _) in zip(cts, spec)]
        plain = [pk.he_hmatmul(ctx, a, b, n, N1_FOR[n], N1_FOR[n]) for (a, b), (ctx, n, _) in zip(cts, spec)]
        batch = pk.he_hmatmul_batch(jobs)
        plan = pk.he_mm_plan_create(jobs)
        runs = [pk.he_mm_plan_run(plan) for _ in range(2)]
        for i, (ctx, n, level) in enumerate(spec):
            want = pk.he_ct_export(ctx, plain[i])
            assert np.array_equal(pk.he_ct_export(ctx, batch[i]), want), i
            for r in runs:
                assert np.array_equal(pk.he_ct_export(ctx, r[i]), want), i
            A, B = mats[i]
            assert np.abs(pk.he_decrypt_matrix(ctx, runs[1][i], n, n) - A @ B).max() < TOL
            assert pk.he_ct_info(runs[1][i])[0] == level - 3
        # a sample of the N = 2^15 jobs against the oracle
        for s in sorted(set(matmul_rot_steps(16, 4, 4, P.S)) | set(matmul_rot_steps(32, 8, 8, P.S))):
            he.gen_rotation_key(s)
        he.gen_relin_key()
        H = HMM(he)
        for i in (0, 1):
            ctx, n, level = spec[i]
            A, B = mats[i]
            za, zb = np.zeros(P.S), np.zeros(P.S)
            za[: n * n], zb[: n * n] = A.ravel(), B.ravel()
            oa, ob = he.encrypt_slots(za, level, obj=2 * i), he.encrypt_slots(zb, level, obj=2 * i + 1)
            assert np.array_equal(pk.he_ct_export(ctx, cts[i][0]), res(oa))
            oc = H.hmatmul(oa, ob, n, N1_FOR[n], N1_FOR[n])
            assert np.array_equal(pk.he_ct_export(ctx, runs[1][i]), res(oc)), i
        pk.he_mm_plan_destroy(plan)
        for h in plain + batch + [x for r in runs for x in r] + [x for c in cts for x in c]:
            pk.he_ct_free(h)
    finally:
        pk.he_ctx_destroy(ctx15)
        pk.he_ctx_destroy(ctx14)
