"""Serving loop (he_server_*): results of jobs served in one mix equal the
same circuits called alone (bit-exact residues), X^T X accumulated from
row-block jobs equals the centred covariance, admission and job failures are
reported per job."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

LOGN, QBITS, PBITS = 12, [60] + [40] * 12, [60]


@pytest.fixture(scope="module")
def env():
    import paper_2305_17341_gb300 as pk
    pk.build()
    ctx = pk.he_ctx_create(pk.make_params(LOGN, QBITS, PBITS), 21)
    n, n1 = 16, 4
    S = 1 << (LOGN - 1)
    steps = set(pk.he_rot_steps_for_matmul(n, n1, n1, S)) | set(pk.he_rot_steps_for_transpose(n, n1, S))
    i = 1
    while i < n * n:
        steps |= {i % (n * n), (-i) % (n * n)}
        i <<= 1
    steps.discard(0)
    pk.he_keygen(ctx, sorted(steps), want_relin=True)
    yield pk, ctx, n, n1
    pk.he_ctx_destroy(ctx)


def _blocks(pk, ctx, X, n, level, base):
    s, t = X.shape
    nrb, k = -(-s // n), -(-t // n)
    Xp = np.zeros((nrb * n, k * n))
    Xp[:s, :t] = X
    return [pk.he_encrypt_matrix(ctx, Xp[l * n:(l + 1) * n, j * n:(j + 1) * n], level, base + l * k + j)
            for l in range(nrb) for j in range(k)], nrb, k


def _same(pk, ctx, a, b):
    return np.array_equal(pk.he_ct_export(ctx, a), pk.he_ct_export(ctx, b))


def test_served_mix_equals_alone(env):
    from paper_2305_17341_gb300.workloads import lowrank_dataset, matmul_pair
    pk, ctx, n, n1 = env
    L = len(QBITS) - 1
    pairs = [matmul_pair(n, 40 + i) for i in range(3)]
    mm = [(pk.he_encrypt_matrix(ctx, A, L - i, 60 + 2 * i), pk.he_encrypt_matrix(ctx, B, L - i, 61 + 2 * i))
          for i, (A, B) in enumerate(pairs)]
    X = lowrank_dataset(40, 32, 5)                       # 3 row blocks (last one ragged), k = 2
    blocks, nrb, k = _blocks(pk, ctx, X, n, L, 100)
    # alone
    want_mm = [pk.he_hmatmul(ctx, a, b, n, n1, n1) for a, b in mm]
    want_cov = pk.he_covariance(ctx, blocks, nrb, k, n, X.shape[0], False, n1, n1)
    want_xtx = pk.he_covariance(ctx, blocks, nrb, k, n, X.shape[0], True, n1, n1)
    # served: everything submitted at once
    srv = pk.he_server_create([ctx], 64e9, max_batch=4)
    try:
        ids_mm = [pk.he_server_submit(srv, pk.HE_JOB_MATMUL, [a, b], n=n, n1z=n1, n1t=n1) for a, b in mm]
        id_cov = pk.he_server_submit(srv, pk.HE_JOB_COVARIANCE, blocks, n=n, n1z=n1, n1t=n1, n_row_blocks=nrb,
                                     k=k, s=X.shape[0])
        ids_blk = [pk.he_server_submit(srv, pk.HE_JOB_XTX_BLOCK, blocks[l * k:(l + 1) * k], n=n, n1z=n1, n1t=n1,
                                       k=k, s=X.shape[0], acc_id=7) for l in (2, 0, 1)]
        id_fin = pk.he_server_submit(srv, pk.HE_JOB_XTX_FINAL, [], ctx=ctx, n=n, n1z=n1, n1t=n1, k=k, acc_id=7)
        for j in ids_mm + [id_cov] + ids_blk + [id_fin]:
            assert pk.he_server_wait(srv, j, 600.0) == pk.HE_JOB_DONE
        got_mm = [pk.he_server_result(srv, j)[0][0] for j in ids_mm]
        got_cov = pk.he_server_result(srv, id_cov)[0]
        for j in ids_blk:
            assert pk.he_server_result(srv, j) == ([], [])
        got_xtx = pk.he_server_result(srv, id_fin)[0]
        st = pk.he_server_stats(srv)
    finally:
        pk.he_server_destroy(srv)
    for g, w in zip(got_mm, want_mm):
        assert _same(pk, ctx, g, w)
    assert len(got_cov) == k * k and len(got_xtx) == k * k
    for i in range(k * k):
        assert _same(pk, ctx, got_cov[i], want_cov[i]), i
        assert _same(pk, ctx, got_xtx[i], want_xtx[i]), i
    Xc = X - X.mean(0)
    ref = Xc.T @ Xc / X.shape[0]
    for a in range(k):
        for b in range(k):
            d = pk.he_decrypt_matrix(ctx, got_cov[a * k + b], n, n)
            assert np.abs(d - ref[a * n:(a + 1) * n, b * n:(b + 1) * n]).max() < 1e-4
    assert st["completed"] == 8 and st["failed"] == 0 and st["rejected"] == 0
    assert st["products"] == 3 + nrb * 3 + 3 * 3
    assert st["charged_bytes"] == pytest.approx(0.0, abs=1.0)
    assert st["p99_ms"] >= st["p50_ms"] > 0
    for h in got_mm + got_cov + got_xtx + want_mm + want_cov + want_xtx + blocks + [x for p in mm for x in p]:
        pk.he_ct_free(h)


def test_admission_and_per_job_failures(env):
    from paper_2305_17341_gb300.workloads import matmul_pair
    pk, ctx, n, n1 = env
    L = len(QBITS) - 1
    A, B = matmul_pair(n, 3)
    a, b = pk.he_encrypt_matrix(ctx, A, L, 1), pk.he_encrypt_matrix(ctx, B, L, 2)
    # a budget below one product's charge rejects it
    srv = pk.he_server_create([ctx], 1e6, max_batch=2)
    try:
        with pytest.raises(pk.HeError) as e:
            pk.he_server_submit(srv, pk.HE_JOB_MATMUL, [a, b], n=n, n1z=n1, n1t=n1)
        assert e.value.code == pk.HE_ERR_ADMISSION
        st = pk.he_server_stats(srv)
        assert (st["submitted"], st["admitted"], st["rejected"]) == (1, 0, 1)
    finally:
        pk.he_server_destroy(srv)
    srv = pk.he_server_create([ctx], 64e9, max_batch=2)
    try:
        # a schedule whose keys were not generated (n1 = 8) is refused at submission
        with pytest.raises(pk.HeError) as e:
            pk.he_server_submit(srv, pk.HE_JOB_MATMUL, [a, b], n=n, n1z=8, n1t=8)
        assert e.value.code == pk.HE_ERR_KEY_MISSING
        # a final without row blocks fails on the worker; the product queued
        # with it still completes and matches the direct call
        j_bad = pk.he_server_submit(srv, pk.HE_JOB_XTX_FINAL, [], ctx=ctx, n=n, n1z=n1, n1t=n1, k=2, acc_id=99)
        j_ok = pk.he_server_submit(srv, pk.HE_JOB_MATMUL, [a, b], n=n, n1z=n1, n1t=n1)
        assert pk.he_server_wait(srv, j_bad, 600.0) == pk.HE_JOB_FAILED
        assert pk.he_server_wait(srv, j_ok, 600.0) == pk.HE_JOB_DONE
        assert pk.he_server_poll(srv, j_bad)[1] == pk.HE_ERR_ARG
        with pytest.raises(pk.HeError):
            pk.he_server_result(srv, j_bad)
        out = pk.he_server_result(srv, j_ok)[0][0]
        st = pk.he_server_stats(srv)
        assert (st["completed"], st["failed"]) == (1, 1)
    finally:
        pk.he_server_destroy(srv)
    ref = pk.he_hmatmul(ctx, a, b, n, n1, n1)
    assert _same(pk, ctx, out, ref)
    for h in (a, b, out, ref):
        pk.he_ct_free(h)


def test_served_pca_equals_alone(env):
    from oracle.pca import lazy_normalization_schedule
    from paper_2305_17341_gb300.workloads import lowrank_dataset
    pk, ctx, n, n1 = env
    L = len(QBITS) - 1
    k, t, l_E, l_P = 2, 32, 2, 2
    X = lowrank_dataset(64, t, 8)
    Xc = X - X.mean(0)
    Cs = (Xc.T @ Xc / 64) * t
    def enc(blk, obj):
        # every n x n period of the slots holds the block (period n^2)
        h = pk.he_encrypt_slots(ctx, np.tile(blk.ravel(), (1 << (LOGN - 1)) // (n * n)), L, obj)
        r = pk.he_ct_import(ctx, pk.he_ct_export(ctx, h), L, pk.he_ct_info(h)[1], n * n)
        pk.he_ct_free(h)
        return r

    cov = [enc(Cs[a * n:(a + 1) * n, b * n:(b + 1) * n], 900 + a * k + b) for a in range(k) for b in range(k)]
    rng = np.random.default_rng(2)
    v0 = []
    for m in range(l_E):
        v = rng.standard_normal(t)
        v /= np.linalg.norm(v)
        v0 += [enc(np.tile(v[j * n:(j + 1) * n], n), 950 + 10 * m + j) for j in range(k)]
    counts = lazy_normalization_schedule(l_P)
    rs = pk.he_refresh_state(1 << 20, 0)
    lams, V, axes = pk.he_pca(ctx, cov, k, n, l_E, v0, 0, l_P, counts, 2.0 ** 16, rs)
    srv = pk.he_server_create([ctx], 64e9, max_batch=2)
    try:
        j = pk.he_server_submit(srv, pk.HE_JOB_PCA, cov + v0, n=n, k=k, l_E=l_E, l_P=l_P, axis=0, counts=counts,
                                B2=2.0 ** 16, refresh_obj=1 << 20)
        assert pk.he_server_wait(srv, j, 900.0) == pk.HE_JOB_DONE
        outs, aux = pk.he_server_result(srv, j)
    finally:
        pk.he_server_destroy(srv)
    assert aux == axes + [rs.count]
    assert len(outs) == l_E + l_E * k
    for m in range(l_E):
        assert _same(pk, ctx, outs[m], lams[m])
        for jj in range(k):
            assert _same(pk, ctx, outs[l_E + m * k + jj], V[m][jj])
    for h in outs + lams + [x for v in V for x in v] + cov + v0:
        pk.he_ct_free(h)


def test_jobs_wait_for_memory_and_are_admitted_in_order(env):
    """A budget that holds one product's charge: later products wait
    (HE_JOB_WAITING) and are admitted in order as results are taken; each
    result equals the direct call.  reject_when_full turns waiting into
    HE_ERR_ADMISSION."""
    from paper_2305_17341_gb300.workloads import matmul_pair
    pk, ctx, n, n1 = env
    L = len(QBITS) - 1
    pairs = [matmul_pair(n, 200 + i) for i in range(3)]
    cts = [(pk.he_encrypt_matrix(ctx, A, L, 2 * i), pk.he_encrypt_matrix(ctx, B, L, 2 * i + 1))
           for i, (A, B) in enumerate(pairs)]
    srv = pk.he_server_create([ctx], 64e9)
    j = pk.he_server_submit(srv, pk.HE_JOB_MATMUL, list(cts[0]), n=n, n1z=n1, n1t=n1)
    charge = pk.he_server_stats(srv)["charged_bytes"]
    pk.he_server_wait(srv, j, 600.0)
    for h in pk.he_server_result(srv, j)[0]:
        pk.he_ct_free(h)
    pk.he_server_destroy(srv)
    assert charge > 0
    srv = pk.he_server_create([ctx], 1.5 * charge, max_batch=2)
    try:
        ids = [pk.he_server_submit(srv, pk.HE_JOB_MATMUL, list(p), n=n, n1z=n1, n1t=n1) for p in cts]
        assert [pk.he_server_poll(srv, i)[0] for i in ids[1:]] == [pk.HE_JOB_WAITING] * 2
        outs = []
        for i in ids:
            assert pk.he_server_wait(srv, i, 600.0) == pk.HE_JOB_DONE
            outs.append(pk.he_server_result(srv, i)[0][0])     # frees the charge: the next job is admitted
        st = pk.he_server_stats(srv)
        assert (st["admitted"], st["waited"], st["rejected"], st["completed"]) == (3, 2, 0, 3)
    finally:
        pk.he_server_destroy(srv)
    for (a, b), o in zip(cts, outs):
        ref = pk.he_hmatmul(ctx, a, b, n, n1, n1)
        assert _same(pk, ctx, o, ref)
        pk.he_ct_free(ref)
    srv = pk.he_server_create([ctx], 1.5 * charge, max_batch=2, reject_when_full=True)
    try:
        j1 = pk.he_server_submit(srv, pk.HE_JOB_MATMUL, list(cts[0]), n=n, n1z=n1, n1t=n1)
        with pytest.raises(pk.HeError) as e:
            pk.he_server_submit(srv, pk.HE_JOB_MATMUL, list(cts[1]), n=n, n1z=n1, n1t=n1)
        assert e.value.code == pk.HE_ERR_ADMISSION
        pk.he_server_wait(srv, j1, 600.0)
        for h in pk.he_server_result(srv, j1)[0]:
            pk.he_ct_free(h)
    finally:
        pk.he_server_destroy(srv)
    for h in outs + [x for p in cts for x in p]:
        pk.he_ct_free(h)


def test_served_decomposed_covariance_and_products(env):
    """Jobs with a Diagonal Convergence Decomposition in their schedule (a
    covariance at n' = 8, a product with Z and T decomposed) served in one
    mix equal the same calls alone, bit for bit."""
    from paper_2305_17341_gb300.workloads import lowrank_dataset, matmul_pair
    pk, ctx, n, n1 = env
    L = len(QBITS) - 1
    A, B = matmul_pair(n, 77)
    a, b = pk.he_encrypt_matrix(ctx, A, L, 700), pk.he_encrypt_matrix(ctx, B, L, 701)
    X = lowrank_dataset(32, 32, 8)
    blocks, nrb, k = _blocks(pk, ctx, X, n, L, 720)
    want_mm = pk.he_hmatmul(ctx, a, b, n, n1, n1, dcd_z=8, dcd_t=8)
    want_cov = pk.he_covariance(ctx, blocks, nrb, k, n, X.shape[0], False, n1, n1, dcd_z=8, dcd_t=8)
    srv = pk.he_server_create([ctx], 64e9, max_batch=4)
    try:
        j_mm = pk.he_server_submit(srv, pk.HE_JOB_MATMUL, [a, b], n=n, n1z=n1, n1t=n1, dcd_z=8, dcd_t=8)
        j_cov = pk.he_server_submit(srv, pk.HE_JOB_COVARIANCE, blocks, n=n, n1z=n1, n1t=n1, n_row_blocks=nrb, k=k,
                                    s=X.shape[0], dcd_z=8, dcd_t=8)
        for j in (j_mm, j_cov):
            assert pk.he_server_wait(srv, j, 600.0) == pk.HE_JOB_DONE
        got_mm = pk.he_server_result(srv, j_mm)[0][0]
        got_cov = pk.he_server_result(srv, j_cov)[0]
    finally:
        pk.he_server_destroy(srv)
    assert _same(pk, ctx, got_mm, want_mm)
    for i in range(k * k):
        assert _same(pk, ctx, got_cov[i], want_cov[i]), i
    for h in [a, b, want_mm, got_mm] + blocks + list(want_cov) + list(got_cov):
        pk.he_ct_free(h)
