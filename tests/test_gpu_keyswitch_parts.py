"""Decompose and ModDown alone through the C ABI (he_decompose, he_moddown)
against the oracle, word for word, in coefficient form.

Chains: config 1 (N = 2^14, q 60 + 3x40, one 60-bit special prime) and the
128x128 chain (N = 2^16, q 60 + 20x40, two 60-bit special primes), at the
top level (a one-prime last digit at level 20 with alpha = 2), a level with
full digits and level 0.  ModDown also runs on coefficients placed at the
overflow boundary of its fast conversion (sum_j y_j / p_j just below an
integer), where the result must still be round(X / P) (App. A KeySwitch)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

CHAINS = [(14, [60, 40, 40, 40], [60]), (16, [60] + [40] * 20, [60, 60])]
LEVELS = {14: [3, 2, 0], 16: [20, 19, 0]}
B = 2


@pytest.fixture(scope="module")
def lib():
    import paper_2305_17341_gb300 as pk
    pk.build()
    return pk


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64).copy()).cuda()


def _host(t):
    return t.cpu().numpy().view(np.uint64)


def _crt(res, qs):
    Q = 1
    for q in qs:
        Q *= q
    x = 0
    for r, q in zip(res, qs):
        Qi = Q // q
        x += int(r) * Qi * pow(Qi, -1, q)
    return x % Q, Q


def _boundary_p_residues(ps, ks):
    """uP with S = sum_j y_j (P/p_j) = -k mod P: y_j = -k (P/p_j)^-1 mod p_j,
    uP_j = y_j (P/p_j) - (P-1)/2 mod p_j."""
    P = 1
    for p in ps:
        P *= p
    h = (P - 1) // 2
    uP = np.zeros((len(ps), len(ks)), dtype=np.uint64)
    for c, k in enumerate(ks):
        for j, p in enumerate(ps):
            ph = P // p
            uP[j, c] = (((-k * pow(ph, -1, p)) % p) * ph - h) % p
    return uP, P


def _setup(lib, chain):
    from oracle.ckks import CKKS, Params
    logN, qbits, pbits = chain
    ctx = lib.he_ctx_create(lib.make_params(logN, qbits, pbits), 5)
    P = Params(logN, qbits, pbits)
    q, p = lib.he_ctx_primes(ctx)
    assert list(q) == P.q and list(p) == P.p
    return ctx, P, CKKS(P, 5)


@pytest.mark.parametrize("chain", CHAINS, ids=["n14_alpha1", "n16_alpha2"])
def test_decompose_equals_oracle(lib, chain):
    import torch
    ctx, P, he = _setup(lib, chain)
    try:
        rng = np.random.default_rng(21)
        for level in LEVELS[P.logN]:
            nq, rows, nd = level + 1, level + 1 + P.alpha, P.ndigits(level)
            c = np.stack([np.stack([rng.integers(0, q, P.N, dtype=np.uint64) for q in P.qs(level)])
                          for _ in range(B)])
            d = _dev(c)
            for b in range(B):   # he_ntt maps row r to prime r mod (level+1+alpha): one item per call
                lib.he_ntt(ctx, d[b].data_ptr(), nq, level)
            dig = torch.empty(B * nd * rows * P.N, dtype=torch.int64, device="cuda")
            lib.he_decompose(ctx, d.data_ptr(), B, level, dig.data_ptr())
            dig = dig.view(B, nd, rows, P.N)
            for b in range(B):
                for k in range(nd):
                    lib.he_ntt(ctx, dig[b, k].data_ptr(), rows, level, inverse=True)
            got = _host(dig)
            for b in range(B):
                want = he.modup(c[b], level)
                assert len(want) == nd
                for k in range(nd):
                    assert np.array_equal(got[b, k], want[k]), (level, b, k)
    finally:
        lib.he_ctx_destroy(ctx)


@pytest.mark.parametrize("chain", CHAINS, ids=["n14_alpha1", "n16_alpha2"])
def test_moddown_equals_oracle_and_rounds_at_the_boundary(lib, chain):
    import torch
    ctx, P, he = _setup(lib, chain)
    try:
        rng = np.random.default_rng(22)
        ks = list(range(1, 65))
        uP, Pbig = _boundary_p_residues(P.p, ks)
        for level in LEVELS[P.logN]:
            nq, rows = level + 1, level + 1 + P.alpha
            qp = P.qp(level)
            u = np.stack([np.stack([rng.integers(0, q, P.N, dtype=np.uint64) for q in qp]) for _ in range(B)])
            u[0, nq:, : len(ks)] = uP          # item 0: the boundary cases first
            u[1, nq:, -len(ks):] = uP          # item 1: the same at the last coefficients
            d = _dev(u)
            for b in range(B):
                lib.he_ntt(ctx, d[b].data_ptr(), rows, level)
            out = torch.empty(B * nq * P.N, dtype=torch.int64, device="cuda")
            lib.he_moddown(ctx, d.data_ptr(), B, level, out.data_ptr())
            out = out.view(B, nq, P.N)
            for b in range(B):
                lib.he_ntt(ctx, out[b].data_ptr(), nq, level, inverse=True)
            got = _host(out)
            for b in range(B):
                assert np.array_equal(got[b], he.moddown(u[b], level)), (level, b)
            Qs = P.qs(level)
            for b, cols in ((0, range(len(ks))), (1, range(P.N - len(ks), P.N))):
                for x in cols:
                    X, _ = _crt(u[b, :, x], qp)
                    Y, Q = _crt(got[b, :, x], Qs)
                    assert Y == ((2 * X + Pbig) // (2 * Pbig)) % Q, (level, b, x)
    finally:
        lib.he_ctx_destroy(ctx)


def test_decompose_and_moddown_refuse_bad_arguments(lib):
    import torch
    ctx = lib.he_ctx_create(lib.he_params_default(1), 5)
    try:
        buf = torch.zeros(8 << 14, dtype=torch.int64, device="cuda")
        with pytest.raises(lib.HeError):
            lib.he_moddown(ctx, buf.data_ptr() + 8, 1, 0, buf.data_ptr())      # misaligned
        with pytest.raises(lib.HeError):
            lib.he_decompose(ctx, buf.data_ptr(), 1, 9, buf.data_ptr())        # level above L
        with pytest.raises(lib.HeError):
            lib.he_moddown(ctx, buf.data_ptr(), -1, 0, buf.data_ptr())
        lib.he_moddown(ctx, buf.data_ptr(), 0, 0, buf.data_ptr())              # nothing to do
    finally:
        lib.he_ctx_destroy(ctx)


def test_rotation_with_48_digits_equals_oracle(lib):
    """A key switch whose inner product runs over 48 digits (logN 12, q 60 +
    47 x 40, one 60-bit special prime, top level): on the 60-bit rows the
    sum of 48 digit-key products reaches past q 2^64, the bound of one
    Montgomery reduction, unless the accumulator is kept below it.  The
    rotated ciphertext equals the oracle's word for word."""
    from oracle.ckks import CKKS, Params
    qbits, pbits = [60] + [40] * 47, [60]
    P = Params(12, qbits, pbits)
    ctx = lib.he_ctx_create(lib.make_params(12, qbits, pbits), 7)
    try:
        q, p = lib.he_ctx_primes(ctx)
        assert list(q) == P.q and list(p) == P.p
        he = CKKS(P, 7)
        lib.he_keygen(ctx, [1], want_relin=False)
        he.gen_rotation_key(1)
        z = np.random.default_rng(5).uniform(-1, 1, P.S)
        g = lib.he_encrypt_slots(ctx, z, P.L, 31)
        o = he.encrypt_slots(z, P.L, obj=31)
        assert P.ndigits(P.L) == 48
        gr = lib.he_rotate(ctx, g, 1)
        orr = he.rotate(o, 1)
        assert np.array_equal(lib.he_ct_export(ctx, gr), np.stack([orr.c0, orr.c1]))
        assert np.abs(lib.he_decrypt_slots(ctx, gr, P.S) - np.roll(z, -1)).max() < 1e-4
        for h in (g, gr):
            lib.he_ct_free(h)
    finally:
        lib.he_ctx_destroy(ctx)


def test_multsum_products_are_counted_and_the_product_rate_is_measured(lib):
    """The MultSum trace counts every digit-key product (one rotation at
    config 1's top level: 4 digits x 5 rows x N x 2 polynomials), and the
    product-accumulate microbenchmark runs."""
    ctx = lib.he_ctx_create(lib.he_params_default(1), 5)
    try:
        lib.he_keygen(ctx, [1], want_relin=False)
        z = np.random.default_rng(2).uniform(-1, 1, 1 << 13)
        g = lib.he_encrypt_slots(ctx, z, 3, 9)
        lib.he_ctx_set_autotune(ctx, False)
        lib.he_trace_enable(ctx, True)
        for c in range(5):
            lib.he_trace_read(ctx, c, reset=True)
        r = lib.he_rotate(ctx, g, 1)
        t = lib.he_trace_read(ctx, 0, reset=True)
        lib.he_trace_enable(ctx, False)
        assert t["count"] == 1 and t["ops"] == 4 * 5 * (1 << 14) * 2
        for h in (g, r):
            lib.he_ct_free(h)
    finally:
        lib.he_ctx_destroy(ctx)
    assert lib.he_bench_mac(200) > 1e11
