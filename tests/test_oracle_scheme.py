"""Pins of the oracle's CKKS scheme and matrix product against what the
mathematics fixes: decryption within the noise bound, rotation equal to the
slot permutation, Table 1 operation counts, and the decrypted product against
FP64 A.B."""
import numpy as np
import pytest

from oracle.ckks import CKKS, Params, centred
from oracle.hmm import HMM, matmul_rot_steps


@pytest.fixture(scope="module")
def small():
    P = Params(6, [60, 40, 40, 40], [60])
    he = CKKS(P, 101)
    return P, he


def test_encrypt_decrypt_noise(small):
    P, he = small
    z = np.random.default_rng(1).uniform(-1, 1, P.S)
    m = he.encode(z, P.delta, P.qs(P.L))
    ct = he.encrypt_poly(m, P.L, P.delta, 1, P.S)
    # Dec(Enc(m)) - m = v e + e0 + e1 s: bounded by N*19 + 19 + N*19 for ternary v, s
    d = he.decrypt_poly(ct)
    diff = centred(((d[0].astype(object) - m[0].astype(object)) % P.q[0]).astype(np.uint64), P.q[0])
    assert np.abs(diff).max() <= 2 * P.N * 19 + 19
    assert np.abs(diff).max() > 0


def test_rotation_is_slot_permutation_and_keyswitch_noise(small):
    P, he = small
    z = np.random.default_rng(2).uniform(-1, 1, P.S)
    ct = he.encrypt_slots(z, P.L, obj=2)
    for k in [1, 5, P.S - 1]:
        he.gen_rotation_key(k)
        r = he.rotate(ct, k)
        assert np.abs(he.decrypt_slots(r).real - np.roll(z, -k)).max() < 1e-6
    # every level
    for lv in range(P.L + 1):
        r = he.rotate(he.drop(ct, lv), 1)
        assert np.abs(he.decrypt_slots(r).real - np.roll(z, -1)).max() < 1e-6


def test_mult_relin_rescale(small):
    P, he = small
    he.gen_relin_key()
    rng = np.random.default_rng(3)
    x, y = rng.uniform(-1, 1, P.S), rng.uniform(-1, 1, P.S)
    a, b = he.encrypt_slots(x, P.L, obj=3), he.encrypt_slots(y, P.L, obj=4)
    m = he.rescale(he.mult_relin(a, b))
    assert m.level == P.L - 1
    assert abs(m.scale - P.delta ** 2 / P.q[P.L]) < 1e-3
    assert np.abs(he.decrypt_slots(m).real - x * y).max() < 1e-6


def test_refresh_keeps_message(small):
    P, he = small
    z = np.random.default_rng(5).uniform(-1, 1, P.S)
    ct = he.drop(he.encrypt_slots(z, P.L, obj=6), 0)
    r = he.refresh(ct, 77)
    assert r.level == P.L
    assert (he.decrypt_int(r) == he.decrypt_int(ct)).sum() < P.N  # fresh noise differs
    assert np.abs(he.decrypt_slots(r).real - z).max() < 1e-6


def _mm(P, he, n, n1z, n1t, seed, relin_once=False):
    H = HMM(he)
    for s in matmul_rot_steps(n, n1z, n1t, P.S):
        he.gen_rotation_key(s)
    he.gen_relin_key()
    rng = np.random.default_rng(seed)
    A = rng.uniform(-1, 1, (n, n))
    B = rng.uniform(-1, 1, (n, n))
    za = np.zeros(P.S); za[: n * n] = A.ravel()
    zb = np.zeros(P.S); zb[: n * n] = B.ravel()
    ca = he.encrypt_slots(za, P.L, obj=10)
    cb = he.encrypt_slots(zb, P.L, obj=11)
    he.cnt.reset()
    cc = H.hmatmul(ca, cb, n, n1z, n1t, relin_once=relin_once)
    out = he.decrypt_slots(cc).real[: n * n].reshape(n, n)
    return A, B, cc, out


@pytest.mark.parametrize("logN,n,n1z,n1t", [(6, 4, 2, 2), (8, 8, 4, 2), (9, 16, 4, 4)])
def test_hmatmul_decrypts_to_product(logN, n, n1z, n1t):
    P = Params(logN, [60, 40, 40, 40], [60])
    he = CKKS(P, 7)
    A, B, cc, out = _mm(P, he, n, n1z, n1t, seed=logN)
    assert cc.level == P.L - 3
    assert np.abs(out - A @ B).max() < 1e-4
    # replicated output: every copy of the n^2 block holds A.B
    full = he.decrypt_slots(cc).real.reshape(-1, n * n)
    assert np.abs(full - (A @ B).ravel()).max() < 1e-4


def test_hmatmul_operation_counts_table1():
    # Table 1 "Optimized" rows, counted by the oracle for n=16, n1=4 (no
    # replication: n^2 = S).  Table 1 counts the trivial j=0 baby / i=0 giant
    # and the +2 chain steps as operations; the schedule performs:
    #   Z: MS+Pm n1+2n2-2, Dp 2n2, MD 2n2      T: MS n1+n2-2, Dp n2, MD n2
    #   C^k: MS 2(n1-1)n2 + 2n2-1, Dp 2n2, MD (n-1) + 2n2-1
    #   R^k: MS (n1-1)n2 + n2-1, Dp n2, MD n-1 (chain rotations replace the b=0 ones)
    #   Mult: n relinearisations (MS, Dp, MD each n)
    n, n1 = 16, 4
    P = Params(9, [60, 40, 40, 40], [60])
    he = CKKS(P, 8)
    _mm(P, he, n, n1, n1, seed=1)
    n2 = n // n1
    ms = (n1 + 2 * n2 - 2) + (n1 + n2 - 2) + (2 * (n1 - 1) * n2 + 2 * n2 - 1) + ((n1 - 1) * n2 + n2 - 1) + n
    dp = 2 * n2 + n2 + 2 * n2 + n2 + n
    md = 2 * n2 + n2 + (n - 1 + 2 * n2 - 1) + (n - 1) + n
    assert (he.cnt.MS, he.cnt.Dp, he.cnt.MD) == (ms, dp, md)
    # within Table 1's bounds: (n1+2n2)+(n1+n2)+(2n-1)+(n-1)+n MS, ...
    assert he.cnt.MS <= (n1 + 2 * n2) + (n1 + n2) + (2 * n - 1) + (n - 1) + n
    assert he.cnt.Dp <= (2 * n2 + 1) + (n2 + 1) + (2 * n // n1 + 2) + (n // n1 + 1) + n
    assert he.cnt.MD <= (2 * n2 + 1) + (n2 + 1) + (2 * n // n1 + n) + (n - 1) + n


def test_tensor_decrypts_to_product_of_decryptions(small):
    """(d0, d1, d2) of Mult (App. A) satisfies d0 + d1 s + d2 s^2 =
    (a0 + a1 s)(b0 + b1 s) in every limb; the right side is computed from the
    two decryptions with the oracle's negacyclic product (pinned against
    schoolbook convolution)."""
    from oracle import _c
    from oracle.ckks import to_rns
    P, he = small
    rng = np.random.default_rng(5)
    a = he.encrypt_slots(rng.uniform(-1, 1, P.S), 2, obj=30)
    b = he.encrypt_slots(rng.uniform(-1, 1, P.S), 2, obj=31)
    d0, d1, d2 = he.tensor(a, b)
    s = to_rns(he.s_int, P.qs(2))
    for i, q in enumerate(P.qs(2)):
        ma = (a.c0[i].astype(object) + np.array(_c.polymul(q, a.c1[i], s[i]), dtype=object)) % q
        mb = (b.c0[i].astype(object) + np.array(_c.polymul(q, b.c1[i], s[i]), dtype=object)) % q
        want = np.array(_c.polymul(q, ma.astype(np.uint64), mb.astype(np.uint64)), dtype=object)
        s2 = np.array(_c.polymul(q, s[i], s[i]), dtype=np.uint64)
        got = (d0[i].astype(object) + np.array(_c.polymul(q, d1[i], s[i]), dtype=object)
               + np.array(_c.polymul(q, d2[i], s2), dtype=object)) % q
        assert np.array_equal(got, want)


def test_hmatmul_single_relinearisation():
    """relin_once: the product still decrypts to A.B, with n - 1 fewer
    MultSum, Decompose and ModDown than the per-product schedule."""
    n, n1 = 16, 4
    P = Params(9, [60, 40, 40, 40], [60])
    he = CKKS(P, 8)
    A, B, cc, out = _mm(P, he, n, n1, n1, seed=1, relin_once=True)
    assert cc.level == P.L - 3
    assert np.abs(out - A @ B).max() < 1e-4
    got = (he.cnt.MS, he.cnt.Dp, he.cnt.MD)
    he2 = CKKS(P, 8)
    _mm(P, he2, n, n1, n1, seed=1)
    assert got == (he2.cnt.MS - (n - 1), he2.cnt.Dp - (n - 1), he2.cnt.MD - (n - 1))



@pytest.mark.parametrize("n1,n_prime", [(4, 4), (4, 8), (1, 3), (1, 5), (1, 15)])
def test_dcd_sigma_tau_and_product_decrypt(n1, n_prime):
    """Sec. 4.2 DMatrixMult: sigma and tau through their decomposition chains
    decrypt to the index maps of eq. 5 / eq. 6 and consume floor((n-1)/n') + 1
    (Z) and floor((n-2)/n') + 1 (T) levels; the product with both decomposed
    decrypts to A.B -- also for an n' dividing n - 1 (n1 = 1), where a chain
    one factor shorter would leave diagonal n' outside the left factor's
    BSGS range."""
    n = 16
    P = Params(9, [60] + [40] * 9, [60])
    he = CKKS(P, 3)
    from oracle.hmm import HMM, matmul_rot_steps
    for s in matmul_rot_steps(n, n1, n1, P.S, n_prime, n_prime):
        he.gen_rotation_key(s)
    he.gen_relin_key()
    H = HMM(he)
    rng = np.random.default_rng(n_prime)
    A, B = rng.uniform(-1, 1, (n, n)), rng.uniform(-1, 1, (n, n))
    za, zb = np.zeros(P.S), np.zeros(P.S)
    za[: n * n], zb[: n * n] = A.ravel(), B.ravel()
    ca, cb = he.encrypt_slots(za, P.L, obj=10), he.encrypt_slots(zb, P.L, obj=11)
    mz, mt = (n - 1) // n_prime + 1, (n - 2) // n_prime + 1
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    s = H.sigma_dcd(H.replicate(ca, n), n, n1, n_prime)
    t = H.tau_dcd(H.replicate(cb, n), n, n1, n_prime)
    assert (s.level, t.level) == (P.L - mz, P.L - mt)
    assert np.abs(he.decrypt_slots(s).real[: n * n].reshape(n, n) - A[i, (i + j) % n]).max() < 1e-6
    assert np.abs(he.decrypt_slots(t).real[: n * n].reshape(n, n) - B[(i + j) % n, j]).max() < 1e-6
    cc = H.hmatmul(ca, cb, n, n1, n1, dcd_z=n_prime, dcd_t=n_prime)
    assert cc.level == P.L - max(mz, mt) - 2
    assert np.abs(he.decrypt_slots(cc).real[: n * n].reshape(n, n) - A @ B).max() < 1e-4


def test_relin_once_with_decomposed_transforms_decrypts():
    """One relinearisation per product combined with decomposed Z and T
    (both schedule options together) still decrypts to A.B."""
    n, n1, n_prime = 16, 4, 8
    P = Params(9, [60] + [40] * 6, [60])
    he = CKKS(P, 5)
    from oracle.hmm import HMM, matmul_rot_steps
    for s in matmul_rot_steps(n, n1, n1, P.S, n_prime, n_prime):
        he.gen_rotation_key(s)
    he.gen_relin_key()
    rng = np.random.default_rng(21)
    A, B = rng.uniform(-1, 1, (n, n)), rng.uniform(-1, 1, (n, n))
    za, zb = np.zeros(P.S), np.zeros(P.S)
    za[: n * n], zb[: n * n] = A.ravel(), B.ravel()
    ca, cb = he.encrypt_slots(za, P.L, obj=12), he.encrypt_slots(zb, P.L, obj=13)
    he.cnt.reset()
    cc = HMM(he).hmatmul(ca, cb, n, n1, n1, relin_once=True, dcd_z=n_prime, dcd_t=n_prime)
    assert cc.level == P.L - ((n - 1) // n_prime + 1) - 2
    assert np.abs(he.decrypt_slots(cc).real[: n * n].reshape(n, n) - A @ B).max() < 1e-4


@pytest.mark.parametrize("n1,n1_sub", [(8, 2), (8, 3), (8, 5), (4, 3)])
def test_key_substitution_sigma_tau_decrypt_with_fewer_keys(n1, n1_sub):
    """Simple key substitution (Sec. 4.2): sigma and tau with only the keys
    of the babies' head (a s, s < n1') decrypt to the index maps of eq. 5 /
    eq. 6 within 1e-6.  It keeps the dh-BSGS MultSum count and adds one
    Decompose and one ModDown per later group of n1' - 1 babies:
    ceil((n1 - 1)/(n1' - 1)) - 1 of each."""
    n = 16
    P = Params(9, [60] + [40] * 4, [60])
    he = CKKS(P, 4)
    from oracle.hmm import HMM, ksub_rot_steps
    r = n * n
    rep = []
    while r < P.S:
        rep.append((-r) % P.S)
        r *= 2
    for s in sorted(set(ksub_rot_steps(n, 0, n1, n1_sub)) | set(ksub_rot_steps(n, 1, n1, n1_sub)) | set(rep)):
        he.gen_rotation_key(s)
    H = HMM(he)
    rng = np.random.default_rng(n1 * 10 + n1_sub)
    A = rng.uniform(-1, 1, (n, n))
    za = np.zeros(P.S)
    za[: n * n] = A.ravel()
    ca = H.replicate(he.encrypt_slots(za, P.L, obj=14), n)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    extra = -(-(n1 - 1) // (n1_sub - 1)) - 1
    counts = []
    for kind in (0, 1):
        he.cnt.reset()
        out = H.sigma(ca, n, n1, n1_sub) if kind == 0 else H.tau(ca, n, n1, n1_sub)
        got = (he.cnt.MS, he.cnt.Dp, he.cnt.MD)
        want = A[i, (i + j) % n] if kind == 0 else A[(i + j) % n, j]
        assert out.level == P.L - 1
        assert np.abs(he.decrypt_slots(out).real[: n * n].reshape(n, n) - want).max() < 1e-6
        counts.append(got)
    # the same transforms with all baby keys (dh-BSGS)
    for s in range(1, n1):
        he.gen_rotation_key(s % (n * n))
        he.gen_rotation_key((n * s) % (n * n))
    for kind in (0, 1):
        he.cnt.reset()
        _ = H.sigma(ca, n, n1) if kind == 0 else H.tau(ca, n, n1)
        ms, dp, md = counts[kind]
        assert (ms, dp, md) == (he.cnt.MS, he.cnt.Dp + extra, he.cnt.MD + extra)


def test_key_substitution_with_the_whole_head_is_dh_bsgs():
    """n1' = n1 uses every baby key: the transform is the plain double-hoisted
    BSGS, word for word."""
    n, n1 = 16, 4
    P = Params(9, [60] + [40] * 3, [60])
    he = CKKS(P, 6)
    from oracle.hmm import HMM, ksub_rot_steps
    for s in ksub_rot_steps(n, 0, n1, n1):
        he.gen_rotation_key(s)
    z = np.random.default_rng(3).uniform(-1, 1, P.S)
    ca = he.encrypt_slots(z, P.L, obj=15)
    ca.period = n * n
    H = HMM(he)
    a, b = H.sigma(ca, n, n1, n1), H.sigma(ca, n, n1)
    assert np.array_equal(a.c0, b.c0) and np.array_equal(a.c1, b.c1)
