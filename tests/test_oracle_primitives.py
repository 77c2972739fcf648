"""Pins of the oracle's integer and FP64 primitives against definitions that
do not go through the oracle's own code: published known-answer vectors,
Python big-integer arithmetic, schoolbook convolution and sympy."""
import math
import random

import numpy as np
import pytest
import sympy

import oracle._c as c
from oracle.ckks import Params, automorph, centred, to_rns


# ----------------------------------------------------------- Philox4x32-10

def test_philox_known_answers():
    # Known-answer vectors of Philox4x32-10 published with the Random123
    # library (Salmon et al., "Parallel random numbers: as easy as 1, 2, 3",
    # SC'11); see tests/golden/philox4x32_10_kat.txt.
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")
    rows = 0
    for line in open(path):
        line = line.split("#")[0].strip()
        if not line:
            continue
        w = [int(x, 16) for x in line.split()]
        ctr, key, want = w[0:4], w[4:6], w[6:10]
        assert c.philox(ctr, key) == want
        rows += 1
    assert rows == 3


# ------------------------------------------------------------------ primes

@pytest.mark.parametrize("logN,qbits,pbits", [
    (14, [60, 40, 40, 40], [60]),
    (16, [60] + [40] * 20, [60, 60]),
    (15, [60] + [40] * 13, [60, 60]),
])
def test_prime_chain(logN, qbits, pbits):
    q, p = c.gen_primes(logN, qbits, pbits)
    M = 2 << logN
    allp = q + p
    assert len(set(allp)) == len(allp)
    for x, b in zip(allp, qbits + pbits):
        assert sympy.isprime(x)
        assert x % M == 1
        assert abs(math.log2(x) - b) < 1.0
    # q0 and the p's are the largest primes = 1 mod 2N below 2^60, in order
    found = []
    x = ((1 << 60) - 1) // M * M + 1
    while len(found) < 1 + len(p):
        if sympy.isprime(x):
            found.append(x)
        x -= M
    assert [q[0]] + p == found
    # q_1.. alternate: smallest above 2^40, largest below, second above, ...
    ups, downs = [], []
    x = ((1 << 40) + M - 1) // M * M + 1
    while len(ups) < len(q):
        if sympy.isprime(x):
            ups.append(x)
        x += M
    x = ((1 << 40) - 1) // M * M + 1
    while len(downs) < len(q):
        if sympy.isprime(x):
            downs.append(x)
        x -= M
    want = []
    for k in range(len(q) - 1):
        want.append(ups[k // 2] if k % 2 == 0 else downs[k // 2])
    assert q[1:] == want


def test_is_prime_matches_sympy():
    rng = random.Random(5)
    for _ in range(300):
        n = rng.randrange(2, 1 << 62)
        assert c.is_prime(n) == sympy.isprime(n)
    for n in [2, 3, 4, 561, 1105, (1 << 61) - 1, 3215031751, 3825123056546413051]:
        assert c.is_prime(n) == sympy.isprime(n)


# --------------------------------------------------------- ring arithmetic

def _bigint_negacyclic(a, b, q):
    N = len(a)
    out = [0] * N
    for i in range(N):
        for j in range(N):
            k = i + j
            if k < N:
                out[k] += int(a[i]) * int(b[j])
            else:
                out[k - N] -= int(a[i]) * int(b[j])
    return [x % q for x in out]


@pytest.mark.parametrize("N", [2, 8, 64, 256])
def test_polymul_vs_bigint_convolution(N):
    q, _ = c.gen_primes(int(math.log2(N)), [60, 40], [60])
    rng = np.random.default_rng(N)
    for qq in q:
        a = rng.integers(0, qq, N, dtype=np.uint64)
        b = rng.integers(0, qq, N, dtype=np.uint64)
        want = _bigint_negacyclic(a, b, qq)
        assert list(map(int, c.polymul(qq, a, b))) == want
        assert list(map(int, c.polymul_schoolbook(qq, a, b))) == want


def test_polymul_sum_matches_single_products():
    P = Params(8, [60, 40, 40], [60])
    rng = np.random.default_rng(3)
    qs = P.q
    a = np.stack([np.stack([rng.integers(0, q, P.N, dtype=np.uint64) for q in qs]) for _ in range(3)])
    b = np.stack([np.stack([rng.integers(0, q, P.N, dtype=np.uint64) for q in qs]) for _ in range(3)])
    got = c.polymul_sum(qs, a, b)
    for l, q in enumerate(qs):
        acc = [0] * P.N
        for t in range(3):
            pr = _bigint_negacyclic(a[t, l], b[t, l], q)
            acc = [(x + y) % q for x, y in zip(acc, pr)]
        assert list(map(int, got[l])) == acc


def test_automorphism_is_substitution():
    # kappa_g(a)(X) = a(X^g) in Z_q[X]/(X^N+1), checked by evaluating the
    # substitution with big integers.
    N, q = 16, 97
    rng = np.random.default_rng(1)
    a = rng.integers(0, q, (1, N), dtype=np.uint64)
    for g in [3, 5, 25, 2 * N - 1]:
        got = automorph(a, g, N, [q])[0]
        want = [0] * N
        for i in range(N):
            e = (i * g) % (2 * N)
            if e < N:
                want[e] = (want[e] + int(a[0, i])) % q
            else:
                want[e - N] = (want[e - N] - int(a[0, i])) % q
        assert list(map(int, got)) == want


# ------------------------------------------------- basis conversion, rescale

def _crt(res, qs):
    Q = 1
    for q in qs:
        Q *= q
    x = 0
    for r, q in zip(res, qs):
        Qi = Q // q
        x += int(r) * Qi * pow(Qi, -1, q)
    return x % Q, Q


def test_fast_bconv_exact_relation():
    # Decompose / ModUp (Sec. 3.3): BConv(x) = x + u*Q_s with 0 <= u < #source primes.
    P = Params(6, [60, 40, 40, 40], [60, 60])
    rng = np.random.default_rng(7)
    src_q = P.q[1:3]
    dst_q = [P.q[0], P.q[3]] + P.p
    src = np.stack([rng.integers(0, q, P.N, dtype=np.uint64) for q in src_q])
    out = c.bconv(src_q, src, dst_q)
    for x in range(P.N):
        X, Q = _crt(src[:, x], src_q)
        us = set()
        for r, qq in enumerate(dst_q):
            v = int(out[r, x])
            # find u with (X + u Q) mod qq == v and 0 <= u < 2
            cands = [u for u in range(len(src_q)) if (X + u * Q) % qq == v]
            assert cands, "no admissible u"
            us.add(cands[0])
        assert len(us) == 1  # the same u for every target prime


@pytest.mark.parametrize("pbits", [[60], [60, 60], [60, 50, 45]])
def test_moddown_is_rounding(pbits):
    # ModDown (App. A KeySwitch): round(X / P) mod Q_l, exactly, for X the
    # CRT value over Q_l P (P odd: no ties).
    from oracle.ckks import CKKS
    P = Params(8, [60, 40, 40], pbits)
    he = CKKS(P, 9)
    rng = np.random.default_rng(8)
    lv = 2
    qp = P.qp(lv)
    u = np.stack([rng.integers(0, q, P.N, dtype=np.uint64) for q in qp])
    out = he.moddown(u, lv)
    Qs = P.qs(lv)
    for x in range(P.N):
        X, QP = _crt(u[:, x], qp)
        Y, Q = _crt(out[:, x], Qs)
        assert Y == ((2 * X + P.P) // (2 * P.P)) % Q


def overflow_boundary_residues(ps, ks):
    """P-residues uP of coefficients whose fast-conversion sum
    S = sum_j y_j (P/p_j) is congruent to -k mod P (k in ks): S sits k units
    below a multiple of P, so sum_j y_j / p_j lies within k/P of an integer.
    y_j = -k (P/p_j)^-1 mod p_j; v_j = y_j (P/p_j); uP_j = v_j - (P-1)/2."""
    P = 1
    for p in ps:
        P *= p
    h = (P - 1) // 2
    uP = np.zeros((len(ps), len(ks)), dtype=np.uint64)
    ys = []
    for c, k in enumerate(ks):
        yc = []
        for j, p in enumerate(ps):
            ph = P // p
            y = (-k * pow(ph, -1, p)) % p
            yc.append(y)
            uP[j, c] = ((y * ph) - h) % p
        ys.append(yc)
    return uP, ys, P


@pytest.mark.parametrize("pbits", [[60], [60, 60], [60, 50, 45], [60, 60, 60, 60]])
def test_moddown_rounds_at_the_overflow_boundary(pbits):
    # App. A KeySwitch rounds P^-1 x exactly.  Where sum_j y_j / p_j is just
    # below an integer, its FP64 evaluation rounds up to that integer and
    # would subtract P once too often; ModDown must still be round(X / P).
    from oracle.ckks import CKKS
    P = Params(8, [60, 40, 40], pbits)
    he = CKKS(P, 9)
    lv = 2
    qp = P.qp(lv)
    ks = list(range(1, 65))
    uP, ys, Pbig = overflow_boundary_residues(P.p, ks)
    rng = np.random.default_rng(3)
    u = np.stack([rng.integers(0, q, P.N, dtype=np.uint64) for q in qp])
    u[lv + 1:, : len(ks)] = uP
    out = he.moddown(u, lv)
    Qs = P.qs(lv)
    fp64_wrong = 0
    for c in range(len(ks)):
        X, _ = _crt(u[:, c], qp)
        Y, Q = _crt(out[:, c], Qs)
        assert Y == ((2 * X + Pbig) // (2 * Pbig)) % Q, c
        exact = sum(y * (Pbig // p) for y, p in zip(ys[c], P.p)) // Pbig
        est = 0.0
        for y, p in zip(ys[c], P.p):
            est = est + float(y) / float(p)
        fp64_wrong += int(np.floor(est)) != exact
    # the cases do reach past what an FP64 overflow estimate resolves
    assert fp64_wrong > 0


def test_keyswitch_noise_is_centred():
    # The rounding ModDown leaves no systematic offset in the key-switch
    # noise: Dec(Rot(ct)) - kappa(Dec(ct)) has mean ~0 (a floor-type ModDown
    # gives a mean near -alpha * (sum of s) / 2, which decodes to large slot
    # errors next to slot 0).
    from oracle.ckks import CKKS, psub
    P = Params(12, [60] + [40] * 6, [60, 60])
    he = CKKS(P, 5)
    z = np.random.default_rng(1).uniform(-1, 1, P.S)
    ct = he.encrypt_slots(z, P.L, obj=1)
    he.gen_rotation_key(1)
    r = he.rotate(ct, 1)
    want = automorph(he.decrypt_poly(ct), P.galois(1), P.N, P.qs(P.L))
    noise = centred(psub(he.decrypt_poly(r), want, P.qs(P.L))[0], P.q[0])
    assert abs(noise.mean()) < 3 * noise.std() / np.sqrt(P.N) + 0.5
    assert noise.std() < 100


def test_rescale_is_rounding():
    # Rescale (App. A): round(X / q_l) mod Q_(l-1), exactly (q_l odd: no ties).
    from oracle.ckks import CKKS
    P = Params(6, [60, 40, 40, 40], [60])
    he = CKKS(P, 9)
    rng = np.random.default_rng(9)
    lv = 3
    qs = P.qs(lv)
    a = np.stack([rng.integers(0, q, P.N, dtype=np.uint64) for q in qs])
    out = he.rescale_poly(a, lv)
    ql = qs[-1]
    for x in range(P.N):
        X, Q = _crt(a[:, x], qs)
        want = (2 * X + ql) // (2 * ql)          # round half up; no ties occur
        Y, Q1 = _crt(out[:, x], qs[:-1])
        assert Y == want % Q1


def test_centred_residue():
    q = 97
    x = np.arange(q, dtype=np.uint64)
    r = centred(x, q)
    assert r.min() == -48 and r.max() == 48
    assert all((int(a) - int(b)) % q == 0 for a, b in zip(x, r))


# --------------------------------------------------------------- sampling

def test_gauss_table_and_samples():
    T = c.gauss_table(3.2)
    assert int(T[-1]) == 1 << 63
    assert all(int(T[k]) < int(T[k + 1]) for k in range(19))
    # P(x = 0) = rho(0) / sum rho, rho(v) = exp(-v^2 / (2 sigma^2))
    rho = [math.exp(-v * v / (2 * 3.2 * 3.2)) for v in range(20)]
    tot = rho[0] + 2 * sum(rho[1:])
    assert abs(int(T[0]) / 2 ** 63 - rho[0] / tot) < 1e-12
    s = c.sample_gauss(42, 1, 3, 3.2, 1 << 16)
    assert abs(s.mean()) < 0.05
    assert abs(s.std() - 3.2) < 0.05
    assert np.abs(s).max() <= 19


def test_ternary_and_uniform():
    t = c.sample_ternary(42, 1, 1, 1 << 15)
    for v in (-1, 0, 1):
        assert abs((t == v).mean() - 1 / 3) < 0.01
    q = 1099511922689
    u = c.sample_uniform(42, 1, 2, 0, q, 1 << 15)
    assert u.max() < q
    assert abs(u.astype(np.float64).mean() / q - 0.5) < 0.01
    # sample j of the uniform stream is Philox block (j, limb, obj, tag) mod q
    w = c.philox([5, 0, 1, 2], [42, 0])
    assert int(u[5]) == ((w[3] << 96) | (w[2] << 64) | (w[1] << 32) | w[0]) % q


# --------------------------------------------------------- encode / decode

@pytest.mark.parametrize("logN", [3, 6, 10])
def test_encode_matches_direct_sum(logN):
    N = 1 << logN
    rng = np.random.default_rng(logN)
    z = rng.uniform(-1, 1, N // 2) + 1j * rng.uniform(-1, 1, N // 2)
    scale = 2.0 ** 30
    m = c.encode(z, N, scale)
    md = c.encode_direct(z, N, scale)
    assert np.abs(m - md).max() <= 0.5 + 1e-3
    back = c.decode(m.astype(np.float64), scale)
    assert np.abs(back - z).max() < 1e-6


def test_encode_constant_is_constant_polynomial():
    N = 1 << 10
    m = c.encode(np.full(N // 2, 0.75), N, 2.0 ** 40)
    assert m[0] == round(0.75 * 2 ** 40)
    assert not m[1:].any()


def test_slot_rotation_is_automorphism_by_5():
    # App. A Rotation: X -> X^(5^k) rotates the slots left by k.
    N = 1 << 8
    q = 1152921504606846883
    rng = np.random.default_rng(4)
    z = rng.uniform(-1, 1, N // 2)
    m = c.encode(z, N, 2.0 ** 40)
    for k in [1, 3, N // 2 - 1]:
        g = pow(5, k, 2 * N)
        mr = centred(automorph(to_rns(m, [q]), g, N, [q])[0], q).astype(np.float64)
        zr = c.decode(mr, 2.0 ** 40)
        assert np.abs(zr.real - np.roll(z, -k)).max() < 1e-9
