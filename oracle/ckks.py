"""Full-RNS CKKS in coefficient form (App. A) -- the oracle's scheme layer.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Polynomials are numpy uint64 arrays [limbs][N] in coefficient form with every
residue in [0, q).  A ciphertext at level l has limbs q_0..q_l.  Extended
polynomials (Decompose output, hoisted products) have limbs q_0..q_l followed
by the special primes p_0..p_{alpha-1}.

Readings of points the paper leaves open (they bind the GPU path too):
  * Philox counter = (coefficient i, limb j, object id, purpose tag), key =
    (seed lo, seed hi); object = Galois element for rotation keys, 0 for the
    relinearisation key and the public key, the caller's counter for
    encryptions.
  * Hybrid key switching with digits of alpha consecutive q's; the switching
    key is (-a_d s + e_d + P B_d s', a_d) over Q_L P (App. A SwitchKeyGen).
  * Decompose extends every digit with the fast basis conversion; ModDown is
    the rounding round(u / P) of App. A KeySwitch, computed exactly (the
    overflow of the basis conversion is removed with an FP64 estimate).
  * Hoisting: Decompose first, then the automorphism on the extended digits
    (Sec. 3.3 hoisting order).
  * Rescale = round(c / q_l) via the centred residue of the last limb.
"""
import math

import numpy as np

from . import _c

TAG_SK, TAG_PK_A, TAG_PK_E = 1, 2, 3
TAG_ENC_V, TAG_ENC_E0, TAG_ENC_E1 = 4, 5, 6
TAG_REF_V, TAG_REF_E0, TAG_REF_E1 = 7, 8, 9
TAG_SWK_A, TAG_SWK_E = 0x100, 0x200


class Counters:
    """Counts of the four internal steps of a rotation (Table 1 caption):
    MultSum (MS), Permute (Pm), Decompose (Dp), ModDown (MD)."""

    def __init__(self):
        self.reset()

    def reset(self):
        self.MS = self.Pm = self.Dp = self.MD = 0
        self.keys = set()


class Params:
    """Setparams (App. A): ring degree N = 2^logN, q's and p's = 1 mod 2N."""

    def __init__(self, logN, qbits, pbits, log_delta=40, sigma=3.2):
        self.logN = logN
        self.N = 1 << logN
        self.S = self.N // 2
        self.M = 2 * self.N
        self.q, self.p = _c.gen_primes(logN, list(qbits), list(pbits))
        self.L = len(self.q) - 1
        self.alpha = len(self.p)
        self.dnum = -(-(self.L + 1) // self.alpha)
        self.delta = float(2.0 ** log_delta)
        self.sigma = float(sigma)
        self.P = 1
        for p in self.p:
            self.P *= p

    def qs(self, level):
        return self.q[: level + 1]

    def qp(self, level):
        return self.q[: level + 1] + self.p

    def digit(self, d, level):
        """Indices of the q's of digit d that exist at this level."""
        return [i for i in range(self.alpha * d, min(self.alpha * d + self.alpha, level + 1))]

    def ndigits(self, level):
        return -(-(level + 1) // self.alpha)

    def galois(self, step):
        """Galois element 5^step mod 2N of the slot rotation by `step` (App. A Rotation)."""
        return pow(5, step % self.S, self.M)


# ------------------------------------------------------------ limb helpers

def _qa(qs):
    return np.array(qs, dtype=np.uint64)[:, None]


def to_rns(x, qs):
    """Signed integers (int64 array or list of Python ints) -> [len(qs)][N]."""
    x = np.asarray(x)
    if x.dtype == object:
        return np.array([[int(v) % q for v in x] for q in qs], dtype=np.uint64)
    x = x.astype(np.int64)
    return np.stack([np.mod(x, np.int64(q)).astype(np.uint64) for q in qs])


def padd(a, b, qs):
    return (a + b) % _qa(qs)


def psub(a, b, qs):
    return (a + (_qa(qs) - b)) % _qa(qs)


def pneg(a, qs):
    return (_qa(qs) - a) % _qa(qs)


def pmul(a, b, qs):
    return _c.polymul_sum(qs, a[None], b[None])


def pmulconst(a, cs, qs):
    return _c.mulconst_limbs(qs, a, cs)


def automorph(a, g, N, qs):
    """kappa_g: X -> X^g on every limb (coefficient form, App. A Rotation):
    coefficient i moves to i*g mod 2N; landing at or past N wraps with a sign."""
    M = 2 * N
    idx = (np.arange(N, dtype=np.int64) * g) % M
    neg = idx >= N
    dst = np.where(neg, idx - N, idx)
    out = np.zeros_like(a)
    out[:, dst] = a
    q = _qa(qs)
    sel = out[:, dst[neg]]
    out[:, dst[neg]] = (q - sel) % q
    return out


def centred(x, q):
    """[x]_q in (-q/2, q/2] (Sec. 3.1 notation), as int64."""
    x = x.astype(np.uint64)
    half = np.uint64(q // 2)
    return np.where(x > half, x.astype(np.int64) - np.int64(q), x.astype(np.int64))


# ----------------------------------------------------------------- objects

class Ct:
    def __init__(self, c0, c1, level, scale, period):
        self.c0, self.c1, self.level, self.scale, self.period = c0, c1, level, scale, period

    def copy(self):
        return Ct(self.c0.copy(), self.c1.copy(), self.level, self.scale, self.period)


class CKKS:
    """Key material and evaluation routines of full-RNS CKKS (App. A)."""

    def __init__(self, params, seed):
        self.P = params
        self.seed = int(seed)
        self.cnt = Counters()
        self.rtk = {}
        self.rlk = None
        N = params.N
        # SecKeyGen: s <- chi_s (ternary)
        self.s_int = _c.sample_ternary(self.seed, 0, TAG_SK, N)
        allq = params.q + params.p
        self.s_all = to_rns(self.s_int, allq)              # over Q_L P
        # PubKeyGen: (-a s + e, a) over Q_L
        qL = params.q
        a = np.stack([_c.sample_uniform(self.seed, 0, TAG_PK_A, j, q, N) for j, q in enumerate(qL)])
        e = to_rns(_c.sample_gauss(self.seed, 0, TAG_PK_E, params.sigma, N), qL)
        s_q = self.s_all[: params.L + 1]
        self.pk0 = padd(pneg(pmul(a, s_q, qL), qL), e, qL)
        self.pk1 = a

    # --- switching keys (App. A SwitchKeyGen, reading C7) ---------------
    def _swk(self, sprime_all, obj):
        P = self.P
        N = P.N
        allq = P.q + P.p
        L = P.L
        key = []
        for d in range(P.dnum):
            a = np.stack([_c.sample_uniform(self.seed, obj, TAG_SWK_A + d, j, q, N)
                          for j, q in enumerate(allq)])
            e = to_rns(_c.sample_gauss(self.seed, obj, TAG_SWK_E + d, P.sigma, N), allq)
            k0 = padd(pneg(pmul(a, self.s_all, allq), allq), e, allq)
            # + P * B_d * s' : nonzero only on the q's of digit d, where it is (P mod q_i) s'
            for i in P.digit(d, L):
                qi = allq[i]
                t = _c.mulconst_limbs([qi], sprime_all[i:i + 1], [P.P % qi])
                k0[i] = (k0[i] + t[0]) % np.uint64(qi)
            key.append((k0, a))
        return key

    def gen_rotation_key(self, step):
        P = self.P
        g = P.galois(step)
        if g in self.rtk:
            return
        allq = P.q + P.p
        sp = automorph(self.s_all, g, P.N, allq)         # s' = kappa_g(s)
        self.rtk[g] = self._swk(sp, g)

    def gen_relin_key(self):
        P = self.P
        allq = P.q + P.p
        s2 = pmul(self.s_all, self.s_all, allq)            # s' = s^2
        self.rlk = self._swk(s2, 0)

    # --- encode / encrypt / decrypt --------------------------------------
    def encode(self, z, scale, qs):
        m = _c.encode(z, self.P.N, scale)
        return to_rns(m, qs)

    def encrypt_poly(self, m_rns, level, scale, obj, period, tags=(TAG_ENC_V, TAG_ENC_E0, TAG_ENC_E1)):
        """Enc (App. A): (v pk0 + m + e0, v pk1 + e1) over Q_level."""
        P = self.P
        qs = P.qs(level)
        N = P.N
        v = to_rns(_c.sample_ternary(self.seed, obj, tags[0], N), qs)
        e0 = to_rns(_c.sample_gauss(self.seed, obj, tags[1], P.sigma, N), qs)
        e1 = to_rns(_c.sample_gauss(self.seed, obj, tags[2], P.sigma, N), qs)
        c0 = padd(padd(pmul(v, self.pk0[: level + 1], qs), m_rns, qs), e0, qs)
        c1 = padd(pmul(v, self.pk1[: level + 1], qs), e1, qs)
        return Ct(c0, c1, level, scale, period)

    def encrypt_slots(self, z, level, obj, scale=None, period=None):
        scale = self.P.delta if scale is None else scale
        m = self.encode(z, scale, self.P.qs(level))
        return self.encrypt_poly(m, level, scale, obj, self.P.S if period is None else period)

    def decrypt_poly(self, ct):
        """Dec (App. A): c0 + c1 s over Q_level (coefficient form)."""
        qs = self.P.qs(ct.level)
        return padd(ct.c0, pmul(ct.c1, self.s_all[: ct.level + 1], qs), qs)

    def decrypt_int(self, ct):
        """Message integers: decrypt after dropping to q_0, lifted to (-q0/2, q0/2]."""
        m0 = padd(ct.c0[:1], pmul(ct.c1[:1], self.s_all[:1], self.P.q[:1]), self.P.q[:1])[0]
        return centred(m0, self.P.q[0])

    def decrypt_slots(self, ct):
        m = self.decrypt_int(ct).astype(np.float64)
        return _c.decode(m, ct.scale)

    # --- arithmetic (App. A Addition / Multiplication modules) -----------
    def add(self, a, b):
        assert a.level == b.level
        qs = self.P.qs(a.level)
        return Ct(padd(a.c0, b.c0, qs), padd(a.c1, b.c1, qs), a.level, a.scale, min(a.period, b.period))

    def sub(self, a, b):
        assert a.level == b.level
        qs = self.P.qs(a.level)
        return Ct(psub(a.c0, b.c0, qs), psub(a.c1, b.c1, qs), a.level, a.scale, min(a.period, b.period))

    def drop(self, ct, level):
        """Level dropping: keep limbs q_0..q_level."""
        assert level <= ct.level
        return Ct(ct.c0[: level + 1].copy(), ct.c1[: level + 1].copy(), level, ct.scale, ct.period)

    def rescale_poly(self, a, level):
        """round(a / q_level) over Q_(level-1) (App. A Rescaling, reading C6)."""
        qs = self.P.qs(level)
        ql = qs[-1]
        r = centred(a[level], ql)                       # Python ints, |r| <= q/2
        rr = to_rns(r, qs[:-1])
        diff = psub(a[:level], rr, qs[:-1])
        inv = [_c.invmod(ql % q, q) for q in qs[:-1]]
        return pmulconst(diff, inv, qs[:-1])

    def rescale(self, ct, keep_scale=False):
        lv = ct.level
        ql = self.P.q[lv]
        c0 = self.rescale_poly(ct.c0, lv)
        c1 = self.rescale_poly(ct.c1, lv)
        scale = ct.scale if keep_scale else ct.scale / float(ql)
        return Ct(c0, c1, lv - 1, scale, ct.period)

    def pmult_pt(self, ct, pt_rns, pt_scale):
        qs = self.P.qs(ct.level)
        return Ct(pmul(ct.c0, pt_rns, qs), pmul(ct.c1, pt_rns, qs), ct.level,
                  ct.scale * pt_scale, ct.period)

    # --- key switching (App. A KeySwitch; Sec. 3.3 Decompose / ModDown) ---
    def modup(self, c, level):
        """Decompose: the digits of c over Q_level, each extended to Q_level P."""
        P = self.P
        self.cnt.Dp += 1
        dst = P.qp(level)
        out = []
        for d in range(P.ndigits(level)):
            idx = P.digit(d, level)
            ext = _c.bconv([P.q[i] for i in idx], c[idx], dst)
            for i in idx:
                ext[i] = c[i]
            out.append(ext)
        return out

    def moddown2(self, u0, u1, level):
        """ModDown of a ciphertext pair (one MD in the Table 1 counts)."""
        self.cnt.MD += 1
        return self.moddown(u0, level), self.moddown(u1, level)

    def moddown(self, u, level):
        """ModDown: round(u / P) over Q_level (App. A KeySwitch, the rounding
        of the inner product by P^-1), computed exactly as floor((u + (P-1)/2) / P)."""
        P = self.P
        return _c.moddown_round(P.qs(level), u[: level + 1], P.p, u[level + 1:])

    def _key_at(self, key, level):
        """Restrict a switching key to the digits and limbs of Q_level P."""
        P = self.P
        rows = list(range(level + 1)) + list(range(P.L + 1, P.L + 1 + P.alpha))
        nd = P.ndigits(level)
        k0 = np.stack([key[d][0][rows] for d in range(nd)])
        k1 = np.stack([key[d][1][rows] for d in range(nd)])
        return k0, k1

    def multsum(self, digits, key, level):
        """MultSum: <digits, swk> over Q_level P -> (u0, u1)."""
        self.cnt.MS += 1
        qp = self.P.qp(level)
        k0, k1 = self._key_at(key, level)
        D = np.stack(digits)
        return _c.polymul_sum(qp, D, k0), _c.polymul_sum(qp, D, k1)

    def rot_qp(self, ct, digits, step):
        """Hoisted rotation kept in Q_l P: (P kappa(c0) + IP0, IP1) with
        IP = <kappa(digits), rtk> (Sec. 3.3, hoisting; double hoisting keeps it in QP)."""
        P = self.P
        g = P.galois(step)
        if g not in self.rtk:
            raise KeyError("rotation key for step %d missing" % step)
        self.cnt.keys.add(g)
        qp = P.qp(ct.level)
        self.cnt.Pm += 1
        pd = [automorph(dg, g, P.N, qp) for dg in digits]
        u0, u1 = self.multsum(pd, self.rtk[g], ct.level)
        c0g = automorph(ct.c0, g, P.N, P.qs(ct.level))
        pc0 = self.lift_P(c0g, ct.level)
        return padd(u0, pc0, qp), u1

    def lift_P(self, a, level):
        """P * a as an element of Q_level P (zero on the p limbs)."""
        P = self.P
        qs = P.qs(level)
        t = pmulconst(a, [P.P % q for q in qs], qs)
        return np.concatenate([t, np.zeros((P.alpha, P.N), dtype=np.uint64)])

    def rotate_hoisted(self, ct, digits, step):
        """Rot (App. A) reusing precomputed Decompose output: kappa(c0) + ModDown(IP0), ModDown(IP1)."""
        P = self.P
        g = P.galois(step)
        if g not in self.rtk:
            raise KeyError("rotation key for step %d missing" % step)
        self.cnt.keys.add(g)
        qp = P.qp(ct.level)
        qs = P.qs(ct.level)
        self.cnt.Pm += 1
        pd = [automorph(dg, g, P.N, qp) for dg in digits]
        u0, u1 = self.multsum(pd, self.rtk[g], ct.level)
        c0g = automorph(ct.c0, g, P.N, qs)
        m0, m1 = self.moddown2(u0, u1, ct.level)
        return Ct(padd(c0g, m0, qs), m1, ct.level, ct.scale, ct.period)

    def rotate(self, ct, step):
        return self.rotate_hoisted(ct, self.modup(ct.c1, ct.level), step)

    def tensor(self, a, b):
        """The tensor of Mult (App. A): (d0, d1, d2) = (a0 b0, a0 b1 + a1 b0, a1 b1),
        decrypting as d0 + d1 s + d2 s^2 = (a0 + a1 s)(b0 + b1 s)."""
        assert a.level == b.level
        qs = self.P.qs(a.level)
        d0 = pmul(a.c0, b.c0, qs)
        d1 = _c.polymul_sum(qs, np.stack([a.c0, a.c1]), np.stack([b.c1, b.c0]))
        d2 = pmul(a.c1, b.c1, qs)
        return d0, d1, d2

    def relin(self, d0, d1, d2, lv, scale, period):
        """(d0, d1) + KeySwitch(d2, rlk) (App. A Mult)."""
        qs = self.P.qs(lv)
        digits = self.modup(d2, lv)
        u0, u1 = self.multsum(digits, self.rlk, lv)
        m0, m1 = self.moddown2(u0, u1, lv)
        return Ct(padd(d0, m0, qs), padd(d1, m1, qs), lv, scale, period)

    def mult_relin(self, a, b):
        """Mult (App. A): tensor (d0, d1, d2), then (d0, d1) + KeySwitch(d2, rlk).
        Scale = scale_a * scale_b; the caller rescales."""
        d0, d1, d2 = self.tensor(a, b)
        return self.relin(d0, d1, d2, a.level, a.scale * b.scale, min(a.period, b.period))

    def refresh(self, ct, obj):
        """Interactive modulus refresh (Sec. 7.2, App. C): decrypt to the
        integer message at q_0, re-encrypt the same integers at level L."""
        m = self.decrypt_int(ct)
        P = self.P
        return self.encrypt_poly(to_rns(m, P.qs(P.L)), P.L, ct.scale, obj, ct.period,
                                 tags=(TAG_REF_V, TAG_REF_E0, TAG_REF_E1))

    # --- export ------------------------------------------------------------
    @staticmethod
    def residues(ct):
        return np.stack([ct.c0, ct.c1])
