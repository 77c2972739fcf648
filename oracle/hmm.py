"""Homomorphic linear transforms and JKLS matrix multiplication -- oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

An n x n matrix is packed row-major into slots [0, n^2) (Sec. 3.4).  Matrix
rotations are cyclic modulo n^2; when n^2 < S the ciphertext is first
replicated to period n^2 (reading C5), after which every slot rotation by a
step taken modulo n^2 acts as the cyclic rotation of eq. 4.

Diagonals (Sec. 3.3, eq. 2): u_t[p] = U[p, p + t mod n^2].
  Z (sigma):  eq. 5, indices -n+1 .. n-1
  T (tau):    eq. 6, indices k*n, 0 <= k < n
  C^k (phi^k): indices k and k-n (Sec. 4.1)
  R^k (psi^k): index n*k (Sec. 4.1)
  G (transpose): indices (n-1)*k, -n < k < n (Sec. 3.4)
"""
import numpy as np

from . import _c, dcd
from .ckks import Ct, padd, pmulconst, to_rns


# ------------------------------------------------------------- diagonals

def diag_Z(n, k):
    """eq. 5: z_k[l] = 1 iff (k >= 0 and 0 <= l - n k < n - k) or
    (k < 0 and -k <= l - (n + k) n < n).  Returns an n^2 vector or None."""
    if not (-n < k < n):
        return None
    l = np.arange(n * n)
    if k >= 0:
        m = (l - n * k >= 0) & (l - n * k < n - k)
    else:
        m = (l - (n + k) * n >= -k) & (l - (n + k) * n < n)
    return m.astype(np.float64)


def diag_T(n, t):
    """eq. 6: diagonal t = k n has ones at l in {k + n i}.  t = k*n, 0 <= k < n."""
    if t % n != 0 or not (0 <= t // n < n):
        return None
    k = t // n
    l = np.arange(n * n)
    return ((l % n) == k).astype(np.float64)


def diag_G(n, t, a):
    """Transpose: (G a)[i n + j] = a[j n + i]; the diagonal with index
    (n-1) k holds ones where j - i = k.  t = (n-1) k."""
    k = t // a if a else 0
    if t != a * k or not (-n < k < n):
        return None
    l = np.arange(n * n)
    i, j = l // n, l % n
    return ((j - i) == k).astype(np.float64)


def mask_C(n, k):
    """phi^k = mask1 * rho(.; k) + mask2 * rho(.; k - n):
    mask1 = columns j < n - k, mask2 = columns j >= n - k (Sec. 4.1)."""
    j = np.arange(n * n) % n
    return (j < n - k).astype(np.float64), (j >= n - k).astype(np.float64)


def tile(u, n, S):
    """Replicate an n^2 vector to the S slots (period n^2)."""
    return np.tile(u, S // (n * n))


def rot_slots(u, r):
    """rho(u; r): left rotation by r (Sec. 3.1)."""
    return np.roll(u, -r)


# ---------------------------------------------------- schedule parameters

def dcd_rot_steps(n, n1z, n1t, dcd_z, dcd_t):
    """Matrix rotation steps of Z and T under the Diagonal Convergence
    Decomposition (mod n^2): Z_1's left factor (babies j, giants n1z i for
    0 < i < n2'), Z_2's left factor (giants n1z i, -n2' <= i < 0), the right
    factors +-n'; T's left factor (babies n j, giants n n1t i, 0 < i <= n2'),
    whose last giant is also the right factors' step n' n (Table 2 DCDmp)."""
    n2 = n * n
    z, t = set(), set()
    if dcd_z:
        n2p = dcd_z // n1z
        z |= {j % n2 for j in range(1, n1z)}
        z |= {(n1z * i) % n2 for i in range(-n2p, n2p) if i}
        z |= {dcd_z % n2, (-dcd_z) % n2}
    if dcd_t:
        n2p = dcd_t // n1t
        t |= {(n * j) % n2 for j in range(1, n1t)}
        t |= {(n * n1t * i) % n2 for i in range(1, n2p + 1)}
        t.add((n * dcd_t) % n2)
    z.discard(0)
    t.discard(0)
    return sorted(z), sorted(t)


def matmul_rot_steps(n, n1z, n1t, S, dcd_z=0, dcd_t=0):
    """Rotation steps of the hoisted JKLS schedule (Table 1 'Optimized' rows):
    replication steps -n^2 2^j (mod S), Z babies 1..n1z-1 and giants n1z*i
    (i in [-n2z, n2z) minus 0), T babies n*j and giants n*n1t*i, plus the C^k
    chain step n1z and R^k chain step n*n1t.  Matrix steps are taken mod n^2."""
    n2 = n * n
    steps = set()
    r = n2
    while r < S:
        steps.add((-r) % S)
        r *= 2
    n2z, n2t = n // n1z, n // n1t
    zd, td = dcd_rot_steps(n, n1z, n1t, dcd_z, dcd_t)
    if dcd_z:
        steps |= set(zd)
    else:
        for i in range(-n2z, n2z):
            if i:
                steps.add((n1z * i) % n2)
    for j in range(1, n1z):
        steps.add(j % n2)        # Z babies, also the C^k babies
    if dcd_t:
        steps |= set(td)
    else:
        for i in range(1, n2t):
            steps.add((n * n1t * i) % n2)
    for j in range(1, n1t):
        steps.add((n * j) % n2)  # T babies, also the R^k babies
    steps.add(n1z % n2)          # C^k source chain
    steps.add((-n) % n2)         # C^k second source
    if n2t > 1:
        steps.add((n * n1t) % n2)  # R^k source chain (already a T giant)
    steps.discard(0)
    return sorted(steps)


def ksub_rot_steps(n, kind, n1, n1_sub):
    """Matrix rotation steps (mod n^2) of Z (kind 0) or T (kind 1) under the
    simple key substitution (Sec. 4.2): the babies' head a s, 0 < s < n1_sub,
    and the giants a n1 i (Z: -n2 <= i < n2; T: 0 < i < n2), a = 1 for Z, n
    for T.  Their number is Table 2's MinRotKeys: n1' + 2 n2 - 2 for Z and
    n1' + n2 - 2 for T."""
    n2m, n2 = n * n, n // n1
    a = 1 if kind == 0 else n
    steps = {(a * s) % n2m for s in range(1, n1_sub)}
    giants = range(-n2, n2) if kind == 0 else range(1, n2)
    steps |= {(a * n1 * i) % n2m for i in giants if i}
    steps.discard(0)
    return sorted(steps)


def transpose_rot_steps(n, n1g, S):
    n2 = n * n
    a = n - 1
    steps = set()
    r = n2
    while r < S:
        steps.add((-r) % S)
        r *= 2
    n2g = n // n1g
    for j in range(1, n1g):
        steps.add((a * j) % n2)
    for i in range(-n2g, n2g):
        if i:
            steps.add((a * n1g * i) % n2)
    steps.discard(0)
    return sorted(steps)


# --------------------------------------------------------------- routines

class HMM:
    def __init__(self, ckks):
        self.he = ckks
        self.P = ckks.P

    def replicate(self, ct, n):
        """ct <- ct + Rot(ct, -n^2 2^j), j = 0 .. log2(S/n^2)-1 (reading C5)."""
        he, P = self.he, self.P
        n2 = n * n
        if ct.period == n2:
            return ct
        out = ct
        r = n2
        while r < P.S:
            out = he.add(out, he.rotate(out, (-r) % P.S))
            r *= 2
        out.period = n2
        return out

    def encode_pt_qp(self, u, level):
        """Encode a slot vector at scale q_level, reduced mod every prime of Q_level P."""
        P = self.P
        m = _c.encode(u.astype(np.complex128), P.N, float(P.q[level]))
        return to_rns(m, P.qp(level))

    def lintrans(self, ct, diag, a, n, n1, giants, n1_sub=0):
        """Double-hoisted BSGS (eq. 3', Sec. 3.3, reading C10):
        U m = sum_i rho( sum_j rho(u_{a(n1 i + j)}; -a n1 i) . rho(m; a j) ; a n1 i ).
        Babies rho(m; a j) share one Decompose and stay in Q_l P; each giant
        group is summed in Q_l P, ModDown'd, rotated (kept in Q_l P) and added;
        one final ModDown, then Rescale by q_l (plaintexts at scale q_l).

        n1_sub (simple key substitution, Sec. 4.2): the babies use only the
        keys a s, 0 < s < n1_sub, of the progression's head.  They come in
        groups of n1_sub - 1: group 0 rotates m by a s; every later group
        takes the last baby of the previous one, ModDown'd to a ciphertext
        and Decomposed, as its source c and rotates it by a s, so baby
        j = b + s is rho(c; a s) with c = rho(m; a b) (reading C28)."""
        he, P = self.he, self.P
        n2 = n * n
        lv = ct.level
        qp = P.qp(lv)
        digits = he.modup(ct.c1, lv)
        R = [(he.lift_P(ct.c0, lv), he.lift_P(ct.c1, lv))]
        if n1_sub and n1_sub < n1:
            assert n1_sub >= 2
            src, dg, base = ct, digits, 0
            for j in range(1, n1):
                if j - base == n1_sub:
                    u0, u1 = R[j - 1]
                    src = Ct(*he.moddown2(u0, u1, lv), lv, ct.scale, ct.period)
                    dg, base = he.modup(src.c1, lv), j - 1
                R.append(he.rot_qp(src, dg, (a * (j - base)) % n2))
        else:
            for j in range(1, n1):
                R.append(he.rot_qp(ct, digits, (a * j) % n2))
        acc0 = acc1 = None
        for i in giants:
            pts, idx = [], []
            for j in range(n1):
                u = diag(a * (n1 * i + j))
                if u is None or not u.any():
                    continue
                v = tile(rot_slots(u, (-a * n1 * i) % n2), n, P.S)
                pts.append(self.encode_pt_qp(v, lv))
                idx.append(j)
            if not pts:
                continue
            Pt = np.stack(pts)
            s0 = _c.polymul_sum(qp, Pt, np.stack([R[j][0] for j in idx]))
            s1 = _c.polymul_sum(qp, Pt, np.stack([R[j][1] for j in idx]))
            if i == 0:
                t0, t1 = s0, s1
            else:
                c = Ct(*he.moddown2(s0, s1, lv), lv, ct.scale, ct.period)
                t0, t1 = he.rot_qp(c, he.modup(c.c1, lv), (a * n1 * i) % n2)
            acc0 = t0 if acc0 is None else padd(acc0, t0, qp)
            acc1 = t1 if acc1 is None else padd(acc1, t1, qp)
        out = Ct(*he.moddown2(acc0, acc1, lv), lv, ct.scale, ct.period)
        return he.rescale(out, keep_scale=True)

    def sigma(self, ct, n, n1, n1_sub=0):
        n2 = n // n1
        return self.lintrans(ct, lambda t: diag_Z(n, t), 1, n, n1, range(-n2, n2), n1_sub)

    def tau(self, ct, n, n1, n1_sub=0):
        n2 = n // n1
        return self.lintrans(ct, lambda t: diag_T(n, t), n, n, n1, range(0, n2), n1_sub)

    # --- Diagonal Convergence Decomposition (Sec. 4.2, DMatrixMult) -------
    def _chain(self, ct, chain, n, a_left, n1, giants_left):
        """Applies a factor chain [R_1, ..., R_{m-1}, L]: every right factor
        (diagonals 0 and one step d) as a LinTrans with babies {0, d}; the
        left factor by double-hoisted BSGS.  One level per factor."""
        size = n * n
        for f in chain[:-1]:
            d = [k for k in dcd.diagonal_set(f, size, True) if k != 0]
            ct = self.lintrans(ct, lambda t, f=f: dcd.diagonal(f, size, t), d[0], n, 2, range(0, 1))
        f = chain[-1]
        return self.lintrans(ct, lambda t: dcd.diagonal(f, size, t), a_left, n, n1, giants_left)

    def sigma_dcd(self, ct, n, n1, n_prime):
        """Z = Z_1 + Z_2, each the chain of DCDforZ with maximum diagonal n'
        (n1 | n'); floor((n-1)/n') + 1 levels."""
        n2p = n_prime // n1
        c1, c2 = dcd.dcd_Z(n, n_prime)
        a1 = self._chain(ct, c1, n, 1, n1, range(0, n2p))
        a2 = self._chain(ct, c2, n, 1, n1, range(-n2p, 1))
        return self.he.add(a1, a2)

    def tau_dcd(self, ct, n, n1, n_prime):
        """T as the chain of DCDforT with maximum diagonal n' n (n1 | n');
        floor((n-2)/n') + 1 levels."""
        n2p = n_prime // n1
        return self._chain(ct, dcd.dcd_T(n, n_prime), n, n, n1, range(0, n2p + 1))

    def transpose(self, ct, n, n1, prescale=None):
        """G (Sec. 3.4): BSGS with a = n - 1 over the 2n-1 diagonals.
        `prescale` multiplies every diagonal by a constant (used to fold 1/s
        of the covariance into the transposition)."""
        ct = self.replicate(ct, n)
        n2g = n // n1
        a = n - 1

        def d(t):
            u = diag_G(n, t, a)
            if u is None or prescale is None:
                return u
            return u * prescale
        return self.lintrans(ct, d, a, n, n1, range(-n2g, n2g))

    def hmatmul(self, ctA, ctB, n, n1z, n1t, relin_once=False, dcd_z=0, dcd_t=0):
        """JKLS product (eq. 4) with the hoisting of Sec. 4.1 (DMatrixMult with
        no decomposition, reading C11).  Consumes 3 levels.

        relin_once: instead of DMatrixMult's relinearised Mult per k, sum the
        tensors (d0, d1, d2) of the n products (exact modular sums: decryption
        d0 + d1 s + d2 s^2 is linear) and relinearise the sum once (App. A
        Mult applied to the sum).  Not in the paper; n - 1 fewer key switches.

        dcd_z, dcd_t: when non-zero, Z and T are applied as their Diagonal
        Convergence Decompositions with maximum diagonal n' = dcd_z (resp.
        n' n, n' = dcd_t) (DMatrixMult, Sec. 4.2); the product then consumes
        2 + max(floor((n-1)/dcd_z) + 1, floor((n-2)/dcd_t) + 1) levels."""
        he, P = self.he, self.P
        n2m = n * n
        A = self.replicate(ctA, n)
        B = self.replicate(ctB, n)
        assert A.level == B.level
        A0 = self.sigma_dcd(A, n, n1z, dcd_z) if dcd_z else self.sigma(A, n, n1z)   # level l-1 (or l-m)
        B0 = self.tau_dcd(B, n, n1t, dcd_t) if dcd_t else self.tau(B, n, n1t)
        l1 = min(A0.level, B0.level)
        A0, B0 = he.drop(A0, l1), he.drop(B0, l1)
        qp = P.qp(l1)
        n2z, n2t = n // n1z, n // n1t

        # --- C^k sources: A_g = Rot(A_{g-1}, n1z), A'_g = Rot(A'_{g-1}, n1z), A'_0 = Rot(A0, -n)
        A_src, A_dig, Ap_src, Ap_dig = [], [], [], []
        cur = A0
        curd = he.modup(cur.c1, l1)
        for g in range(n2z):
            if g > 0:
                cur = he.rotate_hoisted(A_src[-1], A_dig[-1], n1z % n2m)
                curd = he.modup(cur.c1, l1)
            A_src.append(cur)
            A_dig.append(curd)
        cur = he.rotate_hoisted(A0, A_dig[0], (-n) % n2m)
        curd = he.modup(cur.c1, l1)
        for g in range(n2z):
            if g > 0:
                cur = he.rotate_hoisted(Ap_src[-1], Ap_dig[-1], n1z % n2m)
                curd = he.modup(cur.c1, l1)
            Ap_src.append(cur)
            Ap_dig.append(curd)

        # --- R^k sources: B_g = Rot(B_{g-1}, n n1t)
        B_src, B_dig = [], []
        cur = B0
        curd = he.modup(cur.c1, l1)
        for g in range(n2t):
            if g > 0:
                cur = he.rotate_hoisted(B_src[-1], B_dig[-1], (n * n1t) % n2m)
                curd = he.modup(cur.c1, l1)
            B_src.append(cur)
            B_dig.append(curd)

        acc = None
        for k in range(n):
            # A^(k) = C^k A0 (level l1 - 1)
            if k == 0:
                Ak = he.drop(A0, l1 - 1)
            else:
                g, b = divmod(k, n1z)
                m1, m2 = mask_C(n, k)
                terms = []
                for src, dig, m in ((A_src[g], A_dig[g], m1), (Ap_src[g], Ap_dig[g], m2)):
                    if b == 0:
                        R = (he.lift_P(src.c0, l1), he.lift_P(src.c1, l1))
                    else:
                        R = he.rot_qp(src, dig, b % n2m)
                    pt = self.encode_pt_qp(tile(m, n, P.S), l1)
                    terms.append((pt, R))
                s0 = _c.polymul_sum(qp, np.stack([t[0] for t in terms]), np.stack([t[1][0] for t in terms]))
                s1 = _c.polymul_sum(qp, np.stack([t[0] for t in terms]), np.stack([t[1][1] for t in terms]))
                c = Ct(*he.moddown2(s0, s1, l1), l1, A0.scale, A0.period)
                Ak = he.rescale(c, keep_scale=True)
            # B^(k) = R^k B0 (level l1, then dropped)
            g, b = divmod(k, n1t)
            if b == 0:
                Bk = B_src[g]
            else:
                Bk = he.rotate_hoisted(B_src[g], B_dig[g], (n * b) % n2m)
            Bk = he.drop(Bk, l1 - 1)
            if relin_once:
                t = he.tensor(Ak, Bk)
                qs = P.qs(Ak.level)
                acc = t if acc is None else tuple(padd(x, y, qs) for x, y in zip(acc, t))
                scale, period = Ak.scale * Bk.scale, min(Ak.period, Bk.period)
            else:
                prod = he.mult_relin(Ak, Bk)
                acc = prod if acc is None else he.add(acc, prod)
        if relin_once:
            acc = he.relin(acc[0], acc[1], acc[2], l1 - 1, scale, period)
        return he.rescale(acc)
