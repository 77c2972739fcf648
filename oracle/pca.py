"""Covariance and PowerMethod circuits (Sec. 5, Sec. 6) -- oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Block convention: X_j[l] is the l-th row block of the j-th feature block of
the dataset (Sec. 5.1); C[a][b] is block row a, block column b of a t x t
matrix.  The paper's Cov_i[j] (the j-th submatrix of the i-th column block)
is C[j][i].  A vector segment v_b is represented either row-replicated
(axis 0: every row of the n x n block equals v_b) or column-replicated
(axis 1: every column equals v_b), Sec. 6.1.1.

Readings (beyond those of ckks.py / hmm.py):
  * constants are encoded as the constant polynomial round(c * q_l) and
    multiplied followed by a rescale by q_l (the scale is kept);
  * HCovMtrx: blocks a <= b (diagonal included) by matrix products, a > b by
    transposing block (b, a); the mean of block j is (1/s) Aggregate_0 of the
    summed row blocks; 1/s of X^T X is folded into the transposition's
    diagonals; mu[j]^T = G(mu[j]); Cov = X^T X - mu^T mu;
  * the Newton step is y <- (3y - x y^3)/2 (Newton's Method algorithm; the
    IterativInvSRTbyNewton listing has the sign of both terms flipped), in
    three levels: t1 = y y, t2 = y x, t3 = t1 t2, then (3y - t3) * 1/2;
  * with compose_newton, pairs of Newton steps run as one composite step of
    five levels instead of six (Sec. 7 composites two InvSRT iterations into
    one and saves a level; the circuit is not printed): with u = x y^2,
    y1/2 = (y/4)(3 - u), x y1^2 = (u/4)(3 - u)^2, y2 = (y1/2)(3 - x y1^2);
    the constant 1/4 of u carries the scale that puts y2 at Delta; an odd
    count ends with one single step;
  * HPowerMethod's j-loop multiplies by V_t[j] (the listing writes V_t[i]),
    and its "if n < l_P" reads "if t < l_P";
  * a ciphertext is refreshed (decrypted to the integer message at q_0 and
    re-encrypted at level L) just before an operation that needs more levels
    than it has (App. C); a ciphertext that several products take (a vector
    segment in a covariance transformation, the eigenvector segments and the
    eigenvalue in EigenShift) is refreshed once, before the first of them.
"""
import math

import numpy as np

from . import _c
from .ckks import Ct, padd, psub, to_rns
from .hmm import HMM, tile


# ------------------------------------------------- Lazy Normalization (Sec. 6.1.2)

def taylor_inv_sqrt(x, x0):
    """Order-1 Taylor expansion of 1/sqrt(x) at x0 (TaylorInit)."""
    return x0 ** -0.5 * (1.5 - x / (2.0 * x0))


def newton_inv_sqrt(x, y, iters):
    """Newton's Method for 1/sqrt(x): y <- y (3 - x y^2) / 2."""
    for _ in range(iters):
        y = 0.5 * y * (3.0 - x * y * y)
    return y


def lazy_normalization_schedule(t, S=0.5, e=1e-5, Bp=1e-3, B2=2.0 ** 16, max_iters=64):
    """PowerMethod simulation of Lazy Normalization (Sec. 6.1.2): start from
    length l = 1; per PowerMethod iteration l <- l S, then the smallest Newton
    count whose output S' keeps (l S' S)^2 >= B' and, at the last iteration,
    |1 - l S'| < e; l <- l S'.  Taylor at B^2/2 + 1 over (0, B^2]."""
    x0 = B2 / 2.0 + 1.0
    l, counts = 1.0, []
    for p in range(t):
        l = l * S
        last = p == t - 1
        for tau in range(max_iters + 1):
            Sp = newton_inv_sqrt(l * l, taylor_inv_sqrt(l * l, x0), tau)
            if (l * Sp * S) ** 2 >= Bp and (not last or abs(1.0 - l * Sp) < e):
                break
        counts.append(tau)
        l = l * Sp
    return counts


# ------------------------------------------------------------------ circuits

class PCA:
    def __init__(self, ckks, compose_newton=False, pack_refresh=False):
        self.he = ckks
        self.P = ckks.P
        self.H = HMM(ckks)
        self.refreshes = 0
        self.refresh_obj = 1 << 20
        self.compose_newton = compose_newton
        self.pack_refresh = pack_refresh

    # --- level management ----------------------------------------------------
    def need(self, ct, levels):
        """Refresh ct if it has fewer than `levels` levels left (App. C)."""
        if ct.level < levels:
            self.refreshes += 1
            self.refresh_obj += 1
            return self.he.refresh(ct, self.refresh_obj)
        return ct

    def align(self, a, b):
        lv = min(a.level, b.level)
        return self.he.drop(a, lv), self.he.drop(b, lv)

    def mult(self, a, b):
        a, b = self.need(a, 1), self.need(b, 1)
        a, b = self.align(a, b)
        return self.he.rescale(self.he.mult_relin(a, b))

    def mul_const(self, ct, c, target_scale=None):
        """ct * c with c encoded as the constant polynomial round(c q_l), then a
        rescale by q_l.  The scale is kept, or -- with target_scale -- the
        constant is round(c q_l target / scale) and the result has exactly the
        target scale (resets the drift of repeated products without a level)."""
        ct = self.need(ct, 1)
        P = self.P
        lv = ct.level
        if target_scale is None:
            m = int(round(c * float(P.q[lv])))
        else:
            m = int(round(c * float(P.q[lv]) * target_scale / ct.scale))
        qs = P.qs(lv)
        cs = [m % q for q in qs]
        out = Ct(_c.mulconst_limbs(qs, ct.c0, cs), _c.mulconst_limbs(qs, ct.c1, cs), lv, ct.scale, ct.period)
        out = self.he.rescale(out, keep_scale=True)
        if target_scale is not None:
            out.scale = target_scale
        return out

    def mul_mask(self, ct, slots):
        """ct . slots with the slot vector encoded at scale q_l, then rescale by q_l
        (the ciphertext keeps its scale)."""
        he, P = self.he, self.P
        ct = self.need(ct, 1)
        pt = he.encode(slots.astype(np.complex128), float(P.q[ct.level]), P.qs(ct.level))
        out = he.pmult_pt(ct, pt, 1.0)
        return he.rescale(out, keep_scale=True)

    def add_const(self, ct, c):
        """PAdd of the constant c: c0 += round(c * scale) on the constant coefficient."""
        P = self.P
        m = int(round(c * ct.scale))
        c0 = ct.c0.copy()
        for i, q in enumerate(P.qs(ct.level)):
            c0[i, 0] = (int(c0[i, 0]) + m) % q
        return Ct(c0, ct.c1.copy(), ct.level, ct.scale, ct.period)

    def to_scale(self, ct, level, scale):
        """Bring ct to `level` with scale `scale`: drop to level+1, multiply by
        the integer K = round(q_{level+1} scale / ct.scale), rescale (C13)."""
        P = self.P
        ct = self.need(ct, level + 1)
        ct = self.he.drop(ct, level + 1)
        K = int(round(float(P.q[level + 1]) * scale / ct.scale))
        qs = P.qs(level + 1)
        out = Ct(_c.mulconst_limbs(qs, ct.c0, [K % q for q in qs]),
                 _c.mulconst_limbs(qs, ct.c1, [K % q for q in qs]), level + 1, ct.scale, ct.period)
        out = self.he.rescale(out, keep_scale=True)
        out.scale = scale
        return out

    def sub_matched(self, a, b):
        """a - b after bringing b to a's level and scale (when they differ)."""
        if b.level != a.level or b.scale != a.scale:
            if b.level > a.level and b.scale == a.scale:
                b = self.he.drop(b, a.level)
            elif a.level > b.level and a.scale == b.scale:
                a = self.he.drop(a, b.level)
            else:
                # matching the scales spends one level: refresh an operand that has none
                a = self.need(a, 1)
                b = self.need(b, 1)
                lv = min(a.level, b.level) - 1
                a = self.to_scale(a, lv, a.scale) if a.level != lv else a
                b = self.to_scale(b, lv, a.scale)
        return self.he.sub(a, b)

    # --- Aggregate (Sec. 5.2, algorithm Aggregate) ----------------------------
    def aggregate(self, ct, axis, n):
        """Sum over rows (axis 0) or within rows (axis 1, with the first-column
        mask) of a replicated n x n block."""
        he = self.he
        n2 = n * n
        A = self.H.replicate(ct, n)
        if axis == 0:
            i = n
            while i < n2:
                A = he.add(A, he.rotate(A, i % n2))
                i <<= 1
            return A
        i = 1
        while i < n:
            A = he.add(A, he.rotate(A, i % n2))
            i <<= 1
        mask = tile(((np.arange(n2) % n) == 0).astype(np.float64), n, self.P.S)
        A = self.mul_mask(A, mask)
        i = -1
        while i > -n:
            A = he.add(A, he.rotate(A, i % n2))
            i <<= 1
        return A

    # --- HCovMtrx (Sec. 5.2) -----------------------------------------------------
    def covariance(self, blocks, s, n, n1z, n1t, centered=False, relin_once=False, dcd_z=0, dcd_t=0):
        """blocks[l][j] = ct(X_j[l]); returns C[a][b] for a, b < k.  relin_once
        and dcd_z / dcd_t select the block products' relinearisation and
        Diagonal Convergence Decomposition (HMM.hmatmul; Sec. 7 runs the
        covariance's products decomposed at maximum diagonal 32)."""
        upper, sums = self.covariance_partial(blocks, s, n, n1z, n1t, centered, relin_once, dcd_z, dcd_t)
        return self.covariance_finish(upper, sums, s, n, n1z, blocks[0][0].level, centered, dcd_z, dcd_t)

    def covariance_partial(self, blocks, s, n, n1z, n1t, centered=False, relin_once=False, dcd_z=0, dcd_t=0):
        """The sums over the given row blocks that HCovMtrx needs (Sec. 5.2):
        upper[(a, b)] = sum_l X_a[l]^T X_b[l] / s for a <= b (1/s folded into
        the transposition of X_a[l]), and unless centred sums[j] = sum_l
        X_j[l].  Both are plain sums over the row blocks, so the parts of
        disjoint sets of row blocks add up (mod q) to those of their union."""
        he, H = self.he, self.H
        nrb, k = len(blocks), len(blocks[0])
        inv_s = 1.0 / s
        XT = [[H.transpose(blocks[l][j], n, n1z, prescale=inv_s) for j in range(k)] for l in range(nrb)]
        Xr = [[H.replicate(blocks[l][j], n) for j in range(k)] for l in range(nrb)]
        upper = {}
        for a in range(k):
            for b in range(a, k):
                acc = None
                for l in range(nrb):
                    A = XT[l][a]
                    B = he.drop(Xr[l][b], A.level)
                    p = H.hmatmul(A, B, n, n1z, n1t, relin_once=relin_once, dcd_z=dcd_z, dcd_t=dcd_t)
                    acc = p if acc is None else he.add(acc, p)
                upper[(a, b)] = acc
        sums = []
        if not centered:
            for j in range(k):
                acc = blocks[0][j]
                for l in range(1, nrb):
                    acc = he.add(acc, blocks[l][j])
                sums.append(acc)
        return upper, sums

    def covariance_finish(self, upper, sums, s, n, n1z, block_level, centered=False, dcd_z=0, dcd_t=0):
        """HCovMtrx from the row-block sums: blocks a > b as G of block (b, a),
        one common level, and (not centred) minus mu_a^T mu_b with
        mu_j = (1/s) Aggregate_0(sums[j]); block_level = the input blocks' level."""
        he, H = self.he, self.H
        k = len(sums) if sums else int(round((np.sqrt(8 * len(upper) + 1) - 1) / 2))
        inv_s = 1.0 / s
        C = [[None] * k for _ in range(k)]
        for (a, b), ct in upper.items():
            C[a][b] = ct
        for a in range(k):
            for b in range(a):
                C[a][b] = H.transpose(C[b][a], n, n1z)
        lv = min(C[a][b].level for a in range(k) for b in range(k))
        for a in range(k):
            for b in range(k):
                C[a][b] = he.drop(C[a][b], lv)
        if centered:
            return C
        mu = []
        for j in range(k):
            m = self.aggregate(sums[j], 0, n)
            mu.append(self.mul_const(m, inv_s))
        muT = [H.transpose(m, n, n1z) for m in mu]
        # mu^T mu is multiplied at the level at which the X^T X products were
        # multiplied, so both are rescaled by the same prime and their scales
        # (Delta^2 / q) agree exactly
        depth = 2 + max((n - 1) // dcd_z + 1 if dcd_z else 1, (n - 2) // dcd_t + 1 if dcd_t else 1)
        pl = (block_level - 1) - (depth - 1)
        for a in range(k):
            for b in range(k):
                t = he.rescale(he.mult_relin(he.drop(muT[a], pl), he.drop(mu[b], pl)))
                C[a][b] = self.sub_matched(C[a][b], t)
        return C

    # --- PowerMethod pieces (Sec. 6.1) ------------------------------------------
    def taylor_init(self, x, B2):
        """T(x) = x0^-1/2 (3/2 - x/(2 x0)), x0 = B^2/2 + 1: one constant product, one constant add."""
        x0 = B2 / 2.0 + 1.0
        t = self.mul_const(x, -0.5 * x0 ** -1.5)
        return self.add_const(t, 1.5 * x0 ** -0.5)

    def newton2(self, x, y):
        """Two Newton steps as one composite of five levels (Sec. 7):
        u = x y^2 (2 levels), 3 - u, then (3 - u)^2, y1/2 = (y/4)(3 - u) and
        u/4 (level 3), x y1^2 = (u/4)(3 - u)^2 (level 4), and
        y2 = (y1/2)(3 - x y1^2) (level 5).  Returns (x, y2)."""
        P = self.P
        y = self.need(y, 5)
        x = self.need(x, 5)
        b = self.mult(y, y)
        yq = self.mul_const(y, 0.25)
        u = self.mult(b, x)
        s = self.add_const(self.mul_const_int(u, -1), 3.0)
        s2 = self.mult(s, s)
        y1h = self.mult(yq, s)
        lw = s2.level
        T = P.delta * float(P.q[lw]) * float(P.q[lw - 1]) / (y1h.scale * s2.scale)
        uq = self.mul_const(u, 0.25, target_scale=T)
        w = self.mult(uq, s2)
        s3 = self.add_const(self.mul_const_int(w, -1), 3.0)
        return x, self.mult(y1h, s3)

    def newton(self, x, y, iters):
        """y <- (3y - x y^3)/2, three levels per iteration (with
        compose_newton: pairs of iterations as five-level composites)."""
        if self.compose_newton:
            for _ in range(iters // 2):
                x, y = self.newton2(x, y)
            iters %= 2
        for _ in range(iters):
            y = self.need(y, 3)
            x = self.need(x, 3)
            t1 = self.mult(y, y)
            t2 = self.mult(y, x)
            t3 = self.mult(t1, t2)
            y3 = self.to_scale(self.mul_const_int(y, 3), t3.level, t3.scale)
            d = self.he.sub(y3, t3)
            y = self.mul_const(d, 0.5, target_scale=self.P.delta)
        return y

    def mul_const_int(self, ct, m):
        """ct * m for a small integer m (no rescale, no level)."""
        qs = self.P.qs(ct.level)
        cs = [m % q for q in qs]
        return Ct(_c.mulconst_limbs(qs, ct.c0, cs), _c.mulconst_limbs(qs, ct.c1, cs), ct.level, ct.scale,
                  ct.period)

    def axis_flip(self, V, axis, n):
        """AxisFlipping: identity mask, then Aggregate on the other axis."""
        he = self.he
        n2 = n * n
        eye = tile((np.arange(n2) // n == np.arange(n2) % n).astype(np.float64), n, self.P.S)
        out = []
        for v in V:
            w = self.mul_mask(self.H.replicate(v, n), eye)
            out.append(self.aggregate(w, (axis + 1) % 2, n))
        return out

    def line_mask(self, axis, j, n):
        """Row j (axis 0) or column j (axis 1) of the n x n block, tiled."""
        n2 = n * n
        idx = np.arange(n2)
        m = (idx // n == j) if axis == 0 else (idx % n == j)
        return tile(m.astype(np.float64), n, self.P.S)

    def packed_refresh(self, V, axis, n):
        """App. C: the k segments of the vector (each replicated along `axis`)
        refreshed as one ciphertext: segment j keeps only its row j (axis 0) or
        column j (axis 1) -- one level --, the k lines are added and refreshed
        once, then each segment is cut out again (one level) and replicated
        (rows: rotations by n 2^i; columns: moved to column 0 by a rotation by
        j, then rotations by -2^i)."""
        he = self.he
        n2 = n * n
        packed = None
        for j, v in enumerate(V):
            m = self.mul_mask(self.H.replicate(v, n), self.line_mask(axis, j, n))
            packed = m if packed is None else self.add_aligned(packed, m)
        self.refreshes += 1
        self.refresh_obj += 1
        packed = he.refresh(packed, self.refresh_obj)
        out = []
        for j in range(len(V)):
            u = self.mul_mask(packed, self.line_mask(axis, j, n))
            if axis == 0:
                i = n
                while i < n2:
                    u = he.add(u, he.rotate(u, i % n2))
                    i <<= 1
            else:
                if j:
                    u = he.rotate(u, j % n2)
                i = -1
                while i > -n:
                    u = he.add(u, he.rotate(u, i % n2))
                    i <<= 1
            out.append(u)
        return out

    def refresh_vector(self, V, axis, n):
        """With pack_refresh, before a covariance transformation (which spends
        up to 2 levels): segments with fewer than 2 levels are refreshed
        together by packed_refresh when every segment has a level to spend on
        the cut, else each such segment once."""
        if not self.pack_refresh or min(v.level for v in V) >= 2:
            return V
        if len(V) > 1 and min(v.level for v in V) >= 1:
            return self.packed_refresh(V, axis, n)
        return [self.need(v, 2) for v in V]

    def cov_apply(self, C, V, axis, n):
        """One covariance transformation (Sec. 6.1.1): axis-0 input -> axis-1 output and back."""
        he = self.he
        k = len(V)
        V = [self.need(v, 1) for v in V]      # each segment enters k products
        out = []
        for i in range(k):
            acc = None
            for j in range(k):
                blk = C[i][j] if axis == 0 else C[j][i]
                p = self.mult(blk, V[j])
                acc = p if acc is None else self.add_aligned(acc, p)
            out.append(self.aggregate(acc, (axis + 1) % 2, n))
        return out, (axis + 1) % 2

    def add_aligned(self, a, b):
        a, b = self.align(a, b)
        return self.he.add(a, b)

    def power_method(self, C, V0, axis, n, l_P, newton_counts, B2):
        """HPowerMethod: l_P normalised transformations, then one more for the eigenvalue."""
        V = V0
        for t in range(l_P + 1):
            V = self.refresh_vector(V, axis, n)
            Vn, axis_n = self.cov_apply(C, V, axis, n)
            if t < l_P:
                acc = None
                for v in Vn:
                    p = self.mult(v, v)
                    acc = p if acc is None else self.add_aligned(acc, p)
                norm2 = self.aggregate(acc, (axis_n + 1) % 2, n)
                g = self.taylor_init(self.need(norm2, 1), B2)
                inv = self.newton(norm2, g, newton_counts[t])
                Vn = [self.mult(v, inv) for v in Vn]
                V, axis = Vn, axis_n
            else:
                Vf = self.axis_flip(V, axis, n)       # V in the axis of Vn
                acc = None
                for a_, b_ in zip(Vn, Vf):
                    p = self.mult(a_, b_)
                    acc = p if acc is None else self.add_aligned(acc, p)
                lam = self.aggregate(acc, (axis_n + 1) % 2, n)
                return lam, V, axis, Vf

    def eigen_shift(self, C, lam, V, axis, VT, n):
        """HEigenShift: C[a][b] -= lambda v_a v_b^T (column-replicated v_a times row-replicated v_b)."""
        k = len(V)
        col = [self.need(v, 1) for v in (V if axis == 1 else VT)]
        row = [self.need(v, 1) for v in (VT if axis == 1 else V)]
        lam = self.need(lam, 1)
        out = [[None] * k for _ in range(k)]
        for a in range(k):
            for b in range(k):
                vv = self.mult(col[a], row[b])
                t = self.mult(lam, vv)
                out[a][b] = self.sub_matched(C[a][b], t)
        return out
