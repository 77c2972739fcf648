// eval.cu -- key switching, rotations, products, rescale, the double-hoisted
// linear transforms and the JKLS matrix product, all on batches of B
// ciphertexts laid out contiguously as [B][2][level+1][N] (NTT domain).
#include <algorithm>
#include <cmath>
#include <sstream>

#include "eval.h"

namespace he {

// ------------------------------------------------------------ key switch
// Decompose (Sec. 3.3): poly of every item (stride item_s) -> digits
// [B][ndig][l+1+alpha][N] in the NTT domain.
void modup(Ctx *c, const u64 *poly, long item_s, int B, int level, u64 *digits) {
    const int N = c->N, nq = level + 1;
    Buf coef(&c->pool, (size_t)B * nq * N);
    launch_copy_rows(coef.p, (long)nq * N, poly, item_s, B, (long)nq * N, c->stream);
    ntt_inv(c, coef.p, (long)B * nq, c->map_q(level), c->stream);
    const long rows = (long)B * c->ndig(level) * c->qp_rows(level);
    if (c->logN >= 14 && c->logN <= 16) {
        // the digit's own rows are the input's NTT-domain rows: copy them and
        // transform only the extended rows
        launch_modup_bconv(c, coef.p, digits, B, level, c->stream, poly, item_s);
        RowSkip sk;
        sk.rows_per_digit = c->qp_rows(level);
        sk.ndig = c->ndig(level);
        sk.alpha = c->alpha;
        sk.nq = nq;
        ntt_fwd(c, digits, rows, c->map_qp(level), c->stream, &sk);
    } else {
        launch_modup_bconv(c, coef.p, digits, B, level, c->stream);
        ntt_fwd(c, digits, rows, c->map_qp(level), c->stream);
    }
    c->n_dp += B;
}

// ModDown: items of [rows][N] over Q_l P (contiguous) -> out items of [l+1][N]
// with item stride out_s.
void moddown(Ctx *c, const u64 *u, int items, int level, u64 *out, long out_s, const u64 *add, long add_s) {
    const int N = c->N, rows = c->qp_rows(level), a = c->alpha;
    Buf pc(&c->pool, (size_t)items * a * N), conv(&c->pool, (size_t)items * (level + 1) * N);
    launch_copy_rows(pc.p, (long)a * N, u + (long)(level + 1) * N, (long)rows * N, items, (long)a * N, c->stream);
    ntt_inv(c, pc.p, (long)items * a, c->map_p(), c->stream);
    launch_moddown_bconv(c, pc.p, conv.p, items, level, c->stream);
    if (c->logN >= 14 && c->logN <= 16) {
        // the NTT's last pass writes out = (u_Q - conv) P^-1 directly
        SubScale ep;
        ep.u = u, ep.us = (long)rows * N, ep.out = out, ep.os = out_s, ep.w = c->d_dn_Pinv;
        ep.rows_per_item = level + 1;
        ep.add = add, ep.as = add_s;
        ntt_fwd_subscale(c, conv.p, (long)items * (level + 1), c->map_q(level), c->stream, ep);
    } else {
        ntt_fwd(c, conv.p, (long)items * (level + 1), c->map_q(level), c->stream);
        launch_moddown_final(c, out, u, conv.p, add, items, level, (long)rows * N, out_s, add_s, c->stream);
    }
}

const u64 *need_key(Ctx *c, uint32_t g) {
    auto it = c->rtk.find(g);
    if (it == c->rtk.end()) {
        std::ostringstream os;
        os << "rotation key for Galois element " << g << " missing";
        throw HeError(HE_ERR_KEY_MISSING, os.str());
    }
    return it->second;
}

// Hoisted rotation kept in Q_l P: u = <kappa_g(digits), rtk_g> + (P kappa_g(c0), 0).
// ct: [B][2][l+1][N]; out: [B][2][rows][N].
void rot_qp(Ctx *c, const u64 *ct, int B, int level, const u64 *digits, uint32_t g, u64 *out) {
    const u64 *key = need_key(c, g);
    launch_multsum(c, out, digits, key, g, B, level, ct, 2L * (level + 1) * c->N, c->stream);
    c->n_ms += B;
}

// G hoisted rotations of the same Decompose output, kept in Q_l P; the
// digits are read once per launch for up to kMultSumMaxKeys keys.
void rot_qp_multi(Ctx *c, const u64 *ct, int B, int level, const u64 *digits, const uint32_t *gs, int G,
                  u64 *const *outs) {
    if (G <= 0) return;
    std::vector<const u64 *> keys(G);
    for (int k = 0; k < G; k++) keys[k] = need_key(c, gs[k]);
    launch_multsum_multi(c, outs, digits, keys.data(), gs, G, B, level, ct, 2L * (level + 1) * c->N, c->stream);
    c->n_ms += (long long)B * G;
}

// Full rotation from precomputed digits: ModDown(rot_qp) = kappa(c0) + ModDown(IP0), ModDown(IP1).
void rotate_digits(Ctx *c, const u64 *ct, int B, int level, const u64 *digits, uint32_t g, u64 *out) {
    const int rows = c->qp_rows(level);
    Buf u(&c->pool, (size_t)B * 2 * rows * c->N);
    rot_qp(c, ct, B, level, digits, g, u.p);
    moddown(c, u.p, 2 * B, level, out, (long)(level + 1) * c->N);
    c->n_md += B;
}

void rotate(Ctx *c, const u64 *ct, int B, int level, uint32_t g, u64 *out) {
    const int rows = c->qp_rows(level);
    Buf dg(&c->pool, (size_t)B * c->ndig(level) * rows * c->N);
    modup(c, ct + (long)(level + 1) * c->N, 2L * (level + 1) * c->N, B, level, dg.p);
    rotate_digits(c, ct, B, level, dg.p, g, out);
}

// Rescale (App. A): [B][2][l+1][N] -> [B][2][l][N], round(c / q_l).
void rescale(Ctx *c, const u64 *in, int B, int level, u64 *out) {
    const int N = c->N;
    if (level < 1) throw HeError(HE_ERR_LEVEL, "rescale at level 0");
    Buf last(&c->pool, (size_t)2 * B * N), t(&c->pool, (size_t)2 * B * level * N);
    launch_copy_rows(last.p, N, in + (long)level * N, (long)(level + 1) * N, 2 * B, N, c->stream);
    RowMap one = RowMap::single(level);
    ntt_inv(c, last.p, 2L * B, one, c->stream);
    launch_rescale_prep(c, last.p, t.p, 2 * B, level, c->stream);
    if (c->logN >= 14 && c->logN <= 16) {
        // the NTT's last pass writes out = (in - t) q_l^-1 directly
        SubScale ep;
        ep.u = in, ep.us = (long)(level + 1) * N, ep.out = out, ep.os = (long)level * N, ep.w = c->lc(level).d_rs_inv;
        ep.rows_per_item = level;
        ntt_fwd_subscale(c, t.p, 2L * B * level, c->map_q(level - 1), c->stream, ep);
    } else {
        ntt_fwd(c, t.p, 2L * B * level, c->map_q(level - 1), c->stream);
        launch_rescale_final(c, out, in, t.p, 2 * B, level, (long)(level + 1) * N, (long)level * N, c->stream);
    }
}

// Level drop: keep limbs 0..to of both polys.
void drop(Ctx *c, const u64 *in, int B, int level, int to, u64 *out) {
    const int N = c->N;
    launch_copy_rows(out, (long)(to + 1) * N, in, (long)(level + 1) * N, 2 * B, (long)(to + 1) * N, c->stream);
}

// out[p] = in[idx[p]] dropped from level to `to` (both polynomials).
static void drop_gather(Ctx *c, const u64 *in, const int *idx, int P, int level, int to, u64 *out) {
    const int N = c->N;
    for (int p = 0; p < P; p++)
        launch_copy_rows(out + (size_t)p * 2 * (to + 1) * N, (long)(to + 1) * N,
                         in + (size_t)idx[p] * 2 * (level + 1) * N, (long)(level + 1) * N, 2, (long)(to + 1) * N,
                         c->stream);
}

// out (holding (d0, d1)) += KeySwitch(d2, rlk): the relinearisation of Mult.
// The ModDown's last store adds into out in place.
static void relin_into(Ctx *c, const u64 *d2, int B, int level, u64 *out) {
    if (!c->rlk) throw HeError(HE_ERR_KEY_MISSING, "relinearisation key missing");
    const int N = c->N, nq = level + 1, rows = c->qp_rows(level);
    Buf dg(&c->pool, (size_t)B * c->ndig(level) * rows * N);
    modup(c, d2, (long)nq * N, B, level, dg.p);
    Buf u(&c->pool, (size_t)B * 2 * rows * N);
    launch_multsum(c, u.p, dg.p, c->rlk, 1u, B, level, nullptr, 0, c->stream);
    c->n_ms += B;
    moddown(c, u.p, 2 * B, level, out, (long)nq * N, out, (long)nq * N);
    c->n_md += B;
}

// Mult (App. A): tensor (d0, d1, d2), then (d0, d1) + KeySwitch(d2, rlk);
// with accumulate, the product is added to what out holds (the tensor adds
// (d0, d1), the ModDown's last store adds the key switch).
void mult_relin(Ctx *c, const u64 *a, const u64 *b, int B, int level, u64 *out, bool accumulate, int b_level) {
    if (!c->rlk) throw HeError(HE_ERR_KEY_MISSING, "relinearisation key missing");
    const int N = c->N, nq = level + 1;
    const long cs = 2L * nq * N;
    if (b_level < level) b_level = level;
    Buf d2(&c->pool, (size_t)B * nq * N);
    launch_tensor_acc(c, out, d2.p, a, b, B, nq, cs, 2L * (b_level + 1) * N, c->map_q(level), c->stream, accumulate,
                      false, (long)(b_level + 1) * N);
    relin_into(c, d2.p, B, level, out);
}

void add(Ctx *c, const u64 *a, const u64 *b, int B, int level, u64 *out) {
    launch_add(c, out, a, b, 2L * B * (level + 1), c->map_q(level), c->stream);
}

// --------------------------------------------------- plaintext diagonals
// Cached encodings (NTT, Montgomery) over Q_l P of a diagonal slot vector at
// scale q_l.  kind/n/t/rot/value/k as in k_diag_fill.
const u64 *get_pt(Ctx *c, int kind, int n, long t, long rot, double value, int k, int level,
                  const DcdFactor *fac) {
    std::ostringstream os;
    os << kind << ':' << n << ':' << t << ':' << rot << ':' << k << ':' << level << ':';
    if (fac) os << fac->id << ':';
    os.precision(17);
    os << value;
    std::string key = os.str();
    auto it = c->ptcache.find(key);
    if (it != c->ptcache.end()) return it->second;
    const int N = c->N, rows = c->qp_rows(level);
    u64 *pt = nullptr;
    if (cudaMalloc(&pt, (size_t)rows * N * 8) != cudaSuccess) {
        cudaGetLastError();
        throw HeError(HE_ERR_OOM, "plaintext cache allocation failed");
    }
    Buf zr(&c->pool, c->S), zi(&c->pool, c->S), m(&c->pool, N);
    if (fac)
        launch_dcd_fill(c, (double *)zr.p, fac->dev, n, t, rot, value, c->stream);
    else
        launch_diag_fill(c, (double *)zr.p, kind, n, t, rot, value, k, c->stream);
    cudaMemsetAsync(zi.p, 0, (size_t)c->S * 8, c->stream);
    launch_encode(c, (double *)zr.p, (double *)zi.p, (double)c->primes[level], (i64 *)m.p, c->stream);
    RowMap qp = c->map_qp(level);
    launch_small_to_rns(c, (const i64 *)m.p, pt, rows, qp, c->stream);
    ntt_fwd(c, pt, rows, qp, c->stream);
    launch_to_mont(c, pt, pt, rows, qp, c->stream);
    c->ptcache[key] = pt;
    c->ptcache_bytes += (size_t)rows * N * 8;
    return pt;
}

// Does diagonal `t` of transform `kind` hold a non-zero entry?
static bool diag_nonzero(int kind, int n, long t) {
    switch (kind) {
    case 0: return t > -n && t < n;                         // Z, eq. 5
    case 1: return t >= 0 && t % n == 0 && t / n < n;       // T, eq. 6
    case 2: {                                                // G, (n-1) k
        long a = n - 1;
        if (a == 0) return t == 0;
        if (t % a != 0) return false;
        long kk = t / a;
        return kk > -n && kk < n;
    }
    }
    return false;
}

static long mod_pos(long x, long m) { return ((x % m) + m) % m; }

// Double-hoisted BSGS linear transform (eq. 3', Sec. 3.3):
//   U m = sum_i rho( sum_j rho(u_{a(n1 i + j)}; -a n1 i) . rho(m; a j) ; a n1 i ),
// babies kept in Q_l P from one Decompose; giant groups summed in Q_l P,
// ModDown'd, rotated (kept in Q_l P) and accumulated; one final ModDown and a
// rescale by q_l (plaintexts at scale q_l keep the ciphertext scale).
// in: [B][2][l+1][N]; out: [B][2][l][N].
//
// n1_sub > 0 (simple key substitution, Sec. 4.2): the babies use only the
// keys a s, 0 < s < n1_sub.  They come in groups of n1_sub - 1: the first
// rotates the input by a s; every later group takes the last baby of the
// previous one, ModDown'd to a ciphertext c and Decomposed, and rotates c by
// a s, so that baby j = b + s is rho(c; a s) with c = rho(m; a b).
void lintrans(Ctx *c, const u64 *in, int B, int level, int kind, int n, long a, int n1, int gi0, int gi1,
              double value, u64 *out, const DcdFactor *fac, int n1_sub) {
    const int N = c->N, nq = level + 1, rows = c->qp_rows(level);
    const long n2 = (long)n * n;
    const size_t qpct = (size_t)2 * rows * N;   // one item over Q_l P
    Buf dg(&c->pool, (size_t)B * c->ndig(level) * rows * N);
    modup(c, in + (long)nq * N, 2L * nq * N, B, level, dg.p);
    std::vector<Buf> R;
    R.emplace_back(&c->pool, B * qpct);
    launch_lift_P(c, R[0].p, in, 2 * B, level, (long)nq * N, (long)rows * N, c->stream);
    for (int j = 1; j < n1; j++) R.emplace_back(&c->pool, B * qpct);
    Buf acc(&c->pool, B * qpct), S(&c->pool, B * qpct), ctmp(&c->pool, (size_t)B * 2 * nq * N),
        dg2(&c->pool, (size_t)B * c->ndig(level) * rows * N), T(&c->pool, B * qpct);
    const int head = n1_sub > 1 && n1_sub < n1 ? n1_sub : n1;
    for (int j0 = 1, base = 0; j0 < n1; j0 += head - 1) {
        const u64 *src = in, *sdg = dg.p;
        if (j0 > 1) {
            // the previous group's last baby as the next source
            base = j0 - 1;
            moddown(c, R[base].p, 2 * B, level, ctmp.p, (long)nq * N);
            c->n_md += B;
            modup(c, ctmp.p + (long)nq * N, 2L * nq * N, B, level, dg2.p);
            src = ctmp.p, sdg = dg2.p;
        }
        std::vector<uint32_t> gs;
        std::vector<u64 *> outs;
        for (int j = j0; j < std::min(n1, j0 + head - 1); j++) {
            gs.push_back(galois_of_step(c, mod_pos(a * (j - base), n2)));
            outs.push_back(R[j].p);
        }
        rot_qp_multi(c, src, B, level, sdg, gs.data(), (int)gs.size(), outs.data());
    }
    bool have = false;
    RowMap qp = c->map_qp(level);
    for (int i = gi0; i < gi1; i++) {
        std::vector<const u64 *> pts, Rs;
        for (int j = 0; j < n1; j++) {
            long t = a * ((long)n1 * i + j);
            if (fac ? !fac->diags.count(mod_pos(t, n2)) : !diag_nonzero(kind, n, t)) continue;
            pts.push_back(get_pt(c, kind, n, t, mod_pos(-a * n1 * i, n2), value, 0, level, fac));
            Rs.push_back(R[j].p);
        }
        if (pts.empty()) continue;
        launch_pmul_acc(c, S.p, pts.data(), Rs.data(), (int)pts.size(), B, level, (long)qpct, c->stream);
        const u64 *term = S.p;
        if (i != 0) {
            moddown(c, S.p, 2 * B, level, ctmp.p, (long)nq * N);
            c->n_md += B;
            modup(c, ctmp.p + (long)nq * N, 2L * nq * N, B, level, dg2.p);
            rot_qp(c, ctmp.p, B, level, dg2.p, galois_of_step(c, mod_pos(a * n1 * i, n2)), T.p);
            term = T.p;
        }
        if (!have) {
            cudaMemcpyAsync(acc.p, term, B * qpct * 8, cudaMemcpyDeviceToDevice, c->stream);
            have = true;
        } else {
            launch_add(c, acc.p, acc.p, term, 2L * B * rows, qp, c->stream);
        }
    }
    moddown(c, acc.p, 2 * B, level, ctmp.p, (long)nq * N);
    c->n_md += B;
    rescale(c, ctmp.p, B, level, out);
}

// ct <- ct + Rot(ct, -n^2 2^j) for j = 0 .. log2(S/n^2)-1 (period n^2).
void replicate(Ctx *c, u64 *ct, int B, int level, int n) {
    const long n2 = (long)n * n;
    Buf r(&c->pool, (size_t)B * 2 * (level + 1) * c->N);
    for (long s = n2; s < c->S; s *= 2) {
        rotate(c, ct, B, level, galois_of_step(c, c->S - s), r.p);
        add(c, ct, r.p, B, level, ct);
    }
}

// JKLS product (eq. 4) with the hoisting of Sec. 4.1; A, B: [Bn][2][l+1][N]
// replicated with period n^2; out: [Bn][2][l-2][N].
// A chain of decomposition factors (application order) on B items at
// `level`; the output, one level per factor lower, goes to out.
static void apply_chain(Ctx *c, const u64 *in, int B, int level, const DcdChain &ch, int n, long a_left, int n1,
                        int gi0, int gi1, u64 *out) {
    const size_t w = (size_t)2 * (level + 1) * c->N;
    Buf t0(&c->pool, B * w), t1(&c->pool, B * w);
    const u64 *cur = in;
    int lv = level;
    for (size_t f = 0; f + 1 < ch.factors.size(); f++) {
        u64 *dst = (f % 2 == 0) ? t0.p : t1.p;
        lintrans(c, cur, B, lv, 8, n, ch.factors[f].step, 2, 0, 1, 1.0, dst, &ch.factors[f]);
        cur = dst;
        lv--;
    }
    lintrans(c, cur, B, lv, 8, n, a_left, n1, gi0, gi1, 1.0, out, &ch.factors.back());
}

// sigma (Z) or tau (T) of B items at `level`, undecomposed (one level) or
// through the decomposition chains (Sec. 4.2 DMatrixMult), then dropped to
// level `to`.
static void zt_stage(Ctx *c, const u64 *in, int B, int level, bool is_t, int n, int n1, int np, int to, u64 *out) {
    const int N = c->N;
    const int m = dcd_levels(n, np, is_t), lo = level - m;
    const size_t wlo = (size_t)2 * (lo + 1) * N;
    Buf r(&c->pool, lo == to ? 1 : B * wlo);
    u64 *dst = lo == to ? out : r.p;   // no copy when no level has to be dropped
    if (!np) {
        if (is_t) lintrans(c, in, B, level, 1, n, n, n1, 0, n / n1, 1.0, dst);
        else lintrans(c, in, B, level, 0, n, 1, n1, -(n / n1), n / n1, 1.0, dst);
    } else if (is_t) {
        apply_chain(c, in, B, level, dcd_chain(c, 2, n, np), n, n, n1, 0, np / n1 + 1, dst);
    } else {
        Buf r2(&c->pool, B * wlo);
        apply_chain(c, in, B, level, dcd_chain(c, 0, n, np), n, 1, n1, 0, np / n1, dst);
        apply_chain(c, in, B, level, dcd_chain(c, 1, n, np), n, 1, n1, -(np / n1), 1, r2.p);
        add(c, dst, r2.p, B, lo, dst);
    }
    if (lo != to) drop(c, r.p, B, lo, to, out);
}

void zt_stage_public(Ctx *c, const u64 *in, int B, int level, bool is_t, int n, int n1, int np, int to, u64 *out) {
    zt_stage(c, in, B, level, is_t, n, n1, np, to, out);
}

// Products A[ia[p]] B[ib[p]], p < P, of nA distinct left and nB distinct
// right operands: sigma, C^k and their hoisted rotations run once per left
// operand, tau and R^k once per right operand, whatever the number of
// products each takes part in (Sec. 5.2, covariance Optimizations 1 and 2:
// C^k Z X_j^T and R^k T X_i computed once for every product that uses
// them; the batch of products is the row segment).  Only the current k's
// A^(k), B^(k) are held, so the memory grows with nA + nB + P, not with n.
void hmatmul_pairs(Ctx *c, const u64 *A, int nA, const u64 *Bm, int nB, const int *ia, const int *ib, int P,
                   int level, int n, int n1z, int n1t, u64 *out, bool relin_once, int dcd_z, int dcd_t) {
    const int depth = hmatmul_depth(n, dcd_z, dcd_t);
    if (level < depth) throw HeError(HE_ERR_LEVEL, "matrix product needs more levels");
    if ((dcd_z && (dcd_z >= n || dcd_z % n1z)) || (dcd_t && (dcd_t >= n || dcd_t % n1t)))
        throw HeError(HE_ERR_ARG, "a decomposition needs n' < n with n1 dividing n'");
    const int N = c->N;
    const long n2m = (long)n * n;
    const int l1 = level - (depth - 2), l2 = l1 - 1;
    const size_t ct1 = (size_t)2 * (l1 + 1) * N, ct2 = (size_t)2 * (l2 + 1) * N;
    const int rows1 = c->qp_rows(l1);
    const size_t qp1 = (size_t)2 * rows1 * N, dig1 = (size_t)c->ndig(l1) * rows1 * N;
    bool ident = nA == P && nB == P;
    for (int p = 0; p < P && ident; p++) ident = ia[p] == p && ib[p] == p;
    for (int p = 0; p < P; p++)
        if (ia[p] < 0 || ia[p] >= nA || ib[p] < 0 || ib[p] >= nB) throw HeError(HE_ERR_ARG, "bad operand index");
    Buf A0(&c->pool, nA * ct1), B0(&c->pool, nB * ct1);
    zt_stage(c, A, nA, level, false, n, n1z, dcd_z, l1, A0.p);
    zt_stage(c, Bm, nB, level, true, n, n1t, dcd_t, l1, B0.p);

    // C^k sources A_g, A'_g and R^k sources B_g with their digits
    Buf Ag(&c->pool, nA * ct1), Apg(&c->pool, nA * ct1), Bg(&c->pool, nB * ct1);
    Buf dA(&c->pool, nA * dig1), dAp(&c->pool, nA * dig1), dB(&c->pool, nB * dig1);
    Buf tmpA(&c->pool, nA * ct1), tmpB(&c->pool, nB * ct1);
    cudaMemcpyAsync(Ag.p, A0.p, nA * ct1 * 8, cudaMemcpyDeviceToDevice, c->stream);
    modup(c, Ag.p + (long)(l1 + 1) * N, (long)ct1, nA, l1, dA.p);
    rotate_digits(c, Ag.p, nA, l1, dA.p, galois_of_step(c, mod_pos(-n, n2m)), Apg.p);
    modup(c, Apg.p + (long)(l1 + 1) * N, (long)ct1, nA, l1, dAp.p);
    cudaMemcpyAsync(Bg.p, B0.p, nB * ct1 * 8, cudaMemcpyDeviceToDevice, c->stream);
    modup(c, Bg.p + (long)(l1 + 1) * N, (long)ct1, nB, l1, dB.p);
    int gA = 0, gB = 0;

    Buf acc(&c->pool, P * ct2), Ak(&c->pool, nA * ct2);
    // the operands of every product, gathered when operands are shared
    Buf AkP(&c->pool, ident ? 1 : P * ct2), BkP(&c->pool, ident ? 1 : P * ct2);
    // relin_once: the summed d2 of the n tensors (d0, d1 are summed in acc)
    Buf acc2(&c->pool, relin_once ? (size_t)P * (l2 + 1) * N : 1);
    Buf R1(&c->pool, nA * qp1), R2(&c->pool, nA * qp1), S(&c->pool, nA * qp1), Akp(&c->pool, nA * ct1);
    RowMap q2 = c->map_q(l2);

    // The babies of a source are all its hoisted rotations at once (one
    // read of the source's digits per kMultSumMaxKeys keys):
    //   C^k: rotations by b of A_g and A'_g kept in Q_l P, b = 1..n1z-1;
    //   R^k: rotations by n b of B_g (ModDown'd), b = 1..n1t-1.
    const int nbA = n1z - 1, nbB = n1t - 1;
    Buf SA(&c->pool, (size_t)std::max(1, nbA) * nA * qp1);
    Buf UB(&c->pool, (size_t)std::max(1, nbB) * nB * qp1), BB(&c->pool, (size_t)std::max(1, nbB) * nB * ct1);
    // the babies of giant g, masked and summed in one pass:
    // SA_b = m_k (.) rot_qp(A_g; b) + m'_k (.) rot_qp(A'_g; b), k = n1z g + b
    auto babies_A = [&]() {
        std::vector<uint32_t> gs;
        std::vector<u64 *> o;
        std::vector<const u64 *> m1, m2;
        for (int b = 1; b <= nbA; b++) {
            const int k = n1z * gA + b;
            gs.push_back(galois_of_step(c, b % n2m));
            o.push_back(SA.p + (size_t)(b - 1) * nA * qp1);
            m1.push_back(get_pt(c, 3, n, 0, 0, 1.0, k, l1));
            m2.push_back(get_pt(c, 4, n, 0, 0, 1.0, k, l1));
        }
        std::vector<const u64 *> keys(nbA);
        for (int i = 0; i < nbA; i++) keys[i] = need_key(c, gs[i]);
        launch_multsum_ck(c, o.data(), dA.p, dAp.p, keys.data(), gs.data(), m1.data(), m2.data(), nbA, nA, l1,
                          Ag.p, Apg.p, (long)ct1, c->stream);
        c->n_ms += 2LL * nA * nbA;
    };
    auto babies_B = [&]() {
        std::vector<uint32_t> gs;
        std::vector<u64 *> o;
        for (int b = 1; b <= nbB; b++) {
            gs.push_back(galois_of_step(c, ((long)n * b) % n2m));
            o.push_back(UB.p + (size_t)(b - 1) * nB * qp1);
        }
        rot_qp_multi(c, Bg.p, nB, l1, dB.p, gs.data(), nbB, o.data());
        if (nbB > 0) {
            moddown(c, UB.p, 2 * nB * nbB, l1, BB.p, (long)(l1 + 1) * N);
            c->n_md += (long long)nB * nbB;
        }
    };
    if (nbA > 0) babies_A();
    if (nbB > 0) babies_B();
    for (int k = 0; k < n; k++) {
        // ---- A^(k) = C^k A^(0) at level l2
        int g = k / n1z, b = k % n1z;
        while (gA < g) {
            rotate_digits(c, Ag.p, nA, l1, dA.p, galois_of_step(c, n1z % n2m), tmpA.p);
            std::swap(Ag, tmpA);
            modup(c, Ag.p + (long)(l1 + 1) * N, (long)ct1, nA, l1, dA.p);
            rotate_digits(c, Apg.p, nA, l1, dAp.p, galois_of_step(c, n1z % n2m), tmpA.p);
            std::swap(Apg, tmpA);
            modup(c, Apg.p + (long)(l1 + 1) * N, (long)ct1, nA, l1, dAp.p);
            gA++;
            if (nbA > 0) babies_A();
        }
        if (k == 0) {
            drop(c, A0.p, nA, l1, l2, Ak.p);
        } else {
            const u64 *Sk = S.p;
            if (b > 0) {
                Sk = SA.p + (size_t)(b - 1) * nA * qp1;
            } else {
                // the giant's own sources, lifted to Q_l P, masked and summed
                launch_lift_P(c, R1.p, Ag.p, 2 * nA, l1, (long)(l1 + 1) * N, (long)rows1 * N, c->stream);
                launch_lift_P(c, R2.p, Apg.p, 2 * nA, l1, (long)(l1 + 1) * N, (long)rows1 * N, c->stream);
                const u64 *pts[2] = {get_pt(c, 3, n, 0, 0, 1.0, k, l1), get_pt(c, 4, n, 0, 0, 1.0, k, l1)};
                const u64 *Rs[2] = {R1.p, R2.p};
                launch_pmul_acc(c, S.p, pts, Rs, 2, nA, l1, (long)qp1, c->stream);
            }
            moddown(c, Sk, 2 * nA, l1, Akp.p, (long)(l1 + 1) * N);
            c->n_md += nA;
            rescale(c, Akp.p, nA, l1, Ak.p);
        }
        // ---- B^(k) = R^k B^(0), dropped to l2
        int gb2 = k / n1t, bb = k % n1t;
        while (gB < gb2) {
            rotate_digits(c, Bg.p, nB, l1, dB.p, galois_of_step(c, ((long)n * n1t) % n2m), tmpB.p);
            std::swap(Bg, tmpB);
            modup(c, Bg.p + (long)(l1 + 1) * N, (long)ct1, nB, l1, dB.p);
            gB++;
            if (nbB > 0) babies_B();
        }
        // B^(k) stays at level l1: the tensor reads its first l2 + 1 limbs
        const u64 *bsrc = bb == 0 ? Bg.p : BB.p + (size_t)(bb - 1) * nB * ct1;
        // ---- product, relinearised, accumulated at level l2
        const u64 *xa = Ak.p, *xb = bsrc;
        int b_level = l1;
        if (!ident) {
            for (int p = 0; p < P; p++) {
                cudaMemcpyAsync(AkP.p + (size_t)p * ct2, Ak.p + (size_t)ia[p] * ct2, ct2 * 8,
                                cudaMemcpyDeviceToDevice, c->stream);
            }
            drop_gather(c, bsrc, ib, P, l1, l2, BkP.p);
            xa = AkP.p, xb = BkP.p, b_level = l2;
        }
        if (relin_once) {
            const long cs = 2L * (l2 + 1) * N;
            launch_tensor(c, acc.p, acc2.p, xa, xb, P, l2 + 1, cs, 2L * (b_level + 1) * N, q2, c->stream, k > 0,
                          (long)(b_level + 1) * N);
        } else {
            mult_relin(c, xa, xb, P, l2, acc.p, k > 0, b_level);
        }
    }
    if (relin_once) relin_into(c, acc2.p, P, l2, acc.p);
    rescale(c, acc.p, P, l2, out);
}

void hmatmul(Ctx *c, const u64 *A, const u64 *Bm, int Bn, int level, int n, int n1z, int n1t, u64 *out,
             bool relin_once, int dcd_z, int dcd_t) {
    std::vector<int> id(Bn);
    for (int i = 0; i < Bn; i++) id[i] = i;
    hmatmul_pairs(c, A, Bn, Bm, Bn, id.data(), id.data(), Bn, level, n, n1z, n1t, out, relin_once, dcd_z, dcd_t);
}

}  // namespace he
