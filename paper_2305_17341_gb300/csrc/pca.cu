// pca.cu -- Aggregate, covariance (HCovMtrx), PowerMethod with Lazy
// Normalization, EigenShift and the interactive refresh (Sec. 5, Sec. 6,
// App. C), composed from the batched evaluation routines of eval.cu.
//
// Block convention: blocks[l*k + j] is the l-th row block of the j-th feature
// block of the dataset (Sec. 5.1); cov[a*k + b] is block row a, block column
// b.  A vector segment is row-replicated (axis 0) or column-replicated
// (axis 1) in an n x n block (Sec. 6.1.1).
#include <cfenv>
#include <cmath>
#include <vector>

#include "ctapi.h"
#include "stages.h"

namespace he {

// owned ciphertext handle
struct HC {
    he_ct *p = nullptr;
    HC() = default;
    explicit HC(he_ct *q) : p(q) {}
    HC(const HC &) = delete;
    HC &operator=(const HC &) = delete;
    HC(HC &&o) noexcept : p(o.p) { o.p = nullptr; }
    HC &operator=(HC &&o) noexcept {
        if (this != &o) {
            free_ct(p);
            p = o.p;
            o.p = nullptr;
        }
        return *this;
    }
    ~HC() { free_ct(p); }
    he_ct *operator->() const { return p; }
    he_ct *release() {
        he_ct *q = p;
        p = nullptr;
        return q;
    }
};

struct RefreshState {
    uint32_t next_obj;
    int count;
};

// round half to even, as the oracle's Python round()
static long long rne(double x) { return (long long)std::nearbyint(x); }

static u64 mod_signed(long long m, u64 q) {
    long long r = m % (long long)q;
    return (u64)(r < 0 ? r + (long long)q : r);
}

// products per batched pass inside one covariance (bounds the temporaries)
static const int kCovBatch = 16;

class PcaOps {
public:
    Ctx *c;
    RefreshState *rs;
    PcaOps(Ctx *cc, RefreshState *r) : c(cc), rs(r) {}

    HC make(int level, double scale, int period) { return HC(new_ct(c, level, scale, period)); }

    HC clone(const he_ct *a) {
        HC o = make(a->level, a->scale, a->period);
        cudaMemcpyAsync(o->d, a->d, ct_words(c, a->level) * 8, cudaMemcpyDeviceToDevice, c->stream);
        return o;
    }

    HC dropto(const he_ct *a, int lv) {
        if (lv == a->level) return clone(a);
        HC o = make(lv, a->scale, a->period);
        drop(c, a->d, 1, a->level, lv, o->d);
        return o;
    }

    // App. C / Sec. 7.2.3 refresh: integer message at q_0, re-encrypted at level L
    HC refresh(const he_ct *a) {
        const int N = c->N, L = c->L;
        Buf m(&c->pool, N), mi(&c->pool, N), rns(&c->pool, (size_t)(L + 1) * N);
        launch_dec_q0(c, a->d, a->d + (size_t)(a->level + 1) * N, m.p, c->stream);
        RowMap one = RowMap::single(0);
        ntt_inv(c, m.p, 1, one, c->stream);
        launch_centre_i64_q0(c, m.p, (i64 *)mi.p, c->stream);
        launch_small_to_rns(c, (const i64 *)mi.p, rns.p, L + 1, c->map_q(L), c->stream);
        ntt_fwd(c, rns.p, L + 1, c->map_q(L), c->stream);
        rs->next_obj++;
        rs->count++;
        HC o = make(L, a->scale, a->period);
        encrypt_poly(c, rns.p, L, rs->next_obj, true, o->d);
        return o;
    }

    HC need(HC a, int levels) {
        if (a->level < levels) return refresh(a.p);
        return a;
    }

    std::pair<HC, HC> align(HC a, HC b) {
        int lv = std::min(a->level, b->level);
        if (a->level != lv) a = dropto(a.p, lv);
        if (b->level != lv) b = dropto(b.p, lv);
        return {std::move(a), std::move(b)};
    }

    HC add_ct(const he_ct *a, const he_ct *b) {
        HC o = make(a->level, a->scale, std::min(a->period, b->period));
        add(c, a->d, b->d, 1, a->level, o->d);
        return o;
    }

    HC sub_ct(const he_ct *a, const he_ct *b) {
        HC o = make(a->level, a->scale, std::min(a->period, b->period));
        launch_sub(c, o->d, a->d, b->d, 2L * (a->level + 1), c->map_q(a->level), c->stream);
        return o;
    }

    HC rescale_ct(const he_ct *a, bool keep) {
        double s = keep ? a->scale : a->scale / (double)c->primes[a->level];
        HC o = make(a->level - 1, s, a->period);
        rescale(c, a->d, 1, a->level, o->d);
        return o;
    }

    HC mult(HC a, HC b) {
        a = need(std::move(a), 1);
        b = need(std::move(b), 1);
        auto ab = align(std::move(a), std::move(b));
        const he_ct *x = ab.first.p, *y = ab.second.p;
        HC t = make(x->level, x->scale * y->scale, std::min(x->period, y->period));
        mult_relin(c, x->d, y->d, 1, x->level, t->d);
        return rescale_ct(t.p, false);
    }
    HC mult(const he_ct *a, const he_ct *b) { return mult(clone(a), clone(b)); }

    void scalar_mul(const he_ct *a, long long m, u64 *out) {
        std::vector<ShoupPair> w(a->level + 1);
        for (int i = 0; i <= a->level; i++) w[i] = h_shoup(mod_signed(m, c->primes[i]), c->primes[i]);
        launch_scalar_mul_rows(c, out, a->d, 2L * (a->level + 1), a->level + 1, w.data(), c->map_q(a->level),
                               c->stream);
    }

    // ct * c with c as the constant polynomial round(c q_l) (or scaled to a
    // target scale), then rescale by q_l
    HC mul_const(HC a, double cv, const double *target = nullptr) {
        a = need(std::move(a), 1);
        int lv = a->level;
        double q = (double)c->primes[lv];
        long long m = target ? rne(((cv * q) * (*target)) / a->scale) : rne(cv * q);
        HC t = make(lv, a->scale, a->period);
        scalar_mul(a.p, m, t->d);
        HC o = rescale_ct(t.p, true);
        if (target) o->scale = *target;
        return o;
    }

    HC mul_const_int(const he_ct *a, long long m) {
        HC t = make(a->level, a->scale, a->period);
        scalar_mul(a, m, t->d);
        return t;
    }

    HC add_const(HC a, double cv) {
        long long m = rne(cv * a->scale);
        std::vector<u64> v(a->level + 1);
        for (int i = 0; i <= a->level; i++) v[i] = mod_signed(m, c->primes[i]);
        launch_scalar_add_rows(c, a->d, a->level + 1, v.data(), c->map_q(a->level), c->stream);
        return a;
    }

    // slot-vector mask (kind 6 first column, 7 identity) at scale q_l, rescale keeps the scale
    HC mul_mask(HC a, int kind, int n, int k = 0) {
        a = need(std::move(a), 1);
        int lv = a->level;
        const u64 *pt = get_pt(c, kind, n, 0, 0, 1.0, k, lv);
        HC t = make(lv, a->scale, a->period);
        const long nq = (long)(lv + 1) * c->N;
        launch_mulM(c, t->d, a->d, pt, lv + 1, c->map_q(lv), c->stream);
        launch_mulM(c, t->d + nq, a->d + nq, pt, lv + 1, c->map_q(lv), c->stream);
        return rescale_ct(t.p, true);
    }

    HC to_scale(HC a, int level, double scale) {
        a = need(std::move(a), level + 1);
        a = dropto(a.p, level + 1);
        double q = (double)c->primes[level + 1];
        long long K = rne((q * scale) / a->scale);
        HC t = make(level + 1, a->scale, a->period);
        scalar_mul(a.p, K, t->d);
        HC o = rescale_ct(t.p, true);
        o->scale = scale;
        return o;
    }

    HC sub_matched(HC a, HC b) {
        if (b->level != a->level || b->scale != a->scale) {
            if (b->level > a->level && b->scale == a->scale) {
                b = dropto(b.p, a->level);
            } else if (a->level > b->level && a->scale == b->scale) {
                a = dropto(a.p, b->level);
            } else {
                // matching the scales spends one level: refresh an operand that has none
                a = need(std::move(a), 1);
                b = need(std::move(b), 1);
                const int lv = std::min(a->level, b->level) - 1;
                const double sa = a->scale;  // read before a is moved into the call
                if (a->level != lv) a = to_scale(std::move(a), lv, sa);
                b = to_scale(std::move(b), lv, sa);
            }
        }
        return sub_ct(a.p, b.p);
    }

    HC replicated(const he_ct *a, int n) {
        HC o = clone(a);
        if (o->period != n * n) {
            replicate(c, o->d, 1, o->level, n);
            o->period = n * n;
        }
        return o;
    }

    HC rot(const he_ct *a, long step) {
        HC o = make(a->level, a->scale, a->period);
        rotate(c, a->d, 1, a->level, galois_of_step(c, step), o->d);
        return o;
    }

    // Aggregate (Sec. 5.2)
    HC aggregate(const he_ct *in, int axis, int n) {
        const long n2 = (long)n * n;
        HC A = replicated(in, n);
        if (axis == 0) {
            for (long i = n; i < n2; i <<= 1) {
                HC r = rot(A.p, i % n2);
                A = add_ct(A.p, r.p);
            }
            return A;
        }
        for (long i = 1; i < n; i <<= 1) {
            HC r = rot(A.p, i % n2);
            A = add_ct(A.p, r.p);
        }
        A = mul_mask(std::move(A), 6, n);
        for (long i = -1; i > -n; i *= 2) {
            HC r = rot(A.p, ((i % n2) + n2) % n2);
            A = add_ct(A.p, r.p);
        }
        return A;
    }

    HC transpose(const he_ct *a, int n, int n1, double prescale) {
        HC r = replicated(a, n);
        HC o = make(a->level - 1, a->scale, n * n);
        lintrans(c, r->d, 1, a->level, 2, n, n - 1, n1, -(n / n1), n / n1, prescale, o->d);
        return o;
    }

    // ---------------------------------------------------------- covariance
    // HCovMtrx (Sec. 5.2) in three stages, so that a server can merge the
    // block products of several jobs into one batched pass:
    //   1. cov_prepare: X_j[l]^T with 1/s folded into the G diagonals, and
    //      the replicated X_j[l]; appends the products X_a[l]^T X_b[l]
    //      (a <= b) in the order l, a, b, so that the k(k+1)/2 products of
    //      a row block, which share their operands, run in one batch
    //   2. cov_upper: C[a][b] = sum over l of those products
    //   3. cov_finish: the blocks below the diagonal as G(C[b][a]), one
    //      common level, and (not centred) minus mu_a^T mu_b
    struct CovPlan {
        int nrb = 0, k = 0, n = 0, s = 0, n1z = 0, n1t = 0;
        bool centered = true, relin_once = false;
        int dcd_z = 0, dcd_t = 0;   // Diagonal Convergence Decomposition of the block products
        std::vector<he_ct *> blocks;
        std::vector<HC> XT, Xr;
    };

    void cov_prepare(CovPlan &P, std::vector<ProdSpec> &prods) {
        const double inv_s = 1.0 / P.s;
        const int k = P.k;
        P.XT.clear();
        P.Xr.clear();
        P.XT.resize(P.nrb * k);
        P.Xr.resize(P.nrb * k);
        for (int l = 0; l < P.nrb; l++)
            for (int j = 0; j < k; j++) {
                P.XT[l * k + j] = transpose(P.blocks[l * k + j], P.n, P.n1z, inv_s);
                P.Xr[l * k + j] = replicated(P.blocks[l * k + j], P.n);
            }
        for (int l = 0; l < P.nrb; l++)
            for (int a = 0; a < k; a++)
                for (int b = a; b < k; b++)
                    prods.push_back({P.XT[l * k + a].p, P.Xr[l * k + b].p, P.n, P.n1z, P.n1t, P.relin_once,
                                     P.dcd_z, P.dcd_t});
    }

    // Takes ownership of the products made from cov_prepare's list.
    std::vector<HC> cov_upper(CovPlan &P, he_ct *const *outs) {
        const int k = P.k, ppl = k * (k + 1) / 2;
        std::vector<HC> own;
        for (int t = 0; t < ppl * P.nrb; t++) own.emplace_back(outs[t]);
        std::vector<HC> C(k * k);
        int pr = 0;   // index of the pair (a, b) within a row block
        for (int a = 0; a < k; a++)
            for (int b = a; b < k; b++, pr++) {
                HC acc = std::move(own[pr]);
                for (int l = 1; l < P.nrb; l++) {
                    HC o = std::move(own[(size_t)l * ppl + pr]);
                    add(c, acc->d, o->d, 1, acc->level, acc->d);
                }
                C[a * k + b] = std::move(acc);
            }
        P.XT.clear();
        P.Xr.clear();
        return C;
    }

    std::vector<HC> cov_finish(const CovPlan &P, std::vector<HC> C) {
        const int k = P.k, nrb = P.nrb;
        std::vector<HC> sums;
        if (!P.centered)
            for (int j = 0; j < k; j++) {
                HC acc = clone(P.blocks[j]);
                for (int l = 1; l < nrb; l++) acc = add_ct(acc.p, P.blocks[l * k + j]);
                sums.push_back(std::move(acc));
            }
        return cov_finish_sums(k, P.n, P.s, P.centered, P.n1z, P.dcd_z, P.dcd_t, P.blocks[0]->level, std::move(C),
                               std::move(sums));
    }

    // The last stage from the upper blocks C[a][b] (a <= b) and, when not
    // centred, the column sums sum_l X_j[l] of the input blocks (level
    // block_level): whether they cover all row blocks or were summed from
    // the parts of several devices makes no difference to the words.
    std::vector<HC> cov_finish_sums(int k, int n, int s, bool centered, int n1z, int dcd_z, int dcd_t,
                                    int block_level, std::vector<HC> C, std::vector<HC> sums) {
        for (int a = 0; a < k; a++)
            for (int b = 0; b < a; b++) C[a * k + b] = transpose(C[b * k + a].p, n, n1z, 1.0);
        int lv = C[0]->level;
        for (auto &x : C) lv = std::min(lv, x->level);
        for (auto &x : C)
            if (x->level != lv) x = dropto(x.p, lv);
        if (centered) return C;
        const double inv_s = 1.0 / s;
        std::vector<HC> mu, muT;
        for (int j = 0; j < k; j++) {
            HC m = aggregate(sums[j].p, 0, n);
            mu.push_back(mul_const(std::move(m), inv_s));
        }
        for (int j = 0; j < k; j++) muT.push_back(transpose(mu[j].p, n, n1z, 1.0));
        // the mean product is taken at the level of the block products' inputs minus 2
        const int pl = block_level - hmatmul_depth(n, dcd_z, dcd_t);
        for (int a = 0; a < k; a++)
            for (int b = 0; b < k; b++) {
                HC x = dropto(muT[a].p, pl), y = dropto(mu[b].p, pl);
                HC t = make(pl, x->scale * y->scale, n * n);
                mult_relin(c, x->d, y->d, 1, pl, t->d);
                HC tr = rescale_ct(t.p, false);
                C[a * k + b] = sub_matched(std::move(C[a * k + b]), std::move(tr));
            }
        return C;
    }

    // The part of HCovMtrx that a device computes on its own row blocks
    // when the rows are spread over several devices (Sec. 5.2: the block
    // products of different row blocks are independent): the upper blocks of
    // X^T X / s summed over these row blocks, and (not centred) the column
    // sums of the blocks.  Sums of these parts over the devices, residue by
    // residue mod q, are what cov_finish_sums takes.
    void covariance_partial(he_ct *const *blocks, int nrb, int k, int n, int s, bool centered, int n1z, int n1t,
                            bool relin_once, int dcd_z, int dcd_t, std::vector<HC> &upper, std::vector<HC> &sums) {
        CovPlan P;
        P.relin_once = relin_once;
        P.dcd_z = dcd_z;
        P.dcd_t = dcd_t;
        P.nrb = nrb;
        P.k = k;
        P.n = n;
        P.s = s;
        P.n1z = n1z;
        P.n1t = n1t;
        P.centered = centered;
        P.blocks.assign(blocks, blocks + (size_t)nrb * k);
        std::vector<ProdSpec> prods;
        cov_prepare(P, prods);
        std::vector<he_ct *> outs;
        const int ppl = k * (k + 1) / 2;
        run_products(prods, outs, std::max(1, kCovBatch / ppl) * ppl);
        std::vector<HC> C = cov_upper(P, outs.data());
        upper.clear();
        for (int a = 0; a < k; a++)
            for (int b = a; b < k; b++) upper.push_back(std::move(C[a * k + b]));
        sums.clear();
        if (!centered)
            for (int j = 0; j < k; j++) {
                HC acc = clone(P.blocks[j]);
                for (int l = 1; l < nrb; l++) acc = add_ct(acc.p, P.blocks[l * k + j]);
                sums.push_back(std::move(acc));
            }
    }

    std::vector<HC> covariance(he_ct *const *blocks, int nrb, int k, int n, int s, bool centered, int n1z,
                               int n1t, bool relin_once = false, int dcd_z = 0, int dcd_t = 0) {
        CovPlan P;
        P.relin_once = relin_once;
        P.dcd_z = dcd_z;
        P.dcd_t = dcd_t;
        P.nrb = nrb;
        P.k = k;
        P.n = n;
        P.s = s;
        P.n1z = n1z;
        P.n1t = n1t;
        P.centered = centered;
        P.blocks.assign(blocks, blocks + (size_t)nrb * k);
        std::vector<ProdSpec> prods;
        cov_prepare(P, prods);
        std::vector<he_ct *> outs;
        const int ppl = k * (k + 1) / 2;
        run_products(prods, outs, std::max(1, kCovBatch / ppl) * ppl);
        return cov_finish(P, cov_upper(P, outs.data()));
    }

    // -------------------------------------------------------- PowerMethod
    HC taylor_init(HC x, double B2) {
        double x0 = B2 / 2.0 + 1.0;
        HC t = mul_const(std::move(x), -0.5 * std::pow(x0, -1.5));
        return add_const(std::move(t), 1.5 * std::pow(x0, -0.5));
    }

    // Two Newton steps as one composite of five levels (Sec. 7 composites
    // two InvSRT iterations into one that spends a level less): with
    // u = x y^2, y1/2 = (y/4)(3 - u) and x y1^2 = (u/4)(3 - u)^2 at level 3
    // and 4, y2 = (y1/2)(3 - x y1^2) at level 5; the constant 1/4 of u carries
    // the scale that puts y2 at Delta.
    void newton2(HC &x, HC &y) {
        const double delta = std::ldexp(1.0, c->prm.log_delta);
        y = need(std::move(y), 5);
        x = need(std::move(x), 5);
        HC b = mult(y.p, y.p);
        HC yq = mul_const(clone(y.p), 0.25);
        HC u = mult(b.p, x.p);
        HC s = add_const(mul_const_int(u.p, -1), 3.0);
        HC s2 = mult(s.p, s.p);
        HC y1h = mult(yq.p, s.p);
        const int lw = s2->level;
        const double T = delta * (double)c->primes[lw] * (double)c->primes[lw - 1] / (y1h->scale * s2->scale);
        HC uq = mul_const(std::move(u), 0.25, &T);
        HC w = mult(std::move(uq), std::move(s2));
        HC s3 = add_const(mul_const_int(w.p, -1), 3.0);
        y = mult(std::move(y1h), std::move(s3));
    }

    HC newton(HC x, HC y, int iters) {
        const double delta = std::ldexp(1.0, c->prm.log_delta);
        if (c->newton_compose) {
            for (int it = 0; it < iters / 2; it++) newton2(x, y);
            iters %= 2;
        }
        for (int it = 0; it < iters; it++) {
            y = need(std::move(y), 3);
            x = need(std::move(x), 3);
            HC t1 = mult(y.p, y.p);
            HC t2 = mult(y.p, x.p);
            HC t3 = mult(std::move(t1), std::move(t2));
            HC y3 = to_scale(mul_const_int(y.p, 3), t3->level, t3->scale);
            HC d = sub_ct(y3.p, t3.p);
            y = mul_const(std::move(d), 0.5, &delta);
        }
        return y;
    }

    HC add_aligned(HC a, HC b) {
        auto ab = align(std::move(a), std::move(b));
        return add_ct(ab.first.p, ab.second.p);
    }

    // App. C: the k segments of the vector (each replicated along `axis`)
    // refreshed as one ciphertext: segment j keeps only its row j (axis 0)
    // or column j (axis 1) -- one level --, the k lines are added and
    // refreshed once, then each segment is cut out again (one level) and
    // replicated (rows: rotations by n 2^i; columns: moved to column 0 by a
    // rotation by j, then rotations by -2^i).
    std::vector<HC> packed_refresh(const std::vector<HC> &V, int axis, int n) {
        const long n2 = (long)n * n;
        const int line = axis == 0 ? 10 : 11;
        HC packed;
        for (size_t j = 0; j < V.size(); j++) {
            HC m = mul_mask(replicated(V[j].p, n), line, n, (int)j);
            packed = packed.p ? add_aligned(std::move(packed), std::move(m)) : std::move(m);
        }
        HC fresh = refresh(packed.p);
        std::vector<HC> out;
        for (size_t j = 0; j < V.size(); j++) {
            HC u = mul_mask(clone(fresh.p), line, n, (int)j);
            if (axis == 0) {
                for (long i = n; i < n2; i <<= 1) {
                    HC r = rot(u.p, i % n2);
                    u = add_ct(u.p, r.p);
                }
            } else {
                if (j) u = rot(u.p, (long)j % n2);
                for (long i = -1; i > -n; i *= 2) {
                    HC r = rot(u.p, ((i % n2) + n2) % n2);
                    u = add_ct(u.p, r.p);
                }
            }
            out.push_back(std::move(u));
        }
        return out;
    }

    // Before a covariance transformation (up to 2 levels), with packed
    // refresh on: segments with fewer than 2 levels are refreshed together by
    // packed_refresh when every segment has a level for the cut, else each
    // such segment once.
    std::vector<HC> refresh_vector(std::vector<HC> V, int axis, int n) {
        if (!c->pack_refresh) return V;
        int lo = V[0]->level;
        for (auto &v : V) lo = std::min(lo, v->level);
        if (lo >= 2) return V;
        if (V.size() > 1 && lo >= 1) return packed_refresh(V, axis, n);
        for (auto &v : V) v = need(std::move(v), 2);
        return V;
    }

    // a ciphertext that several products take, refreshed once (kept in hold)
    // when it has no level left
    const he_ct *once(const he_ct *a, std::vector<HC> &hold) {
        if (a->level >= 1) return a;
        hold.push_back(refresh(a));
        return hold.back().p;
    }

    std::vector<HC> cov_apply(he_ct *const *C, int k, const std::vector<HC> &V0, int axis, int n) {
        // each segment enters k products: refreshed once, before the first
        std::vector<HC> hold;
        std::vector<const he_ct *> V;
        for (auto &v : V0) V.push_back(once(v.p, hold));
        std::vector<HC> out;
        for (int i = 0; i < k; i++) {
            HC acc;
            for (int j = 0; j < k; j++) {
                const he_ct *blk = axis == 0 ? C[i * k + j] : C[j * k + i];
                HC p = mult(blk, V[j]);
                acc = acc.p ? add_aligned(std::move(acc), std::move(p)) : std::move(p);
            }
            out.push_back(aggregate(acc.p, (axis + 1) % 2, n));
        }
        return out;
    }

    std::vector<HC> axis_flip(const std::vector<HC> &V, int axis, int n) {
        std::vector<HC> out;
        for (auto &v : V) {
            HC w = mul_mask(replicated(v.p, n), 7, n);
            out.push_back(aggregate(w.p, (axis + 1) % 2, n));
        }
        return out;
    }

    void power_method(he_ct *const *C, int k, int n, he_ct *const *V0, int axis, int l_P, const int *counts,
                      double B2, HC &lam, std::vector<HC> &Vout, std::vector<HC> &VT, int &axis_out) {
        std::vector<HC> V;
        for (int j = 0; j < k; j++) V.push_back(clone(V0[j]));
        for (int t = 0; t <= l_P; t++) {
            V = refresh_vector(std::move(V), axis, n);
            std::vector<HC> Vn = cov_apply(C, k, V, axis, n);
            int axis_n = (axis + 1) % 2;
            if (t < l_P) {
                HC acc;
                for (auto &v : Vn) {
                    HC p = mult(v.p, v.p);
                    acc = acc.p ? add_aligned(std::move(acc), std::move(p)) : std::move(p);
                }
                HC norm2 = aggregate(acc.p, (axis_n + 1) % 2, n);
                HC g = taylor_init(need(clone(norm2.p), 1), B2);
                HC inv = newton(std::move(norm2), std::move(g), counts[t]);
                std::vector<HC> Vs;
                for (auto &v : Vn) Vs.push_back(mult(v.p, inv.p));
                V = std::move(Vs);
                axis = axis_n;
            } else {
                std::vector<HC> Vf = axis_flip(V, axis, n);
                HC acc;
                for (int i = 0; i < k; i++) {
                    HC p = mult(Vn[i].p, Vf[i].p);
                    acc = acc.p ? add_aligned(std::move(acc), std::move(p)) : std::move(p);
                }
                lam = aggregate(acc.p, (axis_n + 1) % 2, n);
                Vout = std::move(V);
                VT = std::move(Vf);
                axis_out = axis;
                return;
            }
        }
    }

    std::vector<HC> eigen_shift(he_ct *const *C, int k, const he_ct *lam, he_ct *const *V, int axis,
                                he_ct *const *VT) {
        // every segment enters k products and lambda k^2: each refreshed
        // once, before the first
        std::vector<HC> hold;
        hold.reserve(2 * k + 1);
        std::vector<const he_ct *> col, row;
        for (int a = 0; a < k; a++) col.push_back(once(axis == 1 ? V[a] : VT[a], hold));
        for (int b = 0; b < k; b++) row.push_back(once(axis == 1 ? VT[b] : V[b], hold));
        const he_ct *lm = once(lam, hold);
        std::vector<HC> out;
        for (int a = 0; a < k; a++)
            for (int b = 0; b < k; b++) {
                HC vv = mult(col[a], row[b]);
                HC t = mult(lm, vv.p);
                out.push_back(sub_matched(clone(C[a * k + b]), std::move(t)));
            }
        return out;
    }

    // Privacy-Preserving PCA (Sec. 6.2): l_E rounds of PowerMethod and
    // EigenShift on a private copy of the covariance blocks.
    void pca(he_ct *const *cov, int k, int n, int l_E, he_ct *const *v0, int axis, int l_P, const int *counts,
             double B2, std::vector<HC> &lam_out, std::vector<HC> &V_out, std::vector<int> &ax_out) {
        std::vector<HC> C;
        for (int i = 0; i < k * k; i++) C.push_back(clone(cov[i]));
        for (int m = 0; m < l_E; m++) {
            std::vector<he_ct *> Cp(k * k);
            for (int i = 0; i < k * k; i++) Cp[i] = C[i].p;
            HC lam;
            std::vector<HC> Vo, VTo;
            int ax = 0;
            power_method(Cp.data(), k, n, v0 + (size_t)m * k, axis, l_P, counts, B2, lam, Vo, VTo, ax);
            if (m + 1 < l_E) {
                std::vector<he_ct *> Vp(k), VTp(k);
                for (int j = 0; j < k; j++) {
                    Vp[j] = Vo[j].p;
                    VTp[j] = VTo[j].p;
                }
                C = eigen_shift(Cp.data(), k, lam.p, Vp.data(), ax, VTp.data());
            }
            lam_out.push_back(std::move(lam));
            for (auto &v : Vo) V_out.push_back(std::move(v));
            ax_out.push_back(ax);
        }
    }
};

// ------------------------------------------------------ stages for serving
struct CovStage {
    PcaOps::CovPlan plan;
};

CovStage *cov_begin(Ctx *c, he_ct *const *blocks, int nrb, int k, int n, int s, bool centered, int n1z, int n1t,
                    std::vector<ProdSpec> &prods, bool relin_once, int dcd_z, int dcd_t) {
    RefreshState st{0, 0};
    PcaOps ops(c, &st);
    CovStage *S = new CovStage;
    PcaOps::CovPlan &P = S->plan;
    P.nrb = nrb;
    P.k = k;
    P.n = n;
    P.s = s;
    P.n1z = n1z;
    P.n1t = n1t;
    P.centered = centered;
    P.relin_once = relin_once;
    P.dcd_z = dcd_z;
    P.dcd_t = dcd_t;
    P.blocks.assign(blocks, blocks + (size_t)nrb * k);
    try {
        ops.cov_prepare(P, prods);
    } catch (...) {
        delete S;
        throw;
    }
    return S;
}

void cov_upper(Ctx *c, CovStage *S, he_ct *const *outs, std::vector<he_ct *> &upper) {
    RefreshState st{0, 0};
    PcaOps ops(c, &st);
    std::vector<HC> C = ops.cov_upper(S->plan, outs);
    upper.assign(C.size(), nullptr);
    for (size_t i = 0; i < C.size(); i++) upper[i] = C[i].release();
}

void cov_finish(Ctx *c, CovStage *S, std::vector<he_ct *> &blocks_io) {
    RefreshState st{0, 0};
    PcaOps ops(c, &st);
    std::vector<HC> C(blocks_io.size());
    for (size_t i = 0; i < C.size(); i++) C[i] = HC(blocks_io[i]), blocks_io[i] = nullptr;
    C = ops.cov_finish(S->plan, std::move(C));
    for (size_t i = 0; i < C.size(); i++) blocks_io[i] = C[i].release();
}

void cov_free(CovStage *S) { delete S; }

void pca_run(Ctx *c, he_ct *const *cov, int k, int n, int l_E, he_ct *const *v0, int axis, int l_P,
             const int *counts, double B2, uint32_t &next_obj, int &count, std::vector<he_ct *> &lams,
             std::vector<he_ct *> &V, std::vector<int> &axes) {
    RefreshState st{next_obj, count};
    PcaOps ops(c, &st);
    std::vector<HC> lo, vo;
    ops.pca(cov, k, n, l_E, v0, axis, l_P, counts, B2, lo, vo, axes);
    next_obj = st.next_obj;
    count = st.count;
    for (auto &x : lo) lams.push_back(x.release());
    for (auto &x : vo) V.push_back(x.release());
}

// Lazy Normalization's PowerMethod simulation (Sec. 6.1.2)
int lazy_schedule(int t, double S, double e, double Bp, double B2, int max_iters, int *counts) {
    const double x0 = B2 / 2.0 + 1.0;
    double l = 1.0;
    for (int p = 0; p < t; p++) {
        l = l * S;
        const bool last = p == t - 1;
        int tau = 0;
        double Sp = 0;
        for (tau = 0; tau <= max_iters; tau++) {
            double x = l * l;
            double y = std::pow(x0, -0.5) * (1.5 - x / (2.0 * x0));
            for (int i = 0; i < tau; i++) y = 0.5 * y * (3.0 - x * y * y);
            Sp = y;
            double a = l * Sp * S;
            if (a * a >= Bp && (!last || std::fabs(1.0 - l * Sp) < e)) break;
        }
        if (tau > max_iters) tau = max_iters;
        counts[p] = tau;
        l = l * Sp;
    }
    return 0;
}

}  // namespace he

using namespace he;

// ----------------------------------------------------------------- C ABI
#define PCA_GUARD_BEGIN try {
#define PCA_GUARD_END                                 \
    }                                                 \
    catch (const HeError &e) {                        \
        set_error(e.what());                          \
        return e.code;                                \
    }                                                 \
    catch (const std::bad_alloc &) {                  \
        set_error("device or host allocation failed"); \
        return HE_ERR_OOM;                            \
    }                                                 \
    catch (const std::exception &e) {                 \
        set_error(e.what());                          \
        return HE_ERR_ARG;                            \
    }

static int sync_status(Ctx &c) {
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("CUDA error: ") + cudaGetErrorString(e));
        return HE_ERR_CUDA;
    }
    return device_status(&c);
}

static bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

extern "C" {

int he_refresh(he_ctx *ctx, const he_ct *ct, he_refresh_state *rs, he_ct **out) {
    if (!ctx || !ct || !rs || !out || ct->ctx != &ctx->c) {
        set_error("bad arguments");
        return HE_ERR_ARG;
    }
    PCA_GUARD_BEGIN
    RefreshState st{rs->next_obj, rs->count};
    PcaOps ops(&ctx->c, &st);
    HC o = ops.refresh(ct);
    if (int rc = sync_status(ctx->c)) return rc;
    rs->next_obj = st.next_obj;
    rs->count = st.count;
    *out = o.release();
    return HE_OK;
    PCA_GUARD_END
}

int he_aggregate(he_ctx *ctx, const he_ct *ct, int axis, int n, he_ct **out) {
    if (!ctx || !ct || !out || ct->ctx != &ctx->c || (axis != 0 && axis != 1) || !pow2(n) ||
        (long)n * n > ctx->c.S) {
        set_error("bad arguments");
        return HE_ERR_ARG;
    }
    if (axis == 1 && ct->level < 1) {
        set_error("Aggregate along rows needs 1 level");
        return HE_ERR_LEVEL;
    }
    PCA_GUARD_BEGIN
    RefreshState st{0, 0};
    PcaOps ops(&ctx->c, &st);
    HC o = ops.aggregate(ct, axis, n);
    if (int rc = sync_status(ctx->c)) return rc;
    *out = o.release();
    return HE_OK;
    PCA_GUARD_END
}

int he_covariance(he_ctx *ctx, he_ct *const *blocks, int n_row_blocks, int k, int n, int s, int centered,
                  const he_mm_sched *sched, he_ct **cov) {
    if (!ctx || !blocks || !cov || !sched || n_row_blocks < 1 || k < 1 || s < 1 || !pow2(n) ||
        (long)n * n > ctx->c.S || !pow2(sched->n1_z) || !pow2(sched->n1_t) || sched->n1_z > n || sched->n1_t > n) {
        set_error("bad arguments");
        return HE_ERR_ARG;
    }
    Ctx &c = ctx->c;
    for (int i = 0; i < n_row_blocks * k; i++) {
        if (!blocks[i] || blocks[i]->ctx != &c) {
            set_error("bad block");
            return HE_ERR_ARG;
        }
        if (blocks[i]->level != blocks[0]->level) {
            set_error("blocks at different levels");
            return HE_ERR_LEVEL;
        }
    }
    if ((sched->dcd_z && (sched->dcd_z >= n || sched->dcd_z % sched->n1_z)) ||
        (sched->dcd_t && (sched->dcd_t >= n || sched->dcd_t % sched->n1_t))) {
        set_error("a decomposition needs n' < n with n1 dividing n'");
        return HE_ERR_ARG;
    }
    // transposition, the products, the mirror transposition and the mean term
    if (blocks[0]->level < hmatmul_depth(n, sched->dcd_z, sched->dcd_t) + 3) {
        set_error("the covariance circuit needs the product's depth + 3 levels");
        return HE_ERR_LEVEL;
    }
    PCA_GUARD_BEGIN
    RefreshState st{0, 0};
    PcaOps ops(&c, &st);
    std::vector<HC> C = ops.covariance(blocks, n_row_blocks, k, n, s, centered != 0, sched->n1_z, sched->n1_t,
                                       sched->relin_once != 0, sched->dcd_z, sched->dcd_t);
    if (int rc = sync_status(c)) return rc;
    for (int i = 0; i < k * k; i++) cov[i] = C[i].release();
    return HE_OK;
    PCA_GUARD_END
}

// Arguments shared by the covariance entry points.
static int check_cov_args(he_ctx *ctx, int k, int n, int s, const he_mm_sched *sched) {
    if (!ctx || !sched || k < 1 || s < 1 || !pow2(n) || (long)n * n > ctx->c.S || !pow2(sched->n1_z) ||
        !pow2(sched->n1_t) || sched->n1_z > n || sched->n1_t > n) {
        set_error("bad arguments");
        return HE_ERR_ARG;
    }
    if ((sched->dcd_z && (sched->dcd_z >= n || sched->dcd_z % sched->n1_z)) ||
        (sched->dcd_t && (sched->dcd_t >= n || sched->dcd_t % sched->n1_t))) {
        set_error("a decomposition needs n' < n with n1 dividing n'");
        return HE_ERR_ARG;
    }
    return HE_OK;
}

int he_covariance_partial(he_ctx *ctx, he_ct *const *blocks, int n_row_blocks, int k, int n, int s, int centered,
                          const he_mm_sched *sched, he_ct **upper, he_ct **colsum) {
    if (int rc = check_cov_args(ctx, k, n, s, sched)) return rc;
    if (!blocks || !upper || n_row_blocks < 1 || (!centered && !colsum)) {
        set_error("bad arguments");
        return HE_ERR_ARG;
    }
    Ctx &c = ctx->c;
    for (int i = 0; i < n_row_blocks * k; i++) {
        if (!blocks[i] || blocks[i]->ctx != &c) {
            set_error("bad block");
            return HE_ERR_ARG;
        }
        if (blocks[i]->level != blocks[0]->level) {
            set_error("blocks at different levels");
            return HE_ERR_LEVEL;
        }
    }
    if (blocks[0]->level < hmatmul_depth(n, sched->dcd_z, sched->dcd_t) + 3) {
        set_error("the covariance circuit needs the product's depth + 3 levels");
        return HE_ERR_LEVEL;
    }
    PCA_GUARD_BEGIN
    RefreshState st{0, 0};
    PcaOps ops(&c, &st);
    std::vector<HC> up, sums;
    ops.covariance_partial(blocks, n_row_blocks, k, n, s, centered != 0, sched->n1_z, sched->n1_t,
                           sched->relin_once != 0, sched->dcd_z, sched->dcd_t, up, sums);
    if (int rc = sync_status(c)) return rc;
    for (size_t i = 0; i < up.size(); i++) upper[i] = up[i].release();
    for (size_t j = 0; j < sums.size(); j++) colsum[j] = sums[j].release();
    return HE_OK;
    PCA_GUARD_END
}

int he_covariance_finish(he_ctx *ctx, he_ct *const *upper, he_ct *const *colsum, int k, int n, int s, int centered,
                         const he_mm_sched *sched, int block_level, he_ct **cov) {
    if (int rc = check_cov_args(ctx, k, n, s, sched)) return rc;
    if (!upper || !cov || (!centered && !colsum)) {
        set_error("bad arguments");
        return HE_ERR_ARG;
    }
    Ctx &c = ctx->c;
    const int nu = k * (k + 1) / 2;
    for (int i = 0; i < nu; i++)
        if (!upper[i] || upper[i]->ctx != &c || upper[i]->level != upper[0]->level || upper[i]->period != n * n) {
            set_error("bad upper block");
            return HE_ERR_ARG;
        }
    if (!centered)
        for (int j = 0; j < k; j++)
            if (!colsum[j] || colsum[j]->ctx != &c || colsum[j]->level != block_level) {
                set_error("bad column sum");
                return HE_ERR_ARG;
            }
    if (upper[0]->level < 1 || block_level < hmatmul_depth(n, sched->dcd_z, sched->dcd_t) + 3) {
        set_error("the covariance circuit needs the product's depth + 3 levels");
        return HE_ERR_LEVEL;
    }
    PCA_GUARD_BEGIN
    RefreshState st{0, 0};
    PcaOps ops(&c, &st);
    std::vector<HC> C(k * k), sums;
    int u = 0;
    for (int a = 0; a < k; a++)
        for (int b = a; b < k; b++) C[a * k + b] = ops.clone(upper[u++]);
    if (!centered)
        for (int j = 0; j < k; j++) sums.push_back(ops.clone(colsum[j]));
    C = ops.cov_finish_sums(k, n, s, centered != 0, sched->n1_z, sched->dcd_z, sched->dcd_t, block_level,
                            std::move(C), std::move(sums));
    if (int rc = sync_status(c)) return rc;
    for (int i = 0; i < k * k; i++) cov[i] = C[i].release();
    return HE_OK;
    PCA_GUARD_END
}

int he_lazy_normalization_schedule(int t, double S, double e, double Bp, double B2, int max_iters, int *counts) {
    if (t < 1 || !counts || S <= 0 || e <= 0 || Bp <= 0 || B2 <= 0 || max_iters < 1) {
        set_error("bad arguments");
        return HE_ERR_ARG;
    }
    return lazy_schedule(t, S, e, Bp, B2, max_iters, counts);
}

int he_power_method(he_ctx *ctx, he_ct *const *cov, int k, int n, he_ct *const *v0, int axis, int l_P,
                    const int *newton_counts, double B2, he_refresh_state *rs, he_ct **lambda, he_ct **V,
                    he_ct **VT, int *axis_out) {
    if (!ctx || !cov || !v0 || !newton_counts || !rs || !lambda || !V || !VT || !axis_out || k < 1 || !pow2(n) ||
        l_P < 1 || (axis != 0 && axis != 1) || B2 <= 0) {
        set_error("bad arguments");
        return HE_ERR_ARG;
    }
    Ctx &c = ctx->c;
    if (c.L < 4) {
        set_error("the PowerMethod needs a chain of at least 4 levels");
        return HE_ERR_LEVEL;
    }
    PCA_GUARD_BEGIN
    RefreshState st{rs->next_obj, rs->count};
    PcaOps ops(&c, &st);
    HC lam;
    std::vector<HC> Vo, VTo;
    int ax = 0;
    ops.power_method(cov, k, n, v0, axis, l_P, newton_counts, B2, lam, Vo, VTo, ax);
    if (int rc = sync_status(c)) return rc;
    rs->next_obj = st.next_obj;
    rs->count = st.count;
    *lambda = lam.release();
    for (int j = 0; j < k; j++) {
        V[j] = Vo[j].release();
        VT[j] = VTo[j].release();
    }
    *axis_out = ax;
    return HE_OK;
    PCA_GUARD_END
}

int he_pca(he_ctx *ctx, he_ct *const *cov, int k, int n, int l_E, he_ct *const *v0, int axis, int l_P,
           const int *newton_counts, double B2, he_refresh_state *rs, he_ct **lambdas, he_ct **V, int *axes) {
    if (!ctx || !cov || !v0 || !newton_counts || !rs || !lambdas || !V || !axes || k < 1 || !pow2(n) || l_E < 1 ||
        l_P < 1 || (axis != 0 && axis != 1) || B2 <= 0) {
        set_error("bad arguments");
        return HE_ERR_ARG;
    }
    Ctx &c = ctx->c;
    PCA_GUARD_BEGIN
    RefreshState st{rs->next_obj, rs->count};
    PcaOps ops(&c, &st);
    std::vector<HC> lam_out, V_out;
    std::vector<int> ax_out;
    ops.pca(cov, k, n, l_E, v0, axis, l_P, newton_counts, B2, lam_out, V_out, ax_out);
    if (int rc = sync_status(c)) return rc;
    rs->next_obj = st.next_obj;
    rs->count = st.count;
    for (int m = 0; m < l_E; m++) {
        lambdas[m] = lam_out[m].release();
        axes[m] = ax_out[m];
    }
    for (size_t i = 0; i < V_out.size(); i++) V[i] = V_out[i].release();
    return HE_OK;
    PCA_GUARD_END
}

int he_eigen_shift(he_ctx *ctx, he_ct **cov, int k, int n, const he_ct *lambda, he_ct *const *V, int axis,
                   he_ct *const *VT, he_refresh_state *rs) {
    if (!ctx || !cov || !lambda || !V || !VT || !rs || k < 1 || !pow2(n) || (axis != 0 && axis != 1)) {
        set_error("bad arguments");
        return HE_ERR_ARG;
    }
    Ctx &c = ctx->c;
    PCA_GUARD_BEGIN
    RefreshState st{rs->next_obj, rs->count};
    PcaOps ops(&c, &st);
    std::vector<HC> out = ops.eigen_shift(cov, k, lambda, V, axis, VT);
    if (int rc = sync_status(c)) return rc;
    for (int i = 0; i < k * k; i++) {
        free_ct(cov[i]);
        cov[i] = out[i].release();
    }
    rs->next_obj = st.next_obj;
    rs->count = st.count;
    return HE_OK;
    PCA_GUARD_END
}

}  // extern "C"
