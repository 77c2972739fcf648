// context.cu -- parameters, tables, keys, encryption and ciphertext I/O.
#include <cmath>
#include <cstring>

#include "he_internal.h"

namespace he {

// -------------------------------------------------------------- errors
static thread_local std::string g_err;
void set_error(const std::string &msg) { g_err = msg; }

int device_status(const Ctx *c) {
    if (c && c->h_err && *(volatile int *)c->h_err) {
        *(volatile int *)c->h_err = 0;
        set_error("a device-side wait ran out of its iteration limit (kernel stopped early; outputs invalid)");
        return HE_ERR_TIMEOUT;
    }
    return HE_OK;
}
const char *last_error() { return g_err.c_str(); }

// --------------------------------------------------------- number theory
typedef unsigned __int128 u128;
u64 h_mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
u64 h_powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    for (; e; e >>= 1) {
        if (e & 1) r = h_mulmod(r, a, q);
        a = h_mulmod(a, a, q);
    }
    return r;
}
u64 h_invmod(u64 a, u64 q) { return h_powmod(a % q, q - 2, q); }
ShoupPair h_shoup(u64 w, u64 q) {
    w %= q;
    return ShoupPair{w, (u64)(((u128)w << 64) / q)};
}

// Miller-Rabin with the prime bases up to 37 (deterministic below 2^64).
static bool h_is_prime(u64 n) {
    if (n < 2) return false;
    const u64 small[] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    for (u64 p : small) {
        if (n % p == 0) return n == p;
    }
    u64 d = n - 1;
    int s = 0;
    while (!(d & 1)) { d >>= 1; s++; }
    for (u64 a : small) {
        u64 x = h_powmod(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool ok = false;
        for (int k = 1; k < s && !ok; k++) {
            x = h_mulmod(x, x, n);
            ok = (x == n - 1);
        }
        if (!ok) return false;
    }
    return true;
}

// Setparams (App. A): primes = 1 mod 2N.  q_0, then the special primes, are
// the largest ones below 2^bits in descending order; q_1..q_L alternate
// around 2^bits: first above, first below, second above, second below, ...
int h_gen_primes(int logN, int nq, const int *qbits, int np, const int *pbits, u64 *q, u64 *p) {
    const u64 M = 2ull << logN;
    std::vector<u64> taken;
    auto descending = [&](int bits) -> u64 {
        u64 lim = 1ull << bits;
        for (u64 c = (lim - 1) / M * M + 1; c > M; c -= M) {
            if (c >= lim) continue;
            bool used = false;
            for (u64 t : taken) used |= (t == c);
            if (!used && h_is_prime(c)) return c;
        }
        return 0;
    };
    q[0] = descending(qbits[0]);
    if (!q[0]) return -1;
    taken.push_back(q[0]);
    for (int j = 0; j < np; j++) {
        p[j] = descending(pbits[j]);
        if (!p[j]) return -1;
        taken.push_back(p[j]);
    }
    for (int i = 1; i < nq; i++) {
        int bits = qbits[i];
        int k = 0;
        for (int j = 1; j < i; j++) k += (qbits[j] == bits);
        u64 centre = 1ull << bits;
        int target = k / 2, seen = -1;
        u64 c;
        if (k % 2 == 0) {
            c = (centre + M - 1) / M * M + 1;
            while (true) {
                if (h_is_prime(c) && ++seen == target) break;
                c += M;
            }
        } else {
            c = (centre - 1) / M * M + 1;
            while (true) {
                if (c <= M) return -1;
                if (h_is_prime(c) && ++seen == target) break;
                c -= M;
            }
        }
        for (u64 t : taken)
            if (t == c) return -1;
        taken.push_back(c);
        q[i] = c;
    }
    return 0;
}

static u64 find_root_2n(u64 q, int N) {
    for (u64 g = 2;; g++) {
        u64 r = h_powmod(g, (q - 1) / (2ull * N), q);
        if (h_powmod(r, (u64)N, q) == q - 1) return r;
    }
}

static int bitrev(int x, int bits) {
    int r = 0;
    for (int i = 0; i < bits; i++) r |= ((x >> i) & 1) << (bits - 1 - i);
    return r;
}

static ModQ make_mod(u64 q) {
    ModQ m;
    m.q = q;
    u64 x = 1;
    for (int i = 0; i < 7; i++) x *= 2 - q * x;  // q^-1 mod 2^64 (Newton)
    m.qinv = (u64)0 - x;
    u64 R = (u64)(((u128)1 << 64) % q);
    m.r2 = h_mulmod(R, R, q);
    m.twoq = 2 * q;
    m.wone = (u64)(((u128)1 << 64) / q);
    return m;
}

// ---------------------------------------------------------------- pool
void DevicePool::set_redirect(DevicePool *r) {
    std::lock_guard<std::mutex> lk(mu_);
    redirect_ = r;
}

bool DevicePool::owns(void *p) {
    std::lock_guard<std::mutex> lk(mu_);
    return sizes_.count(p) != 0;
}

void *DevicePool::get(size_t bytes) {
    DevicePool *r;
    {
        std::lock_guard<std::mutex> lk(mu_);
        r = redirect_;
    }
    if (r) return r->get(bytes);
    std::lock_guard<std::mutex> lk(mu_);
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    auto it = free_.lower_bound(bytes);
    if (it != free_.end() && it->first <= bytes + bytes / 4) {
        void *p = it->second;
        size_t sz = it->first;
        free_.erase(it);
        cached_ -= sz;
        in_use_ += sz;
        if (in_use_ > peak_) peak_ = in_use_;
        return p;
    }
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        // give cached blocks back and retry once
        cudaDeviceSynchronize();
        for (auto &kv : free_) cudaFree(kv.second), sizes_.erase(kv.second);
        free_.clear();
        cached_ = 0;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            throw std::bad_alloc();
        }
    }
    sizes_[p] = bytes;
    in_use_ += bytes;
    if (in_use_ > peak_) peak_ = in_use_;
    return p;
}

void DevicePool::put(void *p) {
    if (!p) return;
    DevicePool *r;
    {
        std::lock_guard<std::mutex> lk(mu_);
        r = redirect_;
    }
    if (r && r->owns(p)) {
        r->put(p);
        return;
    }
    std::lock_guard<std::mutex> lk(mu_);
    size_t sz = sizes_[p];
    in_use_ -= sz;
    cached_ += sz;
    free_.insert({sz, p});
}

void DevicePool::release_all() {
    std::lock_guard<std::mutex> lk(mu_);
    if (sizes_.empty()) return;
    cudaDeviceSynchronize();
    for (auto &kv : sizes_) cudaFree(kv.first);
    sizes_.clear();
    free_.clear();
    in_use_ = cached_ = 0;
}

// --------------------------------------------------------------- tracing
cudaEvent_t Ctx::ev_get() {
    if (!ev_free.empty()) {
        cudaEvent_t e = ev_free.back();
        ev_free.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

void Ctx::trace_begin(int cls, cudaEvent_t &e0) {
    (void)cls;
    e0 = nullptr;
    if (!trace) return;
    e0 = ev_get();
    cudaEventRecord(e0, stream);
}

void Ctx::trace_end(int cls, cudaEvent_t e0, double bytes, double ops) {
    if (!trace || !e0) return;
    cudaEvent_t e1 = ev_get();
    cudaEventRecord(e1, stream);
    tr[cls].pending.push_back({e0, e1});
    tr[cls].bytes += bytes;
    tr[cls].ops += ops;
    tr[cls].count++;
}

void Ctx::trace_collect() {
    cudaStreamSynchronize(stream);
    for (auto &c : tr) {
        for (auto &pr : c.pending) {
            float ms = 0;
            cudaEventElapsedTime(&ms, pr.first, pr.second);
            c.total_ms += ms;
            ev_free.push_back(pr.first);
            ev_free.push_back(pr.second);
        }
        c.pending.clear();
    }
}

// -------------------------------------------------------------- tables
template <typename T>
static T *upload(const std::vector<T> &v) {
    T *d = nullptr;
    if (v.empty()) return nullptr;
    if (cudaMalloc(&d, v.size() * sizeof(T)) != cudaSuccess) throw std::bad_alloc();
    cudaMemcpy(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return d;
}

const LevelConsts &Ctx::lc(int level) {
    LevelConsts &LC = lvl[level];
    if (LC.level == level) return LC;
    LC.level = level;
    LC.ndig = ndig(level);
    int rows = level + 1 + alpha;
    std::vector<ShoupPair> inv((size_t)LC.ndig * alpha), mod((size_t)LC.ndig * alpha * rows);
    for (int d = 0; d < LC.ndig; d++) {
        int i0 = d * alpha, ns = std::min(alpha, level + 1 - i0);
        for (int s = 0; s < ns; s++) {
            u64 qi = primes[i0 + s];
            u64 prod = 1;  // Q_d / q_i mod q_i
            for (int t = 0; t < ns; t++)
                if (t != s) prod = h_mulmod(prod, primes[i0 + t] % qi, qi);
            inv[d * alpha + s] = h_shoup(h_invmod(prod, qi), qi);
            for (int r = 0; r < rows; r++) {
                u64 pr = r <= level ? primes[r] : primes[L + 1 + (r - level - 1)];
                u64 v = 1;
                for (int t = 0; t < ns; t++)
                    if (t != s) v = h_mulmod(v, primes[i0 + t] % pr, pr);
                mod[((size_t)d * alpha + s) * rows + r] = h_shoup(v, pr);
            }
        }
    }
    LC.d_up_inv = upload(inv);
    LC.d_up_mod = upload(mod);
    if (level > 0) {
        std::vector<ShoupPair> ri(level);
        std::vector<u64> rm(level);
        u64 ql = primes[level];
        for (int i = 0; i < level; i++) {
            ri[i] = h_shoup(h_invmod(ql % primes[i], primes[i]), primes[i]);
            rm[i] = ql % primes[i];
        }
        LC.d_rs_inv = upload(ri);
        LC.d_rs_qlmod = upload(rm);
    }
    return LC;
}

void build_tables(Ctx *c) {
    int N = c->N, logN = c->logN;
    std::vector<u64> psi((size_t)c->nprimes * N), psip(psi.size()), ipsi(psi.size()), ipsip(psi.size());
    std::vector<u64> ninv(2 * (size_t)c->nprimes);
    std::vector<u64> pw(N), ipw(N);
    for (int k = 0; k < c->nprimes; k++) {
        u64 q = c->primes[k];
        u64 r = find_root_2n(q, N), ri = h_invmod(r, q);
        pw[0] = ipw[0] = 1;
        for (int i = 1; i < N; i++) {
            pw[i] = h_mulmod(pw[i - 1], r, q);
            ipw[i] = h_mulmod(ipw[i - 1], ri, q);
        }
        for (int i = 0; i < N; i++) {
            int br = bitrev(i, logN);
            ShoupPair a = h_shoup(pw[br], q), b = h_shoup(ipw[br], q);
            psi[(size_t)k * N + i] = a.w;
            psip[(size_t)k * N + i] = a.wp;
            ipsi[(size_t)k * N + i] = b.w;
            ipsip[(size_t)k * N + i] = b.wp;
        }
        ShoupPair ni = h_shoup(h_invmod((u64)N, q), q);
        ninv[2 * k] = ni.w;
        ninv[2 * k + 1] = ni.wp;
    }
    c->d_psi = upload(psi);
    c->d_psip = upload(psip);
    c->d_ipsi = upload(ipsi);
    c->d_ipsip = upload(ipsip);
    {
        std::vector<u64> t2(2 * psi.size()), it2(2 * psi.size());
        for (size_t i = 0; i < psi.size(); i++) {
            t2[2 * i] = psi[i], t2[2 * i + 1] = psip[i];
            it2[2 * i] = ipsi[i], it2[2 * i + 1] = ipsip[i];
        }
        c->d_psi2 = upload(t2);
        c->d_ipsi2 = upload(it2);
    }
    c->d_ninv = upload(ninv);
    c->hmod.resize(c->nprimes);
    for (int k = 0; k < c->nprimes; k++) c->hmod[k] = make_mod(c->primes[k]);
    c->d_mod = upload(c->hmod);

    // ModDown / lift constants
    int L = c->L, a = c->alpha;
    std::vector<ShoupPair> pinv(a), pmod((size_t)a * (L + 1)), Pinv(L + 1), Pmod(L + 1);
    for (int j = 0; j < a; j++) {
        u64 pj = c->primes[L + 1 + j];
        u64 prod = 1;
        for (int t = 0; t < a; t++)
            if (t != j) prod = h_mulmod(prod, c->primes[L + 1 + t] % pj, pj);
        pinv[j] = h_shoup(h_invmod(prod, pj), pj);
        for (int r = 0; r <= L; r++) {
            u64 qr = c->primes[r], v = 1;
            for (int t = 0; t < a; t++)
                if (t != j) v = h_mulmod(v, c->primes[L + 1 + t] % qr, qr);
            pmod[(size_t)j * (L + 1) + r] = h_shoup(v, qr);
        }
    }
    for (int r = 0; r <= L; r++) {
        u64 qr = c->primes[r], v = 1;
        for (int t = 0; t < a; t++) v = h_mulmod(v, c->primes[L + 1 + t] % qr, qr);
        Pmod[r] = h_shoup(v, qr);
        Pinv[r] = h_shoup(h_invmod(v, qr), qr);
    }
    c->d_dn_pinv = upload(pinv);
    c->d_dn_pmod = upload(pmod);
    c->d_dn_Pinv = upload(Pinv);
    c->d_Pmod = upload(Pmod);
    // h = (P-1)/2 reduced mod every prime: 2h = P - 1 exactly (P odd)
    MdExact &mk = c->md_exact;
    mk = MdExact();
    for (int j = 0; j < a; j++) {
        u64 pj = c->primes[L + 1 + j], Pm = 1;
        for (int t = 0; t < a; t++) Pm = h_mulmod(Pm, c->primes[L + 1 + t] % pj, pj);
        mk.p[j] = pj;
        mk.hp[j] = h_mulmod((Pm + pj - 1) % pj, h_invmod(2, pj), pj);
        mk.pinv[j] = pinv[j];
    }
    // P/p_j and k P as 64-bit limbs (P < 2^(62 alpha))
    auto limb_mul = [](u64 *x, int n, u64 m) {
        unsigned __int128 carry = 0;
        for (int i = 0; i < n; i++) {
            unsigned __int128 t = (unsigned __int128)x[i] * m + carry;
            x[i] = (u64)t;
            carry = t >> 64;
        }
    };
    u64 P4[4] = {1, 0, 0, 0};
    for (int t = 0; t < a; t++) limb_mul(P4, 4, c->primes[L + 1 + t]);
    for (int j = 0; j < a; j++) {
        u64 ph[4] = {1, 0, 0, 0};
        for (int t = 0; t < a; t++)
            if (t != j) limb_mul(ph, 4, c->primes[L + 1 + t]);
        for (int i = 0; i < 3; i++) mk.phat[j][i] = ph[i];
    }
    for (int m = 0; m + 1 < a; m++) {
        for (int i = 0; i < 4; i++) mk.kP[m][i] = P4[i];
        limb_mul(mk.kP[m], 4, (u64)(m + 1));
    }
    std::vector<u64> E((size_t)a * (L + 1));
    for (int r = 0; r <= L; r++) {
        u64 qr = c->primes[r];
        const u64 hq = h_mulmod((Pmod[r].w + qr - 1) % qr, h_invmod(2, qr), qr);
        for (int e = 0; e < a; e++) {
            const u64 t = (h_mulmod((u64)e, Pmod[r].w, qr) + hq) % qr;
            E[(size_t)e * (L + 1) + r] = t ? qr - t : 0;
        }
    }
    c->d_dn_E = upload(E);
    c->lvl.assign(L + 1, LevelConsts());

    // encoder: zeta^e = (cos, sin)((pi e) / N); slot j -> t = (5^j mod 2N - 1)/4
    std::vector<double> z(4 * (size_t)N);
    for (int e = 0; e < 2 * N; e++) {
        double ang = (M_PI * (double)e) / (double)N;
        z[2 * e] = cos(ang);
        z[2 * e + 1] = sin(ang);
    }
    c->d_zeta = upload(z);
    std::vector<int> st(c->S);
    u64 g = 1, M = 2ull * N;
    for (int j = 0; j < c->S; j++) {
        st[j] = (int)((g - 1) / 4);
        g = (g * 5) % M;
    }
    c->d_slot_t = upload(st);

    // discrete Gaussian cumulative table T[k] = floor(2^63 P(|x| <= k)), |x| <= 19
    double sigma = c->prm.sigma;
    double denom = (2.0 * sigma) * sigma;
    double rho[20];
    for (int v = 0; v < 20; v++) rho[v] = exp(-((double)(v * v)) / denom);
    double total = rho[0];
    for (int v = 1; v < 20; v++) total += 2.0 * rho[v];
    double cum = rho[0];
    for (int k = 0; k < 19; k++) {
        if (k > 0) cum += 2.0 * rho[k];
        c->gauss_T[k] = (u64)floor((cum / total) * 9223372036854775808.0);
    }
    c->gauss_T[19] = 1ull << 63;
}

// --------------------------------------------------------------- keygen
// purpose tags of the Philox counter (i, limb, object, tag)
enum { TAG_SK = 1, TAG_PK_A = 2, TAG_PK_E = 3, TAG_ENC_V = 4, TAG_ENC_E0 = 5, TAG_ENC_E1 = 6, TAG_REF_V = 7,
       TAG_REF_E0 = 8, TAG_REF_E1 = 9, TAG_SWK_A = 0x100, TAG_SWK_E = 0x200 };

static RowMap map_all(const Ctx *c) {
    RowMap m;
    m.n = c->nprimes, m.lq = c->nprimes - 1;   // every prime, in global order
    return m;
}

// small signed polynomial -> NTT-domain residues over the rows of rm
static void small_ntt(Ctx *c, i64 *tmp_small, u64 *out, int rows, const RowMap &rm, int kind, uint32_t obj,
                      uint32_t tag) {
    launch_sample_small(c, tmp_small, kind, obj, tag, c->stream);
    launch_small_to_rns(c, tmp_small, out, rows, rm, c->stream);
    ntt_fwd(c, out, rows, rm, c->stream);
}

void create_keys(Ctx *c) {
    int N = c->N, np = c->nprimes, L = c->L;
    RowMap all = map_all(c);
    Buf small(&c->pool, N);
    i64 *sm = (i64 *)small.p;
    cudaMalloc(&c->d_sk, (size_t)np * N * 8);
    cudaMalloc(&c->d_skM, (size_t)np * N * 8);
    small_ntt(c, sm, c->d_sk, np, all, 0, 0, TAG_SK);
    launch_to_mont(c, c->d_skM, c->d_sk, np, all, c->stream);
    // pk = (-a s + e, a) over Q_L
    RowMap mq = c->map_q(L);
    Buf a(&c->pool, (size_t)(L + 1) * N), e(&c->pool, (size_t)(L + 1) * N);
    launch_sample_uniform(c, a.p, L + 1, mq, nullptr, 0, TAG_PK_A, c->stream);
    ntt_fwd(c, a.p, L + 1, mq, c->stream);
    small_ntt(c, sm, e.p, L + 1, mq, 1, 0, TAG_PK_E);
    cudaMalloc(&c->d_pkM, (size_t)2 * (L + 1) * N * 8);
    u64 *pk0 = c->d_pkM, *pk1 = c->d_pkM + (size_t)(L + 1) * N;
    launch_mulM(c, pk0, a.p, c->d_skM, L + 1, mq, c->stream);   // a s
    launch_sub(c, pk0, e.p, pk0, L + 1, mq, c->stream);         // e - a s
    launch_to_mont(c, pk0, pk0, L + 1, mq, c->stream);
    launch_to_mont(c, pk1, a.p, L + 1, mq, c->stream);
}

// SwitchKeyGen (App. A, reading of the hybrid gadget): for each digit d,
// (-a_d s + e_d + P B_d s', a_d) over Q_L P; P B_d s' is (P mod q_i) s' on the
// q's of digit d and 0 elsewhere.  sprime: NTT domain over all primes.
static u64 *gen_swk(Ctx *c, const u64 *sprime, uint32_t obj) {
    int N = c->N, np = c->nprimes;
    RowMap all = map_all(c);
    u64 *key = nullptr;
    if (cudaMalloc(&key, c->key_words() * 8) != cudaSuccess) throw std::bad_alloc();
    Buf small(&c->pool, N), e(&c->pool, (size_t)np * N), t(&c->pool, N);
    i64 *sm = (i64 *)small.p;
    std::vector<ShoupPair> hp(c->L + 1);
    for (int d = 0; d < c->dnum; d++) {
        u64 *k0 = key + (size_t)(d * 2 + 0) * np * N;
        u64 *k1 = key + (size_t)(d * 2 + 1) * np * N;
        launch_sample_uniform(c, k1, np, all, nullptr, obj, TAG_SWK_A + d, c->stream);
        ntt_fwd(c, k1, np, all, c->stream);
        small_ntt(c, sm, e.p, np, all, 1, obj, TAG_SWK_E + d);
        launch_mulM(c, k0, k1, c->d_skM, np, all, c->stream);  // a s
        launch_sub(c, k0, e.p, k0, np, all, c->stream);          // e - a s
        for (int i = d * c->alpha; i < std::min((d + 1) * c->alpha, c->L + 1); i++) {
            RowMap one = RowMap::single(i);
            // t = (P mod q_i) s'_i ; k0_i += t
            launch_mulconst_rows(c, t.p, sprime + (size_t)i * N, c->d_Pmod + i, 1, 1, one, c->stream);
            launch_add(c, k0 + (size_t)i * N, k0 + (size_t)i * N, t.p, 1, one, c->stream);
        }
        launch_to_mont(c, k0, k0, np, all, c->stream);
        launch_to_mont(c, k1, k1, np, all, c->stream);
    }
    return key;
}

// The key of kappa_g, stored in the permuted layout MultSum reads (every row
// r of the key at index pi_g(x) holds the switching key's word x).
u64 *gen_rotation_key(Ctx *c, uint32_t g) {
    RowMap all = map_all(c);
    Buf sp(&c->pool, (size_t)c->nprimes * c->N);
    launch_automorph(c, sp.p, c->d_sk, c->nprimes, all, g, c->stream);   // kappa_g(s)
    u64 *key = gen_swk(c, sp.p, g);
    const long rows = (long)c->dnum * 2 * c->nprimes;
    Buf tmp(&c->pool, (size_t)rows * c->N);
    cudaMemcpyAsync(tmp.p, key, (size_t)rows * c->N * 8, cudaMemcpyDeviceToDevice, c->stream);
    launch_permute_key(c, key, tmp.p, rows, g, c->stream);
    return key;
}

u64 *gen_relin_key(Ctx *c) {
    RowMap all = map_all(c);
    Buf s2(&c->pool, (size_t)c->nprimes * c->N);
    launch_mulM(c, s2.p, c->d_sk, c->d_skM, c->nprimes, all, c->stream);  // s^2
    return gen_swk(c, s2.p, 0);
}

uint32_t galois_of_step(const Ctx *c, long step) {
    long S = c->S;
    long k = ((step % S) + S) % S;
    return (uint32_t)h_powmod(5, (u64)k, 2ull * c->N);
}

// ------------------------------------------------------- encrypt/decrypt
void encrypt_poly(Ctx *c, const u64 *m_ntt, int level, uint32_t obj, bool refresh, u64 *out) {
    int N = c->N;
    RowMap mq = c->map_q(level);
    int rows = level + 1;
    Buf small(&c->pool, N), v(&c->pool, (size_t)rows * N), e(&c->pool, (size_t)rows * N);
    i64 *sm = (i64 *)small.p;
    u64 *c0 = out, *c1 = out + (size_t)rows * N;
    const u64 *pk0 = c->d_pkM, *pk1 = c->d_pkM + (size_t)(c->L + 1) * N;
    small_ntt(c, sm, v.p, rows, mq, 0, obj, refresh ? TAG_REF_V : TAG_ENC_V);
    launch_mulM(c, c0, v.p, pk0, rows, mq, c->stream);
    launch_mulM(c, c1, v.p, pk1, rows, mq, c->stream);
    small_ntt(c, sm, e.p, rows, mq, 1, obj, refresh ? TAG_REF_E0 : TAG_ENC_E0);
    launch_add(c, c0, c0, e.p, rows, mq, c->stream);
    launch_add(c, c0, c0, m_ntt, rows, mq, c->stream);
    small_ntt(c, sm, e.p, rows, mq, 1, obj, refresh ? TAG_REF_E1 : TAG_ENC_E1);
    launch_add(c, c1, c1, e.p, rows, mq, c->stream);
}

// Encode z (device, S real values) at `scale` into NTT-domain residues over rm.
void encode_to(Ctx *c, const double *d_zr, const double *d_zi, double scale, u64 *out, int rows, const RowMap &rm) {
    Buf m(&c->pool, c->N);
    launch_encode(c, d_zr, d_zi, scale, (i64 *)m.p, c->stream);
    launch_small_to_rns(c, (const i64 *)m.p, out, rows, rm, c->stream);
    ntt_fwd(c, out, rows, rm, c->stream);
}

}  // namespace he
