// capi.cu -- the extern "C" boundary declared in include/he.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <set>
#include <tuple>

#include "ctapi.h"

using namespace he;

namespace he {
void build_tables(Ctx *c);
}

// --------------------------------------------------------------- helpers
#define GUARD_BEGIN try {
#define GUARD_END                                                      \
    }                                                                  \
    catch (const HeError &e) {                                         \
        set_error(e.what());                                           \
        return e.code;                                                 \
    }                                                                  \
    catch (const std::bad_alloc &) {                                   \
        set_error("device or host allocation failed");                 \
        return HE_ERR_OOM;                                             \
    }                                                                  \
    catch (const std::exception &e) {                                  \
        set_error(e.what());                                           \
        return HE_ERR_ARG;                                             \
    }

static int fail(int code, const char *msg) {
    set_error(msg);
    return code;
}

static int cuda_status(Ctx *c) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("CUDA error: ") + cudaGetErrorString(e));
        return HE_ERR_CUDA;
    }
    (void)c;
    return HE_OK;
}

namespace he {
size_t ct_words(const Ctx *c, int level) { return (size_t)2 * (level + 1) * c->N; }

he_ct *new_ct(Ctx *c, int level, double scale, int period) {
    he_ct *ct = new he_ct;
    ct->ctx = c;
    ct->level = level;
    ct->scale = scale;
    ct->period = period;
    ct->d = (u64 *)c->pool.get(ct_words(c, level) * 8);
    return ct;
}

void free_ct(he_ct *ct) {
    if (!ct) return;
    if (ct->d) ct->ctx->pool.put(ct->d);
    delete ct;
}

static void add_mod(std::set<long> &s, long v, long m) { s.insert(((v % m) + m) % m); }

// Table 1 "Optimized" key set of the product: replication steps -n^2 2^j,
// Z babies j and giants n1z*i (-n2z <= i < n2z), T babies n*j and giants
// n*n1t*i, and the C^k / R^k source steps n1z, -n and n*n1t.
std::vector<long> matmul_steps(int n, int n1z, int n1t, long slots, int dcd_z, int dcd_t) {
    long n2 = (long)n * n;
    std::set<long> st;
    for (long r = n2; r < slots; r *= 2) add_mod(st, -r, slots);
    int n2z = n / n1z, n2t = n / n1t;
    for (int j = 1; j < n1z; j++) add_mod(st, j, n2);   // Z babies, also the C^k babies
    if (dcd_z) {
        // Z_1 left giants 0 < i < n2', Z_2 left giants -n2' <= i < 0, right factors +-n'
        const int p2 = dcd_z / n1z;
        for (int i = -p2; i < p2; i++)
            if (i) add_mod(st, (long)n1z * i, n2);
        add_mod(st, dcd_z, n2);
        add_mod(st, -dcd_z, n2);
    } else {
        for (int i = -n2z; i < n2z; i++)
            if (i) add_mod(st, (long)n1z * i, n2);
    }
    for (int j = 1; j < n1t; j++) add_mod(st, (long)n * j, n2);   // T babies, also the R^k babies
    if (dcd_t) {
        // T left giants n n1t i, 0 < i <= n2' (the last one is the right factors' step n' n)
        const int p2 = dcd_t / n1t;
        for (int i = 1; i <= p2; i++) add_mod(st, (long)n * n1t * i, n2);
    } else {
        for (int i = 1; i < n2t; i++) add_mod(st, (long)n * n1t * i, n2);
    }
    add_mod(st, n1z, n2);
    add_mod(st, -n, n2);
    if (n2t > 1) add_mod(st, (long)n * n1t, n2);
    st.erase(0);
    return std::vector<long>(st.begin(), st.end());
}

// G (transpose) over the diagonals (n-1)k: babies (n-1)j, giants (n-1)n1 i.
std::vector<long> transpose_steps(int n, int n1, long slots) {
    long n2 = (long)n * n, a = n - 1;
    std::set<long> st;
    for (long r = n2; r < slots; r *= 2) add_mod(st, -r, slots);
    int n2g = n / n1;
    for (int j = 1; j < n1; j++) add_mod(st, a * j, n2);
    for (int i = -n2g; i < n2g; i++)
        if (i) add_mod(st, a * n1 * i, n2);
    st.erase(0);
    return std::vector<long>(st.begin(), st.end());
}

long first_missing_key(const Ctx *c, const std::vector<long> &steps, long skip_from) {
    for (long v : steps) {
        if (v >= skip_from) continue;
        if (!c->rtk.count(galois_of_step(c, v))) return v;
    }
    return 0;
}
}  // namespace he

extern "C" {

const char *he_last_error(void) { return last_error(); }

int he_params_default(int cfg_id, he_params *out) {
    if (!out) return fail(HE_ERR_ARG, "null output");
    std::memset(out, 0, sizeof(*out));
    out->log_delta = 40;
    out->sigma = 3.2;
    out->q_bits[0] = 60;
    switch (cfg_id) {
    case 1:
        out->logN = 14; out->n_q = 4; out->n_p = 1; out->p_bits[0] = 60;
        break;
    case 2: case 4:
        out->logN = cfg_id == 2 ? 16 : 15; out->n_q = 21; out->n_p = 2;
        out->p_bits[0] = out->p_bits[1] = 60;
        break;
    case 3:
        out->logN = 16; out->n_q = 14; out->n_p = 2; out->p_bits[0] = out->p_bits[1] = 60;
        break;
    default:
        return fail(HE_ERR_PARAM, "unknown preset");
    }
    for (int i = 1; i < out->n_q; i++) out->q_bits[i] = 40;
    return HE_OK;
}

int he_ctx_create(const he_params *prm, uint64_t seed, he_ctx **out) {
    if (!prm || !out) return fail(HE_ERR_ARG, "null argument");
    if (prm->logN < 10 || prm->logN > 17) return fail(HE_ERR_PARAM, "logN must be in [10, 17]");
    if (prm->n_q < 1 || prm->n_q > 48 || prm->n_p < 1 || prm->n_p > 4)
        return fail(HE_ERR_PARAM, "n_q in [1,48], n_p in [1,4]");
    if (prm->n_q + prm->n_p > 52) return fail(HE_ERR_PARAM, "too many primes");
    for (int i = 0; i < prm->n_q; i++)
        if (prm->q_bits[i] < 30 || prm->q_bits[i] > 60) return fail(HE_ERR_PARAM, "q bits in [30, 60]");
    for (int j = 0; j < prm->n_p; j++)
        if (prm->p_bits[j] < 30 || prm->p_bits[j] > 60) return fail(HE_ERR_PARAM, "p bits in [30, 60]");
    if (prm->sigma <= 0 || prm->log_delta < 1 || prm->log_delta > 60) return fail(HE_ERR_PARAM, "sigma / log_delta");
    GUARD_BEGIN
    he_ctx *h = new he_ctx;
    Ctx &c = h->c;
    c.prm = *prm;
    c.logN = prm->logN;
    c.N = 1 << c.logN;
    c.S = c.N / 2;
    c.L = prm->n_q - 1;
    c.alpha = prm->n_p;
    c.dnum = (c.L + 1 + c.alpha - 1) / c.alpha;
    c.nprimes = prm->n_q + prm->n_p;
    c.seed = seed;
    std::vector<u64> q(prm->n_q), p(prm->n_p);
    if (h_gen_primes(c.logN, prm->n_q, prm->q_bits, prm->n_p, prm->p_bits, q.data(), p.data()) != 0) {
        delete h;
        return fail(HE_ERR_PARAM, "prime search failed");
    }
    c.primes = q;
    c.primes.insert(c.primes.end(), p.begin(), p.end());
    cudaGetDevice(&c.device);
    if (cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete h;
        return fail(HE_ERR_CUDA, "stream creation failed");
    }
    c.own_stream = true;
    if (cudaHostAlloc((void **)&c.h_err, sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void **)&c.d_err, c.h_err, 0) != cudaSuccess) {
        cudaGetLastError();
        if (c.h_err) cudaFreeHost(c.h_err);
        cudaStreamDestroy(c.stream);
        delete h;
        return fail(HE_ERR_CUDA, "mapped host flag allocation failed");
    }
    *c.h_err = 0;
    build_tables(&c);
    create_keys(&c);
    if (cudaStreamSynchronize(c.stream) != cudaSuccess) {
        int rc = cuda_status(&c);
        delete h;
        return rc ? rc : HE_ERR_CUDA;
    }
    int rc = cuda_status(&c);
    if (rc) {
        delete h;
        return rc;
    }
    *out = h;
    return HE_OK;
    GUARD_END
}

int he_ctx_destroy(he_ctx *ctx) {
    if (!ctx) return HE_OK;
    Ctx &c = ctx->c;
    cudaStreamSynchronize(c.stream);
    for (auto &kv : c.rtk) cudaFree(kv.second);
    if (c.rlk) cudaFree(c.rlk);
    for (auto &kv : c.ptcache) cudaFree(kv.second);
    for (auto &kv : c.dcd)
        for (auto &f : kv.second.factors) cudaFree(f.dev);
    void *ptrs[] = {c.d_mod, c.d_psi, c.d_psip, c.d_ipsi, c.d_ipsip, c.d_psi2, c.d_ipsi2, c.d_ninv, c.d_dn_pinv,
                    c.d_dn_pmod,
                    c.d_dn_Pinv, c.d_Pmod, c.d_dn_E, c.d_zeta, c.d_slot_t, c.d_sk, c.d_skM,
                    c.d_pkM};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (auto &l : c.lvl) {
        if (l.d_up_inv) cudaFree(l.d_up_inv);
        if (l.d_up_mod) cudaFree(l.d_up_mod);
        if (l.d_rs_inv) cudaFree(l.d_rs_inv);
        if (l.d_rs_qlmod) cudaFree(l.d_rs_qlmod);
    }
    c.pool.release_all();
    if (c.h_err) cudaFreeHost(c.h_err);
    if (c.own_stream) cudaStreamDestroy(c.stream);
    delete ctx;
    return HE_OK;
}

int he_ctx_set_stream(he_ctx *ctx, void *stream) {
    if (!ctx) return fail(HE_ERR_ARG, "null context");
    Ctx &c = ctx->c;
    cudaStreamSynchronize(c.stream);
    if (stream) {
        if (c.own_stream) cudaStreamDestroy(c.stream);
        c.own_stream = false;
        c.stream = (cudaStream_t)stream;
    } else if (!c.own_stream) {
        cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking);
        c.own_stream = true;
    }
    return HE_OK;
}

int he_ctx_set_autotune(he_ctx *ctx, int on) {
    if (!ctx) return fail(HE_ERR_ARG, "null context");
    ctx->c.autotune = on != 0;
    return HE_OK;
}

int he_ctx_set_multsum_variant(he_ctx *ctx, int variant) {
    if (!ctx) return fail(HE_ERR_ARG, "null context");
    if (variant < -1 ||
        (variant > 10 && variant != 16 && variant != 20 && variant != 32 && variant != 36 && variant != 48 &&
         variant != 64 && variant != 65 && variant != 80 && variant != 84 && variant != 96 && variant != 97))
        return fail(HE_ERR_ARG, "MultSum variant -1..10, 16, 20, 32, 36, 48, 64, 65, 80, 84, 96 or 97");
    ctx->c.force_multsum = variant;
    return HE_OK;
}

int he_ctx_set_ntt_variant(he_ctx *ctx, int variant) {
    if (!ctx) return fail(HE_ERR_ARG, "null context");
    if (variant != -1 && (variant < 2 || variant > 6)) return fail(HE_ERR_ARG, "NTT variant -1 or 2..6");
    Ctx &c = ctx->c;
    cudaStreamSynchronize(c.stream);
    if (variant < 0) {
        c.ntt_tuned = false;   // the tuner picks again at the next transform
        c.ntt_minb = c.ntt_minb_inv = 2;
    } else {
        c.ntt_tuned = true;
        c.ntt_minb = variant == 6 && c.logN != 16 ? 3 : variant;   // the cluster pass is for N = 2^16
        c.ntt_minb_inv = variant == 4 || variant == 6 ? 3 : variant;   // forward-only variants
    }
    return HE_OK;
}

int he_ctx_set_ntt_chunk(he_ctx *ctx, int rows) {
    if (!ctx) return fail(HE_ERR_ARG, "null context");
    if (rows < 0) return fail(HE_ERR_ARG, "rows per launch must be >= 0");
    Ctx &c = ctx->c;
    cudaStreamSynchronize(c.stream);
    c.ntt_chunk = c.ntt_chunk_inv = rows;
    return HE_OK;
}

int he_ctx_set_newton_composition(he_ctx *ctx, int on) {
    if (!ctx) return fail(HE_ERR_ARG, "null context");
    ctx->c.newton_compose = on != 0;
    return HE_OK;
}

int he_ctx_set_packed_refresh(he_ctx *ctx, int on) {
    if (!ctx) return fail(HE_ERR_ARG, "null context");
    ctx->c.pack_refresh = on != 0;
    return HE_OK;
}

int he_autotune_log(const he_ctx *ctx, char *out, int cap, int *len) {
    if (!ctx || (cap > 0 && !out)) return fail(HE_ERR_ARG, "bad arguments");
    const std::string &s = ctx->c.tune_log;
    if (len) *len = (int)s.size();
    if (cap > 0) {
        size_t n = std::min(s.size(), (size_t)cap - 1);
        std::memcpy(out, s.data(), n);
        out[n] = 0;
    }
    return HE_OK;
}

int he_ctx_primes(const he_ctx *ctx, uint64_t *q_out, uint64_t *p_out) {
    if (!ctx) return fail(HE_ERR_ARG, "null context");
    const Ctx &c = ctx->c;
    for (int i = 0; i <= c.L; i++)
        if (q_out) q_out[i] = c.primes[i];
    for (int j = 0; j < c.alpha; j++)
        if (p_out) p_out[j] = c.primes[c.L + 1 + j];
    return HE_OK;
}

int he_ctx_info(const he_ctx *ctx, int *N, int *slots, int *L, int *alpha, int *dnum) {
    if (!ctx) return fail(HE_ERR_ARG, "null context");
    const Ctx &c = ctx->c;
    if (N) *N = c.N;
    if (slots) *slots = c.S;
    if (L) *L = c.L;
    if (alpha) *alpha = c.alpha;
    if (dnum) *dnum = c.dnum;
    return HE_OK;
}

int he_sk_export(const he_ctx *ctx, int64_t *s_out) {
    if (!ctx || !s_out) return fail(HE_ERR_ARG, "null argument");
    const Ctx &c = ctx->c;
    GUARD_BEGIN
    Ctx &cc = const_cast<Ctx &>(c);
    Buf t(&cc.pool, c.N);
    HE_CUDA_CHECK(cudaMemcpyAsync(t.p, c.d_sk, (size_t)c.N * 8, cudaMemcpyDeviceToDevice, c.stream));
    RowMap one = RowMap::single(0);
    ntt_inv(&cc, t.p, 1, one, c.stream);
    std::vector<u64> h(c.N);
    HE_CUDA_CHECK(cudaMemcpyAsync(h.data(), t.p, (size_t)c.N * 8, cudaMemcpyDeviceToHost, c.stream));
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    u64 q = c.primes[0];
    for (int i = 0; i < c.N; i++) s_out[i] = h[i] > q / 2 ? -(int64_t)(q - h[i]) : (int64_t)h[i];
    return HE_OK;
    GUARD_END
}

int he_keygen(he_ctx *ctx, const int32_t *rot_steps, int n_steps, int want_relin) {
    if (!ctx || (n_steps > 0 && !rot_steps) || n_steps < 0) return fail(HE_ERR_ARG, "bad arguments");
    Ctx &c = ctx->c;
    GUARD_BEGIN
    for (int i = 0; i < n_steps; i++) {
        long s = ((long)rot_steps[i] % c.S + c.S) % c.S;
        if (s == 0) continue;
        uint32_t g = galois_of_step(&c, s);
        if (c.rtk.count(g)) continue;
        c.rtk[g] = gen_rotation_key(&c, g);
    }
    if (want_relin && !c.rlk) c.rlk = gen_relin_key(&c);
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    return cuda_status(&c);
    GUARD_END
}

int he_rot_steps_for_matmul(int n, int n1z, int n1t, int slots, int32_t *out, int *count) {
    if (!out || !count || n < 1 || n1z < 1 || n1t < 1 || n % n1z || n % n1t || (long)n * n > slots)
        return fail(HE_ERR_ARG, "bad arguments");
    std::vector<long> st = matmul_steps(n, n1z, n1t, slots);
    for (size_t k = 0; k < st.size(); k++) out[k] = (int32_t)st[k];
    *count = (int)st.size();
    return HE_OK;
}

int he_rot_steps_for_sched(int n, const he_mm_sched *sched, int slots, int32_t *out, int *count) {
    if (!sched || !out || !count || n < 2 || sched->n1_z < 1 || sched->n1_t < 1 || n % sched->n1_z ||
        n % sched->n1_t || (long)n * n > slots)
        return fail(HE_ERR_ARG, "bad arguments");
    if ((sched->dcd_z && (sched->dcd_z >= n || sched->dcd_z % sched->n1_z)) ||
        (sched->dcd_t && (sched->dcd_t >= n || sched->dcd_t % sched->n1_t)))
        return fail(HE_ERR_ARG, "a decomposition needs n' < n with the baby steps dividing n'");
    std::vector<long> st = matmul_steps(n, sched->n1_z, sched->n1_t, slots, sched->dcd_z, sched->dcd_t);
    for (size_t k = 0; k < st.size(); k++) out[k] = (int32_t)st[k];
    *count = (int)st.size();
    return HE_OK;
}

int he_rot_steps_for_transpose(int n, int n1, int slots, int32_t *out, int *count) {
    if (!out || !count || n < 2 || n1 < 1 || n % n1 || (long)n * n > slots) return fail(HE_ERR_ARG, "bad arguments");
    std::vector<long> st = transpose_steps(n, n1, slots);
    for (size_t k = 0; k < st.size(); k++) out[k] = (int32_t)st[k];
    *count = (int)st.size();
    return HE_OK;
}

int he_encrypt_slots(he_ctx *ctx, const double *z, int nslots, int level, uint64_t enc_counter, he_ct **out) {
    if (!ctx || !out || (nslots > 0 && !z)) return fail(HE_ERR_ARG, "null argument");
    Ctx &c = ctx->c;
    if (nslots < 0 || nslots > c.S) return fail(HE_ERR_ARG, "nslots out of range");
    if (level < 0 || level > c.L) return fail(HE_ERR_LEVEL, "level out of range");
    GUARD_BEGIN
    std::vector<double> host(c.S, 0.0);
    if (nslots) std::memcpy(host.data(), z, sizeof(double) * nslots);
    Buf zr(&c.pool, c.S), zi(&c.pool, c.S), m(&c.pool, (size_t)(level + 1) * c.N);
    HE_CUDA_CHECK(cudaMemcpyAsync(zr.p, host.data(), sizeof(double) * c.S, cudaMemcpyHostToDevice, c.stream));
    HE_CUDA_CHECK(cudaMemsetAsync(zi.p, 0, sizeof(double) * c.S, c.stream));
    double delta = std::ldexp(1.0, c.prm.log_delta);
    encode_to(&c, (double *)zr.p, (double *)zi.p, delta, m.p, level + 1, c.map_q(level));
    he_ct *ct = new_ct(&c, level, delta, c.S);
    encrypt_poly(&c, m.p, level, (uint32_t)enc_counter, false, ct->d);
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    int rc = cuda_status(&c);
    if (rc) {
        free_ct(ct);
        return rc;
    }
    *out = ct;
    return HE_OK;
    GUARD_END
}

int he_encrypt_matrix(he_ctx *ctx, const double *A, int rows, int cols, int level, uint64_t enc_counter,
                      he_ct **out) {
    if (!ctx || !A || rows < 1 || cols < 1) return fail(HE_ERR_ARG, "bad arguments");
    if ((long)rows * cols > ctx->c.S) return fail(HE_ERR_ARG, "matrix larger than the slot count");
    return he_encrypt_slots(ctx, A, rows * cols, level, enc_counter, out);
}

int he_decrypt_slots(he_ctx *ctx, const he_ct *ct, double *z, int nslots) {
    if (!ctx || !ct || (nslots > 0 && !z)) return fail(HE_ERR_ARG, "null argument");
    Ctx &c = ctx->c;
    if (ct->ctx != &c) return fail(HE_ERR_ARG, "ciphertext of another context");
    if (nslots < 0 || nslots > c.S) return fail(HE_ERR_ARG, "nslots out of range");
    GUARD_BEGIN
    Buf m(&c.pool, c.N), coef(&c.pool, c.N), zr(&c.pool, c.S), zi(&c.pool, c.S);
    const u64 *c0 = ct->d, *c1 = ct->d + (size_t)(ct->level + 1) * c.N;
    launch_dec_q0(&c, c0, c1, m.p, c.stream);
    RowMap one = RowMap::single(0);
    ntt_inv(&c, m.p, 1, one, c.stream);
    launch_centre_q0(&c, m.p, (double *)coef.p, c.stream);
    launch_decode(&c, (double *)coef.p, ct->scale, (double *)zr.p, (double *)zi.p, c.stream);
    std::vector<double> host(c.S);
    HE_CUDA_CHECK(cudaMemcpyAsync(host.data(), zr.p, sizeof(double) * c.S, cudaMemcpyDeviceToHost, c.stream));
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    if (nslots) std::memcpy(z, host.data(), sizeof(double) * nslots);
    return cuda_status(&c);
    GUARD_END
}

int he_decrypt_matrix(he_ctx *ctx, const he_ct *ct, double *out, int rows, int cols) {
    if (!ctx || !out || rows < 1 || cols < 1) return fail(HE_ERR_ARG, "bad arguments");
    if ((long)rows * cols > ctx->c.S) return fail(HE_ERR_ARG, "matrix larger than the slot count");
    return he_decrypt_slots(ctx, ct, out, rows * cols);
}

int he_ct_info(const he_ct *ct, int *level, double *scale, int *period) {
    if (!ct) return fail(HE_ERR_ARG, "null ciphertext");
    if (level) *level = ct->level;
    if (scale) *scale = ct->scale;
    if (period) *period = ct->period;
    return HE_OK;
}

int he_ct_export(const he_ct *ct, uint64_t *residues) {
    if (!ct || !residues) return fail(HE_ERR_ARG, "null argument");
    Ctx &c = *ct->ctx;
    GUARD_BEGIN
    size_t w = ct_words(&c, ct->level);
    Buf t(&c.pool, w);
    HE_CUDA_CHECK(cudaMemcpyAsync(t.p, ct->d, w * 8, cudaMemcpyDeviceToDevice, c.stream));
    ntt_inv(&c, t.p, 2L * (ct->level + 1), c.map_q(ct->level), c.stream);
    HE_CUDA_CHECK(cudaMemcpyAsync(residues, t.p, w * 8, cudaMemcpyDeviceToHost, c.stream));
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    return cuda_status(&c);
    GUARD_END
}

int he_ct_import(he_ctx *ctx, const uint64_t *residues, int level, double scale, int period, he_ct **out) {
    if (!ctx || !residues || !out) return fail(HE_ERR_ARG, "null argument");
    Ctx &c = ctx->c;
    if (level < 0 || level > c.L) return fail(HE_ERR_LEVEL, "level out of range");
    GUARD_BEGIN
    he_ct *ct = new_ct(&c, level, scale, period > 0 ? period : c.S);
    size_t w = ct_words(&c, level);
    HE_CUDA_CHECK(cudaMemcpyAsync(ct->d, residues, w * 8, cudaMemcpyHostToDevice, c.stream));
    ntt_fwd(&c, ct->d, 2L * (level + 1), c.map_q(level), c.stream);
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    *out = ct;
    return cuda_status(&c);
    GUARD_END
}

int he_ct_free(he_ct *ct) {
    free_ct(ct);
    return HE_OK;
}

static int check_ct(Ctx &c, const he_ct *ct) {
    if (!ct) return fail(HE_ERR_ARG, "null ciphertext");
    if (ct->ctx != &c) return fail(HE_ERR_ARG, "ciphertext of another context");
    return HE_OK;
}

int he_rotate(he_ctx *ctx, const he_ct *ct, int step, he_ct **out) {
    if (!ctx || !out) return fail(HE_ERR_ARG, "null argument");
    Ctx &c = ctx->c;
    if (int rc = check_ct(c, ct)) return rc;
    GUARD_BEGIN
    he_ct *o = new_ct(&c, ct->level, ct->scale, ct->period);
    try {
        rotate(&c, ct->d, 1, ct->level, galois_of_step(&c, step), o->d);
    } catch (...) {
        free_ct(o);
        throw;
    }
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    *out = o;
    return cuda_status(&c);
    GUARD_END
}

int he_rotate_hoisted(he_ctx *ctx, const he_ct *const *cts, int n_cts, const int32_t *steps, int n_steps,
                      he_ct **outs) {
    if (!ctx || !cts || !steps || !outs || n_cts < 1 || n_steps < 1) return fail(HE_ERR_ARG, "bad arguments");
    Ctx &c = ctx->c;
    for (int i = 0; i < n_cts; i++)
        if (int rc = check_ct(c, cts[i])) return rc;
    for (int s = 0; s < n_steps; s++)
        if (!c.rtk.count(galois_of_step(&c, steps[s]))) return fail(HE_ERR_KEY_MISSING, "rotation key missing");
    GUARD_BEGIN
    std::map<int, std::vector<int>> by_level;
    for (int i = 0; i < n_cts; i++) by_level[cts[i]->level].push_back(i);
    std::vector<he_ct *> res((size_t)n_cts * n_steps, nullptr);
    try {
        for (auto &kv : by_level) {
            const int lv = kv.first, Bn = (int)kv.second.size();
            const size_t w = ct_words(&c, lv);
            Buf A(&c.pool, Bn * w);
            Buf dg(&c.pool, (size_t)Bn * c.ndig(lv) * c.qp_rows(lv) * c.N);
            for (int t = 0; t < Bn; t++)
                cudaMemcpyAsync(A.p + t * w, cts[kv.second[t]]->d, w * 8, cudaMemcpyDeviceToDevice, c.stream);
            modup(&c, A.p + (long)(lv + 1) * c.N, (long)w, Bn, lv, dg.p);
            // all steps from one MultSum pass over the digits, one ModDown
            const size_t qp = (size_t)2 * c.qp_rows(lv) * c.N;
            Buf U(&c.pool, (size_t)n_steps * Bn * qp), M(&c.pool, (size_t)n_steps * Bn * w);
            std::vector<uint32_t> gs;
            std::vector<u64 *> uo;
            for (int s = 0; s < n_steps; s++) {
                gs.push_back(galois_of_step(&c, steps[s]));
                uo.push_back(U.p + (size_t)s * Bn * qp);
            }
            rot_qp_multi(&c, A.p, Bn, lv, dg.p, gs.data(), n_steps, uo.data());
            moddown(&c, U.p, 2 * Bn * n_steps, lv, M.p, (long)(lv + 1) * c.N);
            c.n_md += (long long)Bn * n_steps;
            for (int s = 0; s < n_steps; s++)
                for (int t = 0; t < Bn; t++) {
                    const he_ct *in = cts[kv.second[t]];
                    he_ct *o = new_ct(&c, lv, in->scale, in->period);
                    res[(size_t)kv.second[t] * n_steps + s] = o;
                    cudaMemcpyAsync(o->d, M.p + ((size_t)s * Bn + t) * w, w * 8, cudaMemcpyDeviceToDevice, c.stream);
                }
        }
        HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
        if (int rc_dev = device_status(&c)) return rc_dev;
        if (int rc = cuda_status(&c)) throw HeError(rc, last_error());
    } catch (...) {
        for (he_ct *o : res) free_ct(o);
        throw;
    }
    for (size_t i = 0; i < res.size(); i++) outs[i] = res[i];
    return HE_OK;
    GUARD_END
}

int he_add(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct **out) {
    if (!ctx || !out) return fail(HE_ERR_ARG, "null argument");
    Ctx &c = ctx->c;
    if (int rc = check_ct(c, a)) return rc;
    if (int rc = check_ct(c, b)) return rc;
    if (a->level != b->level) return fail(HE_ERR_LEVEL, "operands at different levels");
    if (a->scale != b->scale) return fail(HE_ERR_SCALE, "operands with different scales");
    GUARD_BEGIN
    he_ct *o = new_ct(&c, a->level, a->scale, std::min(a->period, b->period));
    add(&c, a->d, b->d, 1, a->level, o->d);
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    *out = o;
    return cuda_status(&c);
    GUARD_END
}

int he_mult(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct **out) {
    if (!ctx || !out) return fail(HE_ERR_ARG, "null argument");
    Ctx &c = ctx->c;
    if (int rc = check_ct(c, a)) return rc;
    if (int rc = check_ct(c, b)) return rc;
    if (a->level != b->level) return fail(HE_ERR_LEVEL, "operands at different levels");
    GUARD_BEGIN
    he_ct *o = new_ct(&c, a->level, a->scale * b->scale, std::min(a->period, b->period));
    try {
        mult_relin(&c, a->d, b->d, 1, a->level, o->d);
    } catch (...) {
        free_ct(o);
        throw;
    }
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    *out = o;
    return cuda_status(&c);
    GUARD_END
}

int he_rescale(he_ctx *ctx, const he_ct *a, he_ct **out) {
    if (!ctx || !out) return fail(HE_ERR_ARG, "null argument");
    Ctx &c = ctx->c;
    if (int rc = check_ct(c, a)) return rc;
    if (a->level < 1) return fail(HE_ERR_LEVEL, "no level left to rescale");
    GUARD_BEGIN
    he_ct *o = new_ct(&c, a->level - 1, a->scale / (double)c.primes[a->level], a->period);
    rescale(&c, a->d, 1, a->level, o->d);
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    *out = o;
    return cuda_status(&c);
    GUARD_END
}

static he_ct *clone_ct(Ctx &c, const he_ct *a) {
    he_ct *o = new_ct(&c, a->level, a->scale, a->period);
    cudaMemcpyAsync(o->d, a->d, ct_words(&c, a->level) * 8, cudaMemcpyDeviceToDevice, c.stream);
    return o;
}

int he_replicate(he_ctx *ctx, const he_ct *ct, int n, he_ct **out) {
    if (!ctx || !out) return fail(HE_ERR_ARG, "null argument");
    Ctx &c = ctx->c;
    if (int rc = check_ct(c, ct)) return rc;
    if (n < 1 || (long)n * n > c.S || (c.S % (n * n))) return fail(HE_ERR_ARG, "n^2 must divide the slot count");
    GUARD_BEGIN
    he_ct *o = clone_ct(c, ct);
    if (o->period != n * n) {
        try {
            replicate(&c, o->d, 1, o->level, n);
        } catch (...) {
            free_ct(o);
            throw;
        }
        o->period = n * n;
    }
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    *out = o;
    return cuda_status(&c);
    GUARD_END
}

static int check_sched(Ctx &c, int n, const he_mm_sched *s) {
    if (!s) return fail(HE_ERR_ARG, "null schedule");
    auto pow2 = [](int x) { return x > 0 && (x & (x - 1)) == 0; };
    if (!pow2(n) || (long)n * n > c.S) return fail(HE_ERR_ARG, "n must be a power of two with n^2 <= slots");
    if (!pow2(s->n1_z) || !pow2(s->n1_t) || s->n1_z > n || s->n1_t > n || s->n1_z > 32 || s->n1_t > 32)
        return fail(HE_ERR_ARG, "baby-step counts must be powers of two dividing n (<= 32)");
    if (s->dcd_z < 0 || s->dcd_t < 0 || (s->dcd_z && (s->dcd_z >= n || s->dcd_z % s->n1_z)) ||
        (s->dcd_t && (s->dcd_t >= n || s->dcd_t % s->n1_t)))
        return fail(HE_ERR_ARG, "a decomposition needs n' < n with the baby steps dividing n'");
    return HE_OK;
}

// Runs one group of same-shape products: gathers A's and B's, replicates,
// aligns levels, multiplies, scatters.
static void run_group(Ctx &c, const std::vector<const he_ct *> &As, const std::vector<const he_ct *> &Bs, int n,
                      int n1z, int n1t, int level, std::vector<he_ct *> &outs, bool relin_once, int dcd_z,
                      int dcd_t) {
    const int P = (int)As.size();
    // distinct operands: a ciphertext that several products of the group
    // take (as the left or as the right factor) is transformed once
    std::vector<const he_ct *> uA, uB;
    std::vector<int> ia(P), ib(P);
    std::map<const he_ct *, int> mA, mB;
    for (int i = 0; i < P; i++) {
        auto a = mA.emplace(As[i], (int)uA.size());
        if (a.second) uA.push_back(As[i]);
        ia[i] = a.first->second;
        auto b = mB.emplace(Bs[i], (int)uB.size());
        if (b.second) uB.push_back(Bs[i]);
        ib[i] = b.first->second;
    }
    const int nA = (int)uA.size(), nB = (int)uB.size();
    const size_t w = ct_words(&c, level);
    Buf A(&c.pool, nA * w), B(&c.pool, nB * w);
    // drop to the common level while gathering (keep limbs 0..level of both polys)
    auto gather = [&](u64 *dst, const he_ct *x) {
        cudaMemcpy2DAsync(dst, (size_t)(level + 1) * c.N * 8, x->d, (size_t)(x->level + 1) * c.N * 8,
                          (size_t)(level + 1) * c.N * 8, 2, cudaMemcpyDeviceToDevice, c.stream);
    };
    for (int i = 0; i < nA; i++) gather(A.p + i * w, uA[i]);
    for (int i = 0; i < nB; i++) gather(B.p + i * w, uB[i]);
    if (As[0]->period != n * n) replicate(&c, A.p, nA, level, n);
    if (Bs[0]->period != n * n) replicate(&c, B.p, nB, level, n);
    const int depth = hmatmul_depth(n, dcd_z, dcd_t);
    const size_t wo = ct_words(&c, level - depth);
    Buf O(&c.pool, P * wo);
    hmatmul_pairs(&c, A.p, nA, B.p, nB, ia.data(), ib.data(), P, level, n, n1z, n1t, O.p, relin_once, dcd_z, dcd_t);
    double q2 = (double)c.primes[level - depth + 1];   // the prime of the multiplication's rescale
    try {
        for (int i = 0; i < P; i++) {
            he_ct *o = new_ct(&c, level - depth, (As[i]->scale * Bs[i]->scale) / q2, n * n);
            cudaMemcpyAsync(o->d, O.p + i * wo, wo * 8, cudaMemcpyDeviceToDevice, c.stream);
            outs[i] = o;
        }
    } catch (...) {
        for (he_ct *&o : outs) free_ct(o), o = nullptr;
        throw;
    }
}

int he_hmatmul(he_ctx *ctx, const he_ct *A, const he_ct *B, int n, const he_mm_sched *sched, he_ct **out) {
    if (!ctx || !out) return fail(HE_ERR_ARG, "null argument");
    he_mm_job j{A, B, n, sched ? *sched : he_mm_sched{0, 0, 0, 0, 0}};
    if (!sched) return fail(HE_ERR_ARG, "null schedule");
    if (int rc = check_ct(ctx->c, A)) return rc;
    if (int rc = check_ct(ctx->c, B)) return rc;
    return he_hmatmul_batch(&j, 1, out);
}

int he_hmatmul_batch(const he_mm_job *jobs, int n_jobs, he_ct **outs) {
    if (!jobs || !outs || n_jobs < 1) return fail(HE_ERR_ARG, "bad arguments");
    for (int i = 0; i < n_jobs; i++) {
        if (!jobs[i].A || !jobs[i].B || jobs[i].A->ctx != jobs[i].B->ctx) return fail(HE_ERR_ARG, "bad job operands");
        if (int rc = check_sched(*jobs[i].A->ctx, jobs[i].n, &jobs[i].sched)) return rc;
        if (std::min(jobs[i].A->level, jobs[i].B->level) < hmatmul_depth(jobs[i].n, jobs[i].sched.dcd_z, jobs[i].sched.dcd_t))
            return fail(HE_ERR_LEVEL, "not enough levels for the product");
        outs[i] = nullptr;
    }
    GUARD_BEGIN
    std::vector<ProdSpec> prods;
    for (int i = 0; i < n_jobs; i++)
        prods.push_back({jobs[i].A, jobs[i].B, jobs[i].n, jobs[i].sched.n1_z, jobs[i].sched.n1_t,
                         jobs[i].sched.relin_once != 0, jobs[i].sched.dcd_z, jobs[i].sched.dcd_t});
    std::vector<he_ct *> res;
    run_products(prods, res, 0);
    try {
        std::set<Ctx *> ctxs;
        for (auto &p : prods) ctxs.insert(p.A->ctx);
        for (Ctx *c : ctxs) HE_CUDA_CHECK(cudaStreamSynchronize(c->stream));
        for (Ctx *c : ctxs) {
            if (int rc = cuda_status(c)) throw HeError(rc, last_error());
            if (int rc = device_status(c)) throw HeError(rc, last_error());
        }
    } catch (...) {
        for (he_ct *o : res) free_ct(o);
        throw;
    }
    for (int i = 0; i < n_jobs; i++) outs[i] = res[i];
    return HE_OK;
    GUARD_END
}

}  // extern "C"

namespace he {
void run_products(const std::vector<ProdSpec> &prods, std::vector<he_ct *> &outs, int max_batch) {
    typedef std::tuple<Ctx *, int, int, int, int, int, int, int, int, int> Key;
    std::map<Key, std::vector<int>> groups;
    for (size_t i = 0; i < prods.size(); i++) {
        const ProdSpec &j = prods[i];
        int lv = std::min(j.A->level, j.B->level);
        groups[Key(j.A->ctx, lv, j.n, j.n1z, j.n1t, j.A->period == j.n * j.n, j.B->period == j.n * j.n,
                   j.relin_once, j.dcd_z, j.dcd_t)]
            .push_back((int)i);
    }
    outs.assign(prods.size(), nullptr);
    try {
        for (auto &kv : groups) {
            Ctx &c = *std::get<0>(kv.first);
            int lv = std::get<1>(kv.first);
            const std::vector<int> &ix = kv.second;
            const size_t step = max_batch > 0 ? (size_t)max_batch : ix.size();
            // clusters: runs of consecutive products that share an operand
            // with an earlier product of the run; a batch is not cut inside
            // a cluster when an earlier cut fits
            std::vector<char> starts(ix.size() + 1, 1);
            {
                std::set<const he_ct *> ops;
                for (size_t t = 0; t < ix.size(); t++) {
                    const ProdSpec &j = prods[ix[t]];
                    if (t > 0 && (ops.count(j.A) || ops.count(j.B))) {
                        starts[t] = 0;
                    } else {
                        ops.clear();
                    }
                    ops.insert(j.A);
                    ops.insert(j.B);
                }
            }
            for (size_t s0 = 0, s1; s0 < ix.size(); s0 = s1) {
                s1 = std::min(ix.size(), s0 + step);
                size_t cut = s1;
                while (cut > s0 + 1 && !starts[cut]) cut--;
                if (cut > s0 + 1 || starts[cut]) s1 = cut;
                std::vector<const he_ct *> As, Bs;
                for (size_t t = s0; t < s1; t++) {
                    As.push_back(prods[ix[t]].A);
                    Bs.push_back(prods[ix[t]].B);
                }
                std::vector<he_ct *> o(As.size());
                const ProdSpec &j0 = prods[ix[s0]];
                run_group(c, As, Bs, j0.n, j0.n1z, j0.n1t, lv, o, j0.relin_once, j0.dcd_z, j0.dcd_t);
                for (size_t t = s0; t < s1; t++) outs[ix[t]] = o[t - s0];
            }
        }
    } catch (...) {
        for (he_ct *o : outs) free_ct(o);
        outs.clear();
        throw;
    }
}
}  // namespace he

extern "C" {

int he_transpose(he_ctx *ctx, const he_ct *ct, int n, int n1, double prescale, he_ct **out) {
    if (!ctx || !out) return fail(HE_ERR_ARG, "null argument");
    Ctx &c = ctx->c;
    if (int rc = check_ct(c, ct)) return rc;
    he_mm_sched s{n1, n1, 0, 0, 0};
    if (int rc = check_sched(c, n, &s)) return rc;
    if (ct->level < 1) return fail(HE_ERR_LEVEL, "transpose needs 1 level");
    GUARD_BEGIN
    he_ct *tmp = clone_ct(c, ct);
    he_ct *o = nullptr;
    try {
        if (tmp->period != n * n) replicate(&c, tmp->d, 1, tmp->level, n);
        o = new_ct(&c, ct->level - 1, ct->scale, n * n);
        lintrans(&c, tmp->d, 1, ct->level, 2, n, n - 1, n1, -(n / n1), n / n1, prescale, o->d);
    } catch (...) {
        free_ct(tmp);
        free_ct(o);
        throw;
    }
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    free_ct(tmp);
    *out = o;
    return cuda_status(&c);
    GUARD_END
}

int he_linear_transform(he_ctx *ctx, const he_ct *ct, int kind, int n, int n1, int n_prime, he_ct **out) {
    if (!ctx || !out) return fail(HE_ERR_ARG, "null argument");
    if (kind < 0 || kind > 2) return fail(HE_ERR_ARG, "kind must be 0 (sigma), 1 (tau) or 2 (transpose)");
    if (n_prime && kind == 2) return fail(HE_ERR_ARG, "the transpose has no decomposition");
    Ctx &c = ctx->c;
    if (int rc = check_ct(c, ct)) return rc;
    he_mm_sched s{n1, n1, 0, kind == 0 ? n_prime : 0, kind == 1 ? n_prime : 0};
    if (n_prime < 0) return fail(HE_ERR_ARG, "n' must be >= 0");
    if (int rc = check_sched(c, n, &s)) return rc;
    const int m = dcd_levels(n, n_prime, kind == 1);
    if (ct->level < m) return fail(HE_ERR_LEVEL, "not enough levels for the transform");
    GUARD_BEGIN
    he_ct *tmp = clone_ct(c, ct);
    he_ct *o = nullptr;
    try {
        if (tmp->period != n * n) replicate(&c, tmp->d, 1, tmp->level, n);
        o = new_ct(&c, ct->level - m, ct->scale, n * n);
        const int n2 = n / n1;
        if (n_prime) zt_stage_public(&c, tmp->d, 1, ct->level, kind == 1, n, n1, n_prime, ct->level - m, o->d);
        else if (kind == 0) lintrans(&c, tmp->d, 1, ct->level, 0, n, 1, n1, -n2, n2, 1.0, o->d);
        else if (kind == 1) lintrans(&c, tmp->d, 1, ct->level, 1, n, n, n1, 0, n2, 1.0, o->d);
        else lintrans(&c, tmp->d, 1, ct->level, 2, n, n - 1, n1, -n2, n2, 1.0, o->d);
    } catch (...) {
        free_ct(tmp);
        free_ct(o);
        throw;
    }
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    free_ct(tmp);
    *out = o;
    return cuda_status(&c);
    GUARD_END
}

// Matrix rotation steps (mod n^2) of Z (kind 0) or T (kind 1) with the
// simple key substitution: the babies' head a s, 0 < s < n1_sub, and the
// giants a n1 i.
static std::vector<long> ksub_steps(int n, int kind, int n1, int n1_sub) {
    const long n2m = (long)n * n, a = kind == 0 ? 1 : n;
    const int n2 = n / n1;
    std::set<long> st;
    for (int s = 1; s < n1_sub; s++) st.insert(((a * s) % n2m + n2m) % n2m);
    for (int i = kind == 0 ? -n2 : 1; i < n2; i++)
        if (i) st.insert(((a * n1 * i) % n2m + n2m) % n2m);
    st.erase(0);
    return std::vector<long>(st.begin(), st.end());
}

static int check_ksub(int n, int kind, int n1, int n1_sub, long slots) {
    auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
    if (kind < 0 || kind > 1) return fail(HE_ERR_ARG, "kind must be 0 (sigma) or 1 (tau)");
    if (n < 2 || (long)n * n > slots) return fail(HE_ERR_ARG, "n x n must fit the slots");
    if (!pow2(n1) || n1 > n || n % n1) return fail(HE_ERR_ARG, "n1 must be a power of two dividing n");
    if (n1_sub < 2 || n1_sub > n1) return fail(HE_ERR_ARG, "the head length must be in [2, n1]");
    return HE_OK;
}

int he_rot_steps_for_ksub(int n, int kind, int n1, int n1_sub, int slots, int32_t *out, int *count) {
    if (!count) return fail(HE_ERR_ARG, "null count");
    if (int rc = check_ksub(n, kind, n1, n1_sub, slots)) return rc;
    std::set<long> st;
    for (long s : ksub_steps(n, kind, n1, n1_sub)) st.insert(s);
    for (long r = (long)n * n; r < slots; r *= 2) st.insert(slots - r);   // replication
    if (out && *count < (int)st.size()) return fail(HE_ERR_ARG, "output array too small");
    int i = 0;
    if (out)
        for (long s : st) out[i++] = (int32_t)s;
    *count = (int)st.size();
    return HE_OK;
}

int he_linear_transform_ksub(he_ctx *ctx, const he_ct *ct, int kind, int n, int n1, int n1_sub, he_ct **out) {
    if (!ctx || !out) return fail(HE_ERR_ARG, "null argument");
    Ctx &c = ctx->c;
    if (int rc = check_ct(c, ct)) return rc;
    if (int rc = check_ksub(n, kind, n1, n1_sub, c.S)) return rc;
    if (ct->level < 1) return fail(HE_ERR_LEVEL, "not enough levels for the transform");
    GUARD_BEGIN
    he_ct *tmp = clone_ct(c, ct);
    he_ct *o = nullptr;
    try {
        if (tmp->period != n * n) replicate(&c, tmp->d, 1, tmp->level, n);
        o = new_ct(&c, ct->level - 1, ct->scale, n * n);
        const int n2 = n / n1;
        if (kind == 0) lintrans(&c, tmp->d, 1, ct->level, 0, n, 1, n1, -n2, n2, 1.0, o->d, nullptr, n1_sub);
        else lintrans(&c, tmp->d, 1, ct->level, 1, n, n, n1, 0, n2, 1.0, o->d, nullptr, n1_sub);
    } catch (...) {
        free_ct(tmp);
        free_ct(o);
        throw;
    }
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    free_ct(tmp);
    *out = o;
    return cuda_status(&c);
    GUARD_END
}

int he_ntt(he_ctx *ctx, uint64_t *rows_dev, long long n_rows, int level, int inverse) {
    if (!ctx || (n_rows > 0 && !rows_dev) || n_rows < 0) return fail(HE_ERR_ARG, "bad arguments");
    Ctx &c = ctx->c;
    if (level < 0 || level > c.L) return fail(HE_ERR_LEVEL, "level out of range");
    GUARD_BEGIN
    if (inverse)
        ntt_inv(&c, (u64 *)rows_dev, n_rows, c.map_qp(level), c.stream);
    else
        ntt_fwd(&c, (u64 *)rows_dev, n_rows, c.map_qp(level), c.stream);
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    return cuda_status(&c);
    GUARD_END
}

int he_decompose(he_ctx *ctx, const uint64_t *poly_dev, long long n_items, int level, uint64_t *digits_dev) {
    if (!ctx || n_items < 0 || n_items > (1 << 20) || (n_items > 0 && (!poly_dev || !digits_dev)))
        return fail(HE_ERR_ARG, "bad arguments");
    if (((uintptr_t)poly_dev | (uintptr_t)digits_dev) & 15) return fail(HE_ERR_ARG, "buffers must be 16-byte aligned");
    Ctx &c = ctx->c;
    if (level < 0 || level > c.L) return fail(HE_ERR_LEVEL, "level out of range");
    GUARD_BEGIN
    if (n_items > 0) modup(&c, (const u64 *)poly_dev, (long)(level + 1) * c.N, (int)n_items, level, (u64 *)digits_dev);
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    return cuda_status(&c);
    GUARD_END
}

int he_moddown(he_ctx *ctx, const uint64_t *in_dev, long long n_items, int level, uint64_t *out_dev) {
    if (!ctx || n_items < 0 || n_items > (1 << 20) || (n_items > 0 && (!in_dev || !out_dev)))
        return fail(HE_ERR_ARG, "bad arguments");
    if (((uintptr_t)in_dev | (uintptr_t)out_dev) & 15) return fail(HE_ERR_ARG, "buffers must be 16-byte aligned");
    Ctx &c = ctx->c;
    if (level < 0 || level > c.L) return fail(HE_ERR_LEVEL, "level out of range");
    GUARD_BEGIN
    if (n_items > 0)
        moddown(&c, (const u64 *)in_dev, (int)n_items, level, (u64 *)out_dev, (long)(level + 1) * c.N, nullptr, 0);
    HE_CUDA_CHECK(cudaStreamSynchronize(c.stream));
    if (int rc_dev = device_status(&c)) return rc_dev;
    return cuda_status(&c);
    GUARD_END
}

int he_bench_butterfly(int iters, double *bfly_per_s) {
    if (!bfly_per_s || iters < 1) return fail(HE_ERR_ARG, "bad arguments");
    *bfly_per_s = bfly_peak(iters);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HE_ERR_CUDA, cudaGetErrorString(e));
    return HE_OK;
}

int he_trace_enable(he_ctx *ctx, int on) {
    if (!ctx) return fail(HE_ERR_ARG, "null context");
    ctx->c.trace_collect();
    ctx->c.trace = on != 0;
    return HE_OK;
}

int he_trace_read(he_ctx *ctx, int cls, long long *count, double *total_ms, double *bytes, int reset) {
    if (!ctx || cls < 0 || cls > 4) return fail(HE_ERR_ARG, "bad arguments");
    Ctx &c = ctx->c;
    c.trace_collect();
    Ctx::TraceClass &t = c.tr[cls];
    if (count) *count = t.count;
    if (total_ms) *total_ms = t.total_ms;
    if (bytes) *bytes = t.bytes;
    if (reset) {
        t.count = 0;
        t.total_ms = t.bytes = t.ops = 0;
    }
    return HE_OK;
}

int he_trace_ops(he_ctx *ctx, int cls, double *ops) {
    if (!ctx || !ops || cls < 0 || cls > 4) return fail(HE_ERR_ARG, "bad arguments");
    *ops = ctx->c.tr[cls].ops;
    return HE_OK;
}

int he_bench_mac(int iters, double *products_per_s) {
    if (!products_per_s || iters < 1) return fail(HE_ERR_ARG, "bad arguments");
    *products_per_s = mac_peak(iters);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(HE_ERR_CUDA, cudaGetErrorString(e));
    return HE_OK;
}

int he_counters(he_ctx *ctx, long long *ms, long long *dp, long long *md, long long *launches, int reset) {
    if (!ctx) return fail(HE_ERR_ARG, "null context");
    Ctx &c = ctx->c;
    if (ms) *ms = c.n_ms;
    if (dp) *dp = c.n_dp;
    if (md) *md = c.n_md;
    if (launches) *launches = c.n_launch;
    if (reset) c.n_ms = c.n_dp = c.n_md = c.n_launch = 0;
    return HE_OK;
}

}  // extern "C"
