// he_internal.h -- internal declarations of the GB300 RNS-CKKS library.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <set>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/he.h"
#include "modarith.cuh"

namespace he {

// Row -> global prime index map (row r uses prime p[r % n]); passed by value.
// Prime of each row of a multi-row launch (global prime index: q_0..q_L,
// then p_0..p_{alpha-1}).  Row k, after a cyclic shift, is k' = (k + shift)
// mod n; rows k' <= lq are q_{base_q + k'}, the others prime
// base_p + (k' - lq - 1).  Plain integers, so a kernel evaluates it in
// registers (no per-thread copy of a parameter array).
struct RowMap {
    int n = 1, shift = 0, lq = 0, base_q = 0, base_p = 0;
    __host__ __device__ __forceinline__ int at(long k) const {
        int kk = (int)((k + shift) % n);
        return kk <= lq ? base_q + kk : base_p + (kk - lq - 1);
    }
    __host__ __device__ RowMap shifted(long r0) const {
        RowMap m = *this;
        m.shift = (int)((shift + r0) % n);
        return m;
    }
    static RowMap single(int prime) {
        RowMap m;
        m.base_q = prime;
        return m;
    }
};

// Rows a forward NTT leaves untouched: in Decompose output laid out as
// [item][digit][rows_per_digit][N], the digit's own rows r in
// [d alpha, min(d alpha + alpha, nq)) are already in the NTT domain.
// rows_per_digit == 0 disables the skip; row0 is the absolute index of the
// launch's first row.
struct RowSkip {
    int rows_per_digit = 0, ndig = 0, alpha = 0, nq = 0;
    long row0 = 0;
    __host__ __device__ bool skip(long row) const {
        if (!rows_per_digit) return false;
        long a = row0 + row;
        int r = (int)(a % rows_per_digit), d = (int)((a / rows_per_digit) % ndig), i0 = d * alpha;
        return r >= i0 && r < i0 + alpha && r < nq;
    }
};

// Device pool with size-class free lists (no cudaMalloc/cudaFree in steady state).
class DevicePool {
public:
    void *get(size_t bytes);
    void put(void *p);
    void release_all();
    size_t bytes_in_use() const { return in_use_; }
    size_t bytes_cached() const { return cached_; }
    size_t bytes_peak() const { return peak_; }
    // While set, get() serves from `r` and put() returns r's blocks to it
    // (the private scratch of a graph being recorded).
    void set_redirect(DevicePool *r);
    bool owns(void *p);
    ~DevicePool() { release_all(); }

private:
    DevicePool *redirect_ = nullptr;
    // get/put may be called from a serving worker and the caller's thread
    std::mutex mu_;
    std::multimap<size_t, void *> free_;
    std::map<void *, size_t> sizes_;
    size_t in_use_ = 0, cached_ = 0, peak_ = 0;
};

// Scratch buffer handle returned to the pool on scope exit.
struct Buf {
    DevicePool *pool = nullptr;
    u64 *p = nullptr;
    Buf() = default;
    Buf(DevicePool *pl, size_t words) : pool(pl), p((u64 *)pl->get(words * 8)) {}
    Buf(const Buf &) = delete;
    Buf &operator=(const Buf &) = delete;
    Buf(Buf &&o) noexcept : pool(o.pool), p(o.p) { o.p = nullptr; }
    Buf &operator=(Buf &&o) noexcept {
        if (p) pool->put(p);
        pool = o.pool; p = o.p; o.p = nullptr;
        return *this;
    }
    ~Buf() { if (p) pool->put(p); }
};

struct ShoupPair {
    u64 w, wp;
};

// Constants of the exact overflow count of the rounding ModDown, alpha <= 4
// special primes below 2^62 (kernel parameter).
struct MdExact {
    u64 p[4], hp[4];          // p_j, (P-1)/2 mod p_j
    ShoupPair pinv[4];        // (P/p_j)^-1 mod p_j
    u64 phat[4][3];           // P/p_j, little-endian 64-bit limbs (alpha-1 used)
    u64 kP[3][4];             // k P for k = 1..alpha-1 (alpha limbs used)
};

// Constants of one level l (limbs q_0..q_l, then p's).
struct LevelConsts {
    int level = -1;
    int ndig = 0;
    // ModUp: per digit d, per source i (alpha max), qhat_inv (pair); per target row r, qhat_mod[d][i][r]
    ShoupPair *d_up_inv = nullptr;   // [ndig][alpha]
    ShoupPair *d_up_mod = nullptr;   // [ndig][alpha][l+1+alpha]
    // Rescale by q_l: q_l^-1 mod q_i, q_l mod q_i (i < l)
    ShoupPair *d_rs_inv = nullptr;   // [l]
    u64 *d_rs_qlmod = nullptr;       // [l]
};

// One factor of a Diagonal Convergence Decomposition (Sec. 4.2): the
// diagonal of every row (-1 = empty row) on the device, the set of its
// diagonals (mod n^2), the rotation step of a right factor, and a cache id.
struct DcdFactor {
    int *dev = nullptr;
    std::set<long> diags;
    std::string id;
    long step = 0;
};
// Factors in application order: right factors first, the left one last.
struct DcdChain {
    std::vector<DcdFactor> factors;
};

struct Ctx {
    he_params prm;
    int logN, N, S, L, alpha, dnum, nprimes;
    std::vector<u64> primes;       // q_0..q_L, p_0..p_{alpha-1}
    std::vector<ModQ> hmod;
    u64 seed;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;

    ModQ *d_mod = nullptr;         // [nprimes]
    u64 *d_psi = nullptr, *d_psip = nullptr, *d_ipsi = nullptr, *d_ipsip = nullptr;  // [nprimes][N]
    u64 *d_psi2 = nullptr, *d_ipsi2 = nullptr;   // [nprimes][N][2]: (w, w') pairs, one 16-byte load each
    u64 *d_ninv = nullptr;         // [nprimes][2]
    // ModDown constants (level independent)
    ShoupPair *d_dn_pinv = nullptr;  // [alpha]   (P/p_j)^-1 mod p_j
    ShoupPair *d_dn_pmod = nullptr;  // [alpha][L+1] (P/p_j) mod q_r
    ShoupPair *d_dn_Pinv = nullptr;  // [L+1]     P^-1 mod q_r
    ShoupPair *d_Pmod = nullptr;     // [L+1]     P mod q_r
    u64 *d_dn_E = nullptr;           // [alpha][L+1] -(e P + (P-1)/2) mod q_r, e < alpha
    MdExact md_exact;
    std::vector<LevelConsts> lvl;

    // encoder tables
    double *d_zeta = nullptr;      // [2N][2] (cos, sin) of pi e / N
    int *d_slot_t = nullptr;       // [S] t(j) = (5^j mod 2N - 1) / 4
    u64 gauss_T[20];

    // keys (NTT domain): secret key in normal and Montgomery form over all primes
    u64 *d_sk = nullptr, *d_skM = nullptr;  // [nprimes][N]
    u64 *d_pkM = nullptr;                   // [2][L+1][N] Montgomery
    std::map<uint32_t, u64 *> rtk;          // galois -> [dnum][2][nprimes][N] Montgomery
    u64 *rlk = nullptr;

    // cached plaintext diagonals (NTT, Montgomery, over Q_l P), keyed by a string id
    std::map<std::string, u64 *> ptcache;
    std::map<std::string, DcdChain> dcd;     // decompositions by (transform, n, n')
    size_t ptcache_bytes = 0;

    DevicePool pool;
    std::mutex mu;

    // Flag that kernels with bounded waits set when a wait runs out: host
    // memory mapped into the device, read by the host after a synchronise.
    int *h_err = nullptr, *d_err = nullptr;

    // instrumentation
    std::atomic<long long> n_ms{0}, n_dp{0}, n_md{0}, n_launch{0};
    // per-kernel-class tracing: CUDA events on the context stream around each
    // launch of a traced class, with the launch's algorithmic bytes
    struct TraceClass {
        std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
        double total_ms = 0, bytes = 0, ops = 0;   // ops: digit-key products (MultSum)
        long long count = 0;
    };
    bool trace = false;
    // launch-geometry autotuner: per (kernel, shape) the fastest variant,
    // timed on first use (variants compute identical words)
    bool autotune = true;
    int ntt_minb = 2;        // CTAs per SM of the register-blocked forward NTT (2 or 3)
    int ntt_minb_inv = 2;    // and of the inverse NTT
    bool ntt_tuned = false;
    // rows per launch pair of the two-pass NTTs (0: as many as the grid
    // takes): chunks small enough that pass 1 reads pass 0's output from L2
    int ntt_chunk = 0, ntt_chunk_inv = 0;
    // PowerMethod: pairs of Newton steps as five-level composites; the
    // vector's segments refreshed as one packed ciphertext
    bool newton_compose = false;
    bool pack_refresh = false;
    // >= 0: every MultSum launch uses this variant (keys per launch 8), no tuning
    int force_multsum = -1;
    // (level, items, keys) -> (keys per launch << 8) | variant
    std::map<std::tuple<int, int, int>, int> tune_multsum;
    std::map<std::tuple<int, int, int>, int> tune_ck;   // fused C^k babies: (keys per launch << 8) | items per CTA
    std::string tune_log;   // every timed plan, one line each
    TraceClass tr[5];   // 0 MultSum, 1 NTT forward, 2 NTT inverse, 3 ModUp BConv, 4 ModDown BConv
    std::vector<cudaEvent_t> ev_free;
    cudaEvent_t ev_get();
    void trace_begin(int cls, cudaEvent_t &e0);
    void trace_end(int cls, cudaEvent_t e0, double bytes, double ops = 0);
    void trace_collect();

    // helpers
    int qp_rows(int level) const { return level + 1 + alpha; }
    int ndig(int level) const { return (level + 1 + alpha - 1) / alpha; }
    size_t key_words() const { return (size_t)dnum * 2 * nprimes * N; }
    RowMap map_q(int level) const {
        RowMap m;
        m.n = level + 1, m.lq = level;
        return m;
    }
    RowMap map_qp(int level) const {
        RowMap m;
        m.n = level + 1 + alpha, m.lq = level, m.base_p = L + 1;
        return m;
    }
    RowMap map_p() const {
        RowMap m;
        m.n = alpha, m.lq = -1, m.base_p = L + 1;
        return m;
    }
    const LevelConsts &lc(int level);
};

// A ciphertext in the NTT domain: data [2][level+1][N], scale, slot period.
struct Ct {
    Ctx *ctx = nullptr;
    u64 *d = nullptr;
    int level = 0;
    double scale = 1.0;
    int period = 0;
};

// error handling
void set_error(const std::string &msg);
// HE_OK, or HE_ERR_TIMEOUT if a kernel's bounded wait ran out since the last
// check (the flag is cleared).  Call after synchronising the context's stream.
int device_status(const Ctx *c);
#define HE_CUDA_CHECK(expr)                                                          \
    do {                                                                             \
        cudaError_t e__ = (expr);                                                    \
        if (e__ != cudaSuccess) {                                                    \
            he::set_error(std::string("CUDA error: ") + cudaGetErrorString(e__) +     \
                          " at " + __FILE__ + ":" + std::to_string(__LINE__));       \
            return HE_ERR_CUDA;                                                      \
        }                                                                            \
    } while (0)

// host number theory
u64 h_mulmod(u64 a, u64 b, u64 q);
u64 h_powmod(u64 a, u64 e, u64 q);
u64 h_invmod(u64 a, u64 q);
ShoupPair h_shoup(u64 w, u64 q);
int h_gen_primes(int logN, int nq, const int *qbits, int np, const int *pbits, u64 *q, u64 *p);

// NTT
void ntt_fwd(Ctx *ctx, u64 *data, long rows, const RowMap &rm, cudaStream_t st, const RowSkip *skip = nullptr);
// Epilogue of a forward NTT that finishes ModDown or Rescale: the transform
// v of row (item it, limb r) is not stored; instead
//   out[it*os + r*N + x] = (u[it*us + r*N + x] - v) * w[r]  mod q_r.
struct SubScale {
    const u64 *u = nullptr;
    long us = 0;
    u64 *out = nullptr;
    long os = 0;
    const ShoupPair *w = nullptr;
    int rows_per_item = 1;
    long row0 = 0;   // absolute index of the launch's first row
    const u64 *add = nullptr;   // optional addend, laid out like out (item stride as)
    long as = 0;
};
void ntt_fwd_subscale(Ctx *ctx, u64 *data, long rows, const RowMap &rm, cudaStream_t st, const SubScale &ep);
void ntt_inv(Ctx *ctx, u64 *data, long rows, const RowMap &rm, cudaStream_t st);

// ---- kernels.cu launchers (all asynchronous on st) ----
void launch_sample_uniform(Ctx *c, u64 *out, int rows, const RowMap &rm, const int *limb_id, uint32_t obj,
                           uint32_t tag, cudaStream_t st);
void launch_sample_small(Ctx *c, i64 *out, int kind /*0 ternary 1 gauss*/, uint32_t obj, uint32_t tag,
                         cudaStream_t st);
void launch_small_to_rns(Ctx *c, const i64 *x, u64 *out, int rows, const RowMap &rm, cudaStream_t st);
void launch_encode(Ctx *c, const double *zre, const double *zim, double scale, i64 *m_out,
                   cudaStream_t st);
void launch_decode(Ctx *c, const double *coef, double scale, double *zre, double *zim, cudaStream_t st);
// elementwise over rows with a RowMap
void launch_add(Ctx *c, u64 *out, const u64 *a, const u64 *b, long rows, const RowMap &rm, cudaStream_t st);
void launch_sub(Ctx *c, u64 *out, const u64 *a, const u64 *b, long rows, const RowMap &rm, cudaStream_t st);
void launch_neg(Ctx *c, u64 *out, const u64 *a, long rows, const RowMap &rm, cudaStream_t st);
void launch_mul(Ctx *c, u64 *out, const u64 *a, const u64 *b, long rows, const RowMap &rm, cudaStream_t st);
void launch_mulM(Ctx *c, u64 *out, const u64 *a, const u64 *bM, long rows, const RowMap &rm,
                 cudaStream_t st);
void launch_to_mont(Ctx *c, u64 *out, const u64 *a, long rows, const RowMap &rm, cudaStream_t st);
void launch_from_mont(Ctx *c, u64 *out, const u64 *a, long rows, const RowMap &rm, cudaStream_t st);
void launch_mulconst_rows(Ctx *c, u64 *out, const u64 *a, const ShoupPair *w, long rows, int rows_per_item,
                          const RowMap &rm, cudaStream_t st);
void launch_automorph(Ctx *c, u64 *out, const u64 *in, long rows, const RowMap &rm, uint32_t g,
                      cudaStream_t st);
// (d0, d1) -> d01 [B][2][limbs][N], d2 -> [B][limbs][N]; accumulate adds
// the tensor to what d01 and d2 already hold (acc01 / acc2 select the two
// outputs separately when given).  b_poly_stride: words from b's first
// polynomial to its second (0: limbs * N).
void launch_tensor(Ctx *c, u64 *d01, u64 *d2, const u64 *a, const u64 *b, int B, int limbs, long a_item_stride,
                   long b_item_stride, const RowMap &rm, cudaStream_t st, bool accumulate = false,
                   long b_poly_stride = 0);
void launch_tensor_acc(Ctx *c, u64 *d01, u64 *d2, const u64 *a, const u64 *b, int B, int limbs, long as, long bs,
                       const RowMap &rm, cudaStream_t st, bool acc01, bool acc2, long b_poly_stride = 0);
// key switching pieces
// own_ntt (may be null): the input in the NTT domain, item stride own_s; the
// digit's own rows are then copied from it (and the forward NTT must skip
// them), else from coef.
void launch_modup_bconv(Ctx *c, const u64 *coef, u64 *out, int B, int level, cudaStream_t st,
                        const u64 *own_ntt = nullptr, long own_s = 0);
void launch_moddown_bconv(Ctx *c, const u64 *pcoef, u64 *out, int items, int level, cudaStream_t st);
void launch_moddown_final(Ctx *c, u64 *out, const u64 *u, const u64 *conv, const u64 *addend, int items,
                          int level, long u_item_stride, long out_item_stride, long add_item_stride,
                          cudaStream_t st);
void launch_multsum(Ctx *c, u64 *out, const u64 *digits, const u64 *key, uint32_t g, int B, int level,
                    const u64 *c0_for_P, long c0_item_stride, cudaStream_t st);
// Up to kMultSumMaxKeys rotations per launch share one read of the digits
// (longer lists are split); keys must be in the permuted layout.
constexpr int kMultSumMaxKeys = 8;
void launch_multsum_multi(Ctx *c, u64 *const *outs, const u64 *digits, const u64 *const *keys, const uint32_t *gs,
                          int G, int B, int level, const u64 *c0_for_P, long c0s, cudaStream_t st);
// G hoisted rotations of two sources with the same keys, each output the
// masked sum m1_k (.) rot(source 1) + m2_k (.) rot(source 2) over Q_l P.
void launch_multsum_ck(Ctx *c, u64 *const *outs, const u64 *dig1, const u64 *dig2, const u64 *const *keys,
                       const uint32_t *gs, const u64 *const *m1, const u64 *const *m2, int G, int B, int level,
                       const u64 *c01, const u64 *c02, long c0s, cudaStream_t st);
void launch_permute_key(Ctx *c, u64 *out, const u64 *in, long rows, uint32_t g, cudaStream_t st);
void launch_pmul_acc(Ctx *c, u64 *out, const u64 *const *pts, const u64 *const *R, int nterms, int B,
                     int level, long R_item_stride, cudaStream_t st);
void launch_lift_P(Ctx *c, u64 *out_qp, const u64 *in_q, int items, int level, long in_item_stride,
                   long out_item_stride, cudaStream_t st);
void launch_rescale_prep(Ctx *c, const u64 *lastcoef, u64 *out, int items, int level, cudaStream_t st);
void launch_rescale_final(Ctx *c, u64 *out, const u64 *in, const u64 *t, int items, int level,
                          long in_item_stride, long out_item_stride, cudaStream_t st);
void launch_scalar_mul_rows(Ctx *c, u64 *out, const u64 *a, long rows, int rpi, const ShoupPair *vals,
                            const RowMap &rm, cudaStream_t st);
void launch_scalar_add_rows(Ctx *c, u64 *data, long rows, const u64 *vals, const RowMap &rm, cudaStream_t st);
void launch_centre_i64_q0(Ctx *c, const u64 *a, i64 *out, cudaStream_t st);
void launch_dec_q0(Ctx *c, const u64 *c0, const u64 *c1, u64 *out, cudaStream_t st);
void launch_centre_q0(Ctx *c, const u64 *a, double *out, cudaStream_t st);
void launch_diag_fill(Ctx *c, double *out, int kind, int n, long t, long rot, double value, int k,
                      cudaStream_t st);
void launch_copy_rows(u64 *dst, long dst_stride, const u64 *src, long src_stride, int items, long words,
                      cudaStream_t st);

}  // namespace he
