// kernels.cu -- element-wise, sampling, encoding and key-switching kernels.
//
// Layouts: a polynomial is [limbs][N] u64 (limb-major, coalesced along N);
// a ciphertext is [2][level+1][N]; an extended polynomial over Q_l P has
// rows q_0..q_l then p_0..p_{alpha-1}; a batch of B items is contiguous.
#include <cmath>

#include <cstdio>
#include <set>
#include <stdexcept>

#include "bulkcopy.cuh"
#include "he_internal.h"

namespace he {

static inline unsigned nblk(long n, int t) { return (unsigned)((n + t - 1) / t); }

// --------------------------------------------------------------- Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32->64 products
// (multipliers 0xD2511F53, 0xCD9E8D57) with the key bumped by the Weyl
// constants 0x9E3779B9, 0xBB67AE85 between rounds.
__device__ __forceinline__ void philox4x32_10(u32 c[4], u32 k0, u32 k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        u32 lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
        u32 lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
        u32 n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
}

// uniform residue of limb (global prime index) j at coefficient i:
// block (i, j, obj, tag) read as hi64:lo64 = (w3 w2):(w1 w0), reduced mod q.
__global__ void k_sample_uniform(u64 *out, long rows, int N, RowMap rm, const ModQ *mods, u32 obj, u32 tag,
                                 u32 k0, u32 k1) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * N) return;
    long row = idx / N;
    int i = (int)(idx - row * N);
    int pidx = rm.at(row);
    u32 c[4] = {(u32)i, (u32)pidx, obj, tag};
    philox4x32_10(c, k0, k1);
    u64 lo = (u64)c[0] | ((u64)c[1] << 32);
    u64 hi = (u64)c[2] | ((u64)c[3] << 32);
    out[idx] = mod128(hi, lo, mods[pidx]);
}

struct GaussT {
    u64 T[20];
};

// kind 0: ternary from w0 mod 3 -> {0, 1, -1}; kind 1: discrete Gaussian by
// inversion of the cumulative table T on r = (w1:w0) >> 1, sign = w2 bit 0.
__global__ void k_sample_small(i64 *out, int N, int kind, GaussT gt, u32 obj, u32 tag, u32 k0, u32 k1) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    u32 c[4] = {(u32)i, 0u, obj, tag};
    philox4x32_10(c, k0, k1);
    if (kind == 0) {
        u32 r = c[0] % 3u;
        out[i] = r == 0 ? 0 : (r == 1 ? 1 : -1);
    } else {
        u64 r = (((u64)c[1] << 32) | (u64)c[0]) >> 1;
        int k = 0;
        while (k < 19 && r >= gt.T[k]) k++;
        i64 x = k;
        if (x != 0 && (c[2] & 1u)) x = -x;
        out[i] = x;
    }
}

__global__ void k_small_to_rns(const i64 *x, u64 *out, long rows, int N, RowMap rm, const ModQ *mods) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * N) return;
    long row = idx / N;
    int i = (int)(idx - row * N);
    out[idx] = from_signed(x[i], mods[rm.at(row)].q);
}

void launch_sample_uniform(Ctx *c, u64 *out, int rows, const RowMap &rm, const int *, uint32_t obj,
                           uint32_t tag, cudaStream_t st) {
    long n = (long)rows * c->N;
    c->n_launch++;
    k_sample_uniform<<<nblk(n, 256), 256, 0, st>>>(out, rows, c->N, rm, c->d_mod, obj, tag, (u32)c->seed,
                                                   (u32)(c->seed >> 32));
}

void launch_sample_small(Ctx *c, i64 *out, int kind, uint32_t obj, uint32_t tag, cudaStream_t st) {
    GaussT gt;
    for (int k = 0; k < 20; k++) gt.T[k] = c->gauss_T[k];
    c->n_launch++;
    k_sample_small<<<nblk(c->N, 256), 256, 0, st>>>(out, c->N, kind, gt, obj, tag, (u32)c->seed,
                                                   (u32)(c->seed >> 32));
}

void launch_small_to_rns(Ctx *c, const i64 *x, u64 *out, int rows, const RowMap &rm, cudaStream_t st) {
    long n = (long)rows * c->N;
    c->n_launch++;
    k_small_to_rns<<<nblk(n, 256), 256, 0, st>>>(x, out, rows, c->N, rm, c->d_mod);
}

// ------------------------------------------------------ encode / decode
// Inverse canonical embedding (App. A Encode) evaluated in a fixed order so
// that the integer plaintext is reproducible: slot j goes to position
// t = (5^j mod 2N - 1)/4, bit-reversal, radix-2 DIT passes with roots
// conj(zeta^(4 k S/len)), twist by conj(zeta^i), scale by `scale`/S, round
// half away from zero.  Explicit _rn intrinsics: no contraction into FMA.
__device__ __forceinline__ int brev_bits(int x, int bits) { return (int)(__brev((unsigned)x) >> (32 - bits)); }

__global__ void k_enc_permute(const double *zr, const double *zi, double *xr, double *xi, const int *slot_t,
                              int S, int logS) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S) return;
    int t = brev_bits(slot_t[j], logS);
    xr[t] = zr[j];
    xi[t] = zi[j];
}

__global__ void k_dft_pass(double *xr, double *xi, const double *zeta, int S, int len, int sign) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    int half = len >> 1;
    if (e >= S / 2) return;
    int s = (e / half) * len, k = e % half;
    int ex = k * (4 * (S / len));
    double wr = zeta[2 * ex], wi = zeta[2 * ex + 1];
    if (sign < 0) wi = -wi;
    double br = xr[s + k + half], bi = xi[s + k + half];
    double tr = __dsub_rn(__dmul_rn(br, wr), __dmul_rn(bi, wi));
    double ti = __dadd_rn(__dmul_rn(br, wi), __dmul_rn(bi, wr));
    double ar = xr[s + k], ai = xi[s + k];
    xr[s + k] = __dadd_rn(ar, tr);
    xi[s + k] = __dadd_rn(ai, ti);
    xr[s + k + half] = __dsub_rn(ar, tr);
    xi[s + k + half] = __dsub_rn(ai, ti);
}

__global__ void k_enc_final(const double *xr, const double *xi, const double *zeta, double f, i64 *m, int S) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    double wr = zeta[2 * i], wi = -zeta[2 * i + 1];
    double yr = __dsub_rn(__dmul_rn(xr[i], wr), __dmul_rn(xi[i], wi));
    double yi = __dadd_rn(__dmul_rn(xr[i], wi), __dmul_rn(xi[i], wr));
    m[i] = (i64)round(__dmul_rn(yr, f));
    m[i + S] = (i64)round(__dmul_rn(yi, f));
}

// Decode (App. A): x_i = u_i zeta^i with u_i = (m_i + I m_{i+S}) / scale,
// length-S DFT with exponent +1, slot j = x[t(j)].
__global__ void k_dec_twist(const double *coef, double scale, const double *zeta, double *xr, double *xi, int S,
                            int logS) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S) return;
    double ur = coef[i] / scale, ui = coef[i + S] / scale;
    double wr = zeta[2 * i], wi = zeta[2 * i + 1];
    int t = brev_bits(i, logS);
    xr[t] = ur * wr - ui * wi;
    xi[t] = ur * wi + ui * wr;
}

__global__ void k_dec_gather(const double *xr, const double *xi, const int *slot_t, double *zr, double *zi, int S) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= S) return;
    zr[j] = xr[slot_t[j]];
    zi[j] = xi[slot_t[j]];
}

void launch_encode(Ctx *c, const double *zre, const double *zim, double scale, i64 *m_out, cudaStream_t st) {
    int S = c->S, logS = c->logN - 1;
    Buf tmp(&c->pool, (size_t)S), tmp2(&c->pool, (size_t)S);  // S doubles each
    double *xr = (double *)tmp.p, *xi = (double *)tmp2.p;
    c->n_launch++;
    k_enc_permute<<<nblk(S, 256), 256, 0, st>>>(zre, zim, xr, xi, c->d_slot_t, S, logS);
    for (int len = 2; len <= S; len <<= 1) {
        c->n_launch++;
        k_dft_pass<<<nblk(S / 2, 256), 256, 0, st>>>(xr, xi, c->d_zeta, S, len, -1);
    }
    double f = scale / (double)S;
    c->n_launch++;
    k_enc_final<<<nblk(S, 256), 256, 0, st>>>(xr, xi, c->d_zeta, f, m_out, S);
}

void launch_decode(Ctx *c, const double *coef, double scale, double *zre, double *zim, cudaStream_t st) {
    int S = c->S, logS = c->logN - 1;
    Buf tmp(&c->pool, (size_t)S);
    Buf tmp2(&c->pool, (size_t)S);
    double *xr = (double *)tmp.p, *xi = (double *)tmp2.p;
    c->n_launch++;
    k_dec_twist<<<nblk(S, 256), 256, 0, st>>>(coef, scale, c->d_zeta, xr, xi, S, logS);
    for (int len = 2; len <= S; len <<= 1) {
        c->n_launch++;
        k_dft_pass<<<nblk(S / 2, 256), 256, 0, st>>>(xr, xi, c->d_zeta, S, len, +1);
    }
    c->n_launch++;
    k_dec_gather<<<nblk(S, 256), 256, 0, st>>>(xr, xi, c->d_slot_t, zre, zim, S);
}

// ----------------------------------------------------------- elementwise
#define EW_PROLOGUE                                                   \
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;           \
    if (idx >= rows * (long)N) return;                                \
    long row = idx / N;                                               \
    const ModQ &m = mods[rm.at(row)];                           \
    (void)m;

__global__ void k_add(u64 *o, const u64 *a, const u64 *b, long rows, int N, RowMap rm, const ModQ *mods) {
    EW_PROLOGUE
    o[idx] = addmod(a[idx], b[idx], m.q);
}
__global__ void k_sub(u64 *o, const u64 *a, const u64 *b, long rows, int N, RowMap rm, const ModQ *mods) {
    EW_PROLOGUE
    o[idx] = submod(a[idx], b[idx], m.q);
}
__global__ void k_neg(u64 *o, const u64 *a, long rows, int N, RowMap rm, const ModQ *mods) {
    EW_PROLOGUE
    u64 v = a[idx];
    o[idx] = v ? m.q - v : 0;
}
__global__ void k_mul(u64 *o, const u64 *a, const u64 *b, long rows, int N, RowMap rm, const ModQ *mods) {
    EW_PROLOGUE
    o[idx] = mulmod(a[idx], b[idx], m);
}
__global__ void k_mulM(u64 *o, const u64 *a, const u64 *bM, long rows, int N, RowMap rm, const ModQ *mods) {
    EW_PROLOGUE
    o[idx] = mulmont(a[idx], bM[idx], m);
}
__global__ void k_to_mont(u64 *o, const u64 *a, long rows, int N, RowMap rm, const ModQ *mods) {
    EW_PROLOGUE
    o[idx] = mulmont(a[idx], m.r2, m);  // a R^2 R^-1 = a R
}
__global__ void k_from_mont(u64 *o, const u64 *a, long rows, int N, RowMap rm, const ModQ *mods) {
    EW_PROLOGUE
    o[idx] = redc(a[idx], 0, m);
}

#define EW_LAUNCH(kern, ...)                                                         \
    do {                                                                             \
        long n__ = rows * (long)c->N;                                                \
        if (n__ > 0) c->n_launch++, kern<<<nblk(n__, 256), 256, 0, st>>>(__VA_ARGS__, rows, c->N, rm, c->d_mod); \
    } while (0)

void launch_add(Ctx *c, u64 *out, const u64 *a, const u64 *b, long rows, const RowMap &rm, cudaStream_t st) {
    EW_LAUNCH(k_add, out, a, b);
}
void launch_sub(Ctx *c, u64 *out, const u64 *a, const u64 *b, long rows, const RowMap &rm, cudaStream_t st) {
    EW_LAUNCH(k_sub, out, a, b);
}
void launch_neg(Ctx *c, u64 *out, const u64 *a, long rows, const RowMap &rm, cudaStream_t st) {
    EW_LAUNCH(k_neg, out, a);
}
void launch_mul(Ctx *c, u64 *out, const u64 *a, const u64 *b, long rows, const RowMap &rm, cudaStream_t st) {
    EW_LAUNCH(k_mul, out, a, b);
}
void launch_mulM(Ctx *c, u64 *out, const u64 *a, const u64 *bM, long rows, const RowMap &rm, cudaStream_t st) {
    EW_LAUNCH(k_mulM, out, a, bM);
}
void launch_to_mont(Ctx *c, u64 *out, const u64 *a, long rows, const RowMap &rm, cudaStream_t st) {
    EW_LAUNCH(k_to_mont, out, a);
}
void launch_from_mont(Ctx *c, u64 *out, const u64 *a, long rows, const RowMap &rm, cudaStream_t st) {
    EW_LAUNCH(k_from_mont, out, a);
}

// out[row] = a[row] * w[row % rows_per_item] (Shoup constant per row)
__global__ void k_mulconst_rows(u64 *o, const u64 *a, const ShoupPair *w, int rpi, long rows, int N, RowMap rm,
                                const ModQ *mods) {
    EW_PROLOGUE
    ShoupPair s = w[row % rpi];
    o[idx] = shoup(a[idx], s.w, s.wp, m.q);
}
void launch_mulconst_rows(Ctx *c, u64 *out, const u64 *a, const ShoupPair *w, long rows, int rpi,
                          const RowMap &rm, cudaStream_t st) {
    long n = rows * (long)c->N;
    if (n > 0)
        c->n_launch++;
        k_mulconst_rows<<<nblk(n, 256), 256, 0, st>>>(out, a, w, rpi, rows, c->N, rm, c->d_mod);
}

// NTT-domain index of the automorphism X -> X^g: output slot x (evaluation
// point psi^(2 brv(x)+1)) reads input slot brv(((2 brv(x)+1) g mod 2N - 1)/2).
__device__ __forceinline__ int auto_index(int x, u32 g, int logN) {
    int N = 1 << logN;
    u32 e = 2u * (u32)brev_bits(x, logN) + 1u;
    u32 e2 = (u32)(((u64)e * g) & (u64)(2 * N - 1));
    return brev_bits((int)((e2 - 1) >> 1), logN);
}

__global__ void k_automorph(u64 *o, const u64 *in, long rows, int logN, u32 g) {
    int N = 1 << logN;
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * (long)N) return;
    long row = idx / N;
    int x = (int)(idx - row * N);
    o[idx] = in[row * N + auto_index(x, g, logN)];
}
void launch_automorph(Ctx *c, u64 *out, const u64 *in, long rows, const RowMap &, uint32_t g, cudaStream_t st) {
    long n = rows * (long)c->N;
    c->n_launch++;
    if (n > 0) k_automorph<<<nblk(n, 256), 256, 0, st>>>(out, in, rows, c->logN, g);
}

// tensor product in the NTT domain: d0 = a0 b0, d1 = a0 b1 + a1 b0, d2 = a1 b1.
// d01: [B][2][limbs][N] (d0, d1 of each item); d2: [B][limbs][N].  The
// operands' first `limbs` limbs are used: item strides as, bs; b's second
// polynomial starts bps words after its first (a higher-level b is read in
// place, without a level-dropping copy).
__global__ void k_tensor(u64 *d01, u64 *d2, const u64 *a, const u64 *b, int B, int limbs, int N,
                         long as, long bs, long bps, RowMap rm, const ModQ *mods, int accumulate) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long per = (long)limbs * N;
    if (idx >= (long)B * per) return;
    int it = (int)(idx / per);
    long off = idx - (long)it * per;
    int limb = (int)(off / N);
    const ModQ &m = mods[rm.at(limb)];
    const u64 *pa = a + it * as, *pb = b + it * bs;
    u64 a0 = pa[off], a1 = pa[per + off], b0 = pb[off], b1 = pb[bps + off];
    U128 acc = {0, 0};
    mac128(acc, a0, b1);
    mac128(acc, a1, b0);
    u64 t1 = redc(acc.lo, acc.hi, m);
    u64 v0 = mulmod(a0, b0, m), v1 = redc(t1 * m.r2, mulhi64(t1, m.r2), m), v2 = mulmod(a1, b1, m);
    u64 *o = d01 + (long)it * 2 * per + off;
    u64 *o2 = d2 + (long)it * per + off;
    if (accumulate & 1) {
        v0 = addmod(v0, o[0], m.q);
        v1 = addmod(v1, o[per], m.q);
    }
    if (accumulate & 2) v2 = addmod(v2, o2[0], m.q);
    o[0] = v0;
    o[per] = v1;
    o2[0] = v2;
}
void launch_tensor(Ctx *c, u64 *d01, u64 *d2, const u64 *a, const u64 *b, int B, int limbs, long as, long bs,
                   const RowMap &rm, cudaStream_t st, bool accumulate, long bps) {
    long n = (long)B * limbs * c->N;
    c->n_launch++;
    k_tensor<<<nblk(n, 256), 256, 0, st>>>(d01, d2, a, b, B, limbs, c->N, as, bs, bps ? bps : (long)limbs * c->N,
                                           rm, c->d_mod, accumulate ? 3 : 0);
}
void launch_tensor_acc(Ctx *c, u64 *d01, u64 *d2, const u64 *a, const u64 *b, int B, int limbs, long as, long bs,
                       const RowMap &rm, cudaStream_t st, bool acc01, bool acc2, long bps) {
    long n = (long)B * limbs * c->N;
    c->n_launch++;
    k_tensor<<<nblk(n, 256), 256, 0, st>>>(d01, d2, a, b, B, limbs, c->N, as, bs, bps ? bps : (long)limbs * c->N,
                                           rm, c->d_mod, (acc01 ? 1 : 0) | (acc2 ? 2 : 0));
}

// ------------------------------------------------------------- ModUp
// Decompose (Sec. 3.3): per digit d, y_i = [c_i (Q_d/q_i)^-1]_{q_i}; every
// target row r of Q_l P gets sum_i y_i (Q_d/q_i mod r) mod r, except the
// digit's own rows, which keep c_r.  In/out in coefficient form.
// coef: [B][l+1][N]; out: [B][ndig][l+1+alpha][N].
//
// blockIdx.y is the digit: a CTA stages that digit's conversion constants
// and row primes in shared memory once and walks (item, coefficient pair)
// with a grid stride.  Each thread converts two adjacent coefficients with
// 16-byte loads and stores.  When the digit's primes and the row's prime are
// below 2^42 the products y_i (w_i 2^64 mod r) accumulate in 96 bits with
// carry-chained 32-bit multiply-adds and one Montgomery reduction ends the
// row; otherwise the A lazy Shoup products (each in [0, 2r)) are summed and
// reduced once.
static int sm_count(int dev) {
    static int n[64];
    dev &= 63;
    if (!n[dev]) cudaDeviceGetAttribute(&n[dev], cudaDevAttrMultiProcessorCount, dev);
    return n[dev] > 0 ? n[dev] : 1;
}

// C adjacent words, one 16-byte access for C = 2
template <int C>
struct Words {
    u64 w[C];
};
template <int C>
__device__ __forceinline__ Words<C> load_words(const u64 *p) {
    Words<C> r;
    if constexpr (C == 2) {
        const ulonglong2 v = *(const ulonglong2 *)p;
        r.w[0] = v.x, r.w[1] = v.y;
    } else {
        r.w[0] = *p;
    }
    return r;
}
template <int C>
__device__ __forceinline__ void store_words(u64 *p, const Words<C> &r) {
    if constexpr (C == 2) *(ulonglong2 *)p = make_ulonglong2(r.w[0], r.w[1]);
    else *p = r.w[0];
}

// A: special primes per digit; C: adjacent coefficients per thread (2 on
// launches that fill the GPU, 1 on small ones, where more threads hide more
// latency).
template <int A, int C>
__global__ void __launch_bounds__(256) k_modup_bconv(const u64 *coef, u64 *out, int B, int level, int ndig, int N,
                                                     RowMap qp, const ModQ *mods, const ShoupPair *up_inv,
                                                     const ShoupPair *up_mod, const u64 *own_ntt, long own_s) {
    __shared__ ShoupPair s_mod[A * 64];   // [s][r], rows <= 64
    __shared__ u64 s_mont[A * 64];        // w 2^64 mod r of the same constants
    __shared__ u64 s_q[64], s_w1[64], s_qinv[64];
    const int d = blockIdx.y;
    const int rows = level + 1 + A;
    const int i0 = d * A;
    const int ns = min(A, level + 1 - i0);
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const ModQ m = mods[r <= qp.lq ? r : qp.base_p + (r - qp.lq - 1)];   // qp is unshifted
        s_q[r] = m.q, s_w1[r] = m.wone, s_qinv[r] = m.qinv;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < ns * rows; e += blockDim.x) {
        const int sd = e / rows, r = e - sd * rows;
        const ShoupPair w = up_mod[((long)d * A + sd) * rows + r];
        s_mod[e] = w;
        // w 2^64 - w' r is in [0, r) and congruent to -w' r modulo 2^64
        s_mont[e] = (u64)0 - w.wp * s_q[r];
    }
    ShoupPair inv[A];
    u64 qs[A];
    bool narrow = true;   // every source prime below 2^42 (uniform over the CTA)
#pragma unroll
    for (int sd = 0; sd < A; sd++)
        if (sd < ns) inv[sd] = up_inv[d * A + sd], qs[sd] = mods[i0 + sd].q, narrow = narrow && qs[sd] < (1ull << 42);
    __syncthreads();
    const int per = N / C;
    const long units = (long)B * per;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < units; idx += (long)gridDim.x * blockDim.x) {
        const int b = (int)(idx / per);
        const int x = C * (int)(idx - (long)b * per);
        const u64 *cb = coef + (long)b * (level + 1) * N + x;
        u64 *ob = out + ((long)b * ndig + d) * rows * N + x;
        u64 y[C][A];
#pragma unroll
        for (int sd = 0; sd < A; sd++) {
#pragma unroll
            for (int c = 0; c < C; c++) y[c][sd] = 0;
            if (sd < ns) {
                const Words<C> v = load_words<C>(cb + (long)(i0 + sd) * N);
#pragma unroll
                for (int c = 0; c < C; c++) y[c][sd] = shoup(v.w[c], inv[sd].w, inv[sd].wp, qs[sd]);
            }
        }
        for (int r = 0; r < rows; r++) {
            Words<C> o;
            if (r >= i0 && r < i0 + ns) {   // uniform over the CTA
                o = load_words<C>(own_ntt ? own_ntt + (long)b * own_s + (long)r * N + x : cb + (long)r * N);
            } else if (narrow && s_q[r] < (1ull << 42)) {   // uniform over the CTA
                // products below 2^84: A of them stay below 2^86 < r 2^64
                u32 w0[C], w1[C], w2[C];
#pragma unroll
                for (int c = 0; c < C; c++) w0[c] = w1[c] = w2[c] = 0;
#pragma unroll
                for (int sd = 0; sd < A; sd++) {
                    if (sd < ns) {
                        const u64 wm = s_mont[sd * rows + r];
#pragma unroll
                        for (int c = 0; c < C; c++) mac96(w0[c], w1[c], w2[c], y[c][sd], wm);
                    }
                }
#pragma unroll
                for (int c = 0; c < C; c++) o.w[c] = redc_q(((u64)w1[c] << 32) | w0[c], w2[c], s_q[r], s_qinv[r]);
            } else {
                const u64 q = s_q[r];
                u64 acc[C];
#pragma unroll
                for (int c = 0; c < C; c++) acc[c] = 0;
#pragma unroll
                for (int sd = 0; sd < A; sd++) {
                    if (sd < ns) {
                        const ShoupPair w = s_mod[sd * rows + r];
#pragma unroll
                        for (int c = 0; c < C; c++) acc[c] += shoup_lazy(y[c][sd], w.w, w.wp, q);
                    }
                }
                // < 2 A q <= 8q < 2^64
#pragma unroll
                for (int c = 0; c < C; c++) o.w[c] = reduce_any(acc[c], q, s_w1[r]);
            }
            store_words<C>(ob + (long)r * N, o);
        }
    }
}

template <int A>
static void modup_launch_a(Ctx *c, const u64 *coef, u64 *out, int B, int level, int nd, const ShoupPair *up_inv,
                           const ShoupPair *up_mod, const u64 *own_ntt, long own_s, cudaStream_t st) {
    const int nsm = sm_count(c->device);
    // two coefficients per thread once the launch fills the GPU with 8 CTAs
    // of 256 threads per SM, one below that
    const bool wide = (long)B * (c->N / 2) * nd >= (long)nsm * 8 * 256;
    const long units = (long)B * (c->N / (wide ? 2 : 1));
    long gx = std::max(1L, (long)nsm * 8 / nd);
    gx = std::min(gx, (long)nblk(units, 256));
    const dim3 grid((unsigned)gx, (unsigned)nd);
    const RowMap qp = c->map_qp(level);
    if (wide)
        k_modup_bconv<A, 2><<<grid, 256, 0, st>>>(coef, out, B, level, nd, c->N, qp, c->d_mod, up_inv, up_mod, own_ntt, own_s);
    else
        k_modup_bconv<A, 1><<<grid, 256, 0, st>>>(coef, out, B, level, nd, c->N, qp, c->d_mod, up_inv, up_mod, own_ntt, own_s);
}

static void modup_launch(Ctx *c, const u64 *coef, u64 *out, int B, int level, int nd, const ShoupPair *up_inv,
                         const ShoupPair *up_mod, const u64 *own_ntt, long own_s, cudaStream_t st) {
    switch (c->alpha) {
    case 1: modup_launch_a<1>(c, coef, out, B, level, nd, up_inv, up_mod, own_ntt, own_s, st); break;
    case 2: modup_launch_a<2>(c, coef, out, B, level, nd, up_inv, up_mod, own_ntt, own_s, st); break;
    case 3: modup_launch_a<3>(c, coef, out, B, level, nd, up_inv, up_mod, own_ntt, own_s, st); break;
    default: modup_launch_a<4>(c, coef, out, B, level, nd, up_inv, up_mod, own_ntt, own_s, st); break;
    }
}

void launch_modup_bconv(Ctx *c, const u64 *coef, u64 *out, int B, int level, cudaStream_t st, const u64 *own_ntt,
                        long own_s) {
    const LevelConsts &L = c->lc(level);
    c->n_launch++;
    cudaEvent_t e0;
    c->trace_begin(3, e0);
    modup_launch(c, coef, out, B, level, L.ndig, L.d_up_inv, L.d_up_mod, own_ntt, own_s, st);
    // the input limbs once, every digit's extended limbs once
    c->trace_end(3, e0, 8.0 * B * c->N * ((level + 1) + (double)L.ndig * c->qp_rows(level)));
}

// Same conversion with caller-supplied constants (layout of LevelConsts).
void launch_modup_bconv_with(Ctx *c, const u64 *coef, u64 *out, int B, int level, const ShoupPair *up_inv,
                             const ShoupPair *up_mod, cudaStream_t st) {
    c->n_launch++;
    modup_launch(c, coef, out, B, level, c->ndig(level), up_inv, up_mod, nullptr, 0, st);
}

// ----------------------------------------------------- constants per limb
// Multiplying by a constant polynomial m (or adding it) acts on every
// NTT-domain slot of limb i with the scalar m mod q_i.
struct ScalarList {
    ShoupPair w[64];
};
__global__ void k_scalar_mul_rows(u64 *o, const u64 *a, long rows, int rpi, int N, ScalarList s, RowMap rm,
                                  const ModQ *mods) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * (long)N) return;
    long row = idx / N;
    int r = (int)(row % rpi);
    o[idx] = shoup(a[idx], s.w[r].w, s.w[r].wp, mods[rm.at(row)].q);
}
void launch_scalar_mul_rows(Ctx *c, u64 *out, const u64 *a, long rows, int rpi, const ShoupPair *vals,
                            const RowMap &rm, cudaStream_t st) {
    ScalarList s;
    for (int i = 0; i < rpi && i < 64; i++) s.w[i] = vals[i];
    long n = rows * (long)c->N;
    c->n_launch++;
    k_scalar_mul_rows<<<nblk(n, 256), 256, 0, st>>>(out, a, rows, rpi, c->N, s, rm, c->d_mod);
}
__global__ void k_scalar_add_rows(u64 *o, long rows, int N, ScalarList s, RowMap rm, const ModQ *mods) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * (long)N) return;
    long row = idx / N;
    u64 q = mods[rm.at(row)].q;
    o[idx] = addmod(o[idx], s.w[row].w, q);
}
void launch_scalar_add_rows(Ctx *c, u64 *data, long rows, const u64 *vals, const RowMap &rm, cudaStream_t st) {
    ScalarList s;
    for (int i = 0; i < rows && i < 64; i++) s.w[i].w = vals[i];
    long n = rows * (long)c->N;
    c->n_launch++;
    k_scalar_add_rows<<<nblk(n, 256), 256, 0, st>>>(data, rows, c->N, s, rm, c->d_mod);
}
// centred lift of a residue mod q_0 to a signed integer
__global__ void k_centre_i64_q0(const u64 *a, i64 *out, int N, const ModQ *mods) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    u64 q = mods[0].q, v = a[x];
    out[x] = v > (q >> 1) ? -(i64)(q - v) : (i64)v;
}
void launch_centre_i64_q0(Ctx *c, const u64 *a, i64 *out, cudaStream_t st) {
    c->n_launch++;
    k_centre_i64_q0<<<nblk(c->N, 256), 256, 0, st>>>(a, out, c->N, c->d_mod);
}

// ------------------------------------------------------------- ModDown
// Rounding ModDown (App. A KeySwitch: round(P^-1 x)) as floor((x + h) / P),
// h = (P-1)/2.  With v_j = u_{p_j} + h mod p_j and y_j = [v_j (P/p_j)^-1]_{p_j},
// the exact residue (x + h) mod P is S - e P with S = sum_j y_j (P/p_j) and
// the overflow count e = floor(S / P) < A, taken exactly: S is summed in
// 64-bit limbs and compared with P, 2P, ...
// conv_r = ((x + h) mod P) - h mod q_r, coefficient form (h is added to
// every coefficient, so it is folded in here, before the forward NTT):
// conv_r = sum_j y_j (P/p_j mod q_r) + E_{e,r} with E_{e,r} = -(e P + h) mod q_r.
// pcoef: [items][A][N]; out: [items][l+1][N].

// e = floor(S / P) for S = sum_j y[j] (P/p_j): S < A P < 2^(64 A).
template <int A>
__device__ __forceinline__ int md_overflow(const u64 (&y)[A], const MdExact &k) {
    if constexpr (A == 1) {
        return 0;
    } else {
        u64 s[A];
#pragma unroll
        for (int i = 0; i < A; i++) s[i] = 0;
#pragma unroll
        for (int j = 0; j < A; j++) {
            u64 carry = 0;
#pragma unroll
            for (int i = 0; i < A - 1; i++) {
                const u64 lo = y[j] * k.phat[j][i], hi = __umul64hi(y[j], k.phat[j][i]);
                u64 t = s[i] + lo;
                u64 cy = t < lo ? 1ull : 0ull;
                t += carry;
                cy += t < carry ? 1ull : 0ull;
                s[i] = t;
                carry = hi + cy;   // hi < 2^62
            }
            s[A - 1] += carry;     // the partial sums stay below S
        }
        int e = 0;
#pragma unroll
        for (int m = 0; m < A - 1; m++) {
            int cmp = 0;
#pragma unroll
            for (int i = A - 1; i >= 0; i--)
                if (cmp == 0) cmp = s[i] > k.kP[m][i] ? 1 : (s[i] < k.kP[m][i] ? -1 : 0);
            e += cmp >= 0 ? 1 : 0;
        }
        return e;
    }
}

// C adjacent coefficients per thread (2: 16-byte loads and stores, on
// launches that fill the GPU; 1 on small ones), a grid stride over (item,
// coefficient group); per row the lazy Shoup products and E are summed and
// reduced once.
template <int A, int C>
__global__ void __launch_bounds__(256) k_moddown_bconv(const u64 *pcoef, u64 *out, int items, int level, int N,
                                                       const __grid_constant__ MdExact k, const ModQ *mods,
                                                       const ShoupPair *pmod, const u64 *E, int L) {
    __shared__ ShoupPair s_c[A * 64];
    __shared__ u64 s_E[A * 64], s_q[64], s_w1[64];
    const int nr = level + 1;
    for (int r = threadIdx.x; r < nr; r += blockDim.x) s_q[r] = mods[r].q, s_w1[r] = mods[r].wone;
    for (int e = threadIdx.x; e < A * nr; e += blockDim.x) {
        const int j = e / nr, r = e - j * nr;
        s_c[e] = pmod[j * (L + 1) + r];
        s_E[e] = E[j * (L + 1) + r];
    }
    __syncthreads();
    const int per = N / C;
    const long units = (long)items * per;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < units; idx += (long)gridDim.x * blockDim.x) {
        const int it = (int)(idx / per);
        const int x = C * (int)(idx - (long)it * per);
        u64 y[C][A];
#pragma unroll
        for (int j = 0; j < A; j++) {
            const Words<C> v = load_words<C>(pcoef + ((long)it * A + j) * N + x);
            const u64 p = k.p[j];
#pragma unroll
            for (int c = 0; c < C; c++) y[c][j] = shoup(addmod(v.w[c], k.hp[j], p), k.pinv[j].w, k.pinv[j].wp, p);
        }
        int e[C];
#pragma unroll
        for (int c = 0; c < C; c++) e[c] = md_overflow<A>(y[c], k);
        u64 *op = out + (long)it * nr * N + x;
        for (int r = 0; r < nr; r++) {
            const u64 q = s_q[r];
            u64 acc[C];
#pragma unroll
            for (int c = 0; c < C; c++) acc[c] = s_E[e[c] * nr + r];
#pragma unroll
            for (int j = 0; j < A; j++) {
                const ShoupPair w = s_c[j * nr + r];
#pragma unroll
                for (int c = 0; c < C; c++) acc[c] += shoup_lazy(y[c][j], w.w, w.wp, q);
            }
            // < (2 A + 1) q <= 9q < 2^64
            Words<C> o;
#pragma unroll
            for (int c = 0; c < C; c++) o.w[c] = reduce_any(acc[c], q, s_w1[r]);
            store_words<C>(op + (long)r * N, o);
        }
    }
}

template <int A>
static void moddown_launch_a(Ctx *c, const u64 *pcoef, u64 *out, int items, int level, cudaStream_t st) {
    const int nsm = sm_count(c->device);
    const bool wide = (long)items * (c->N / 2) >= (long)nsm * 8 * 256;
    const long units = (long)items * (c->N / (wide ? 2 : 1));
    const unsigned grid = (unsigned)std::min<long>((long)nsm * 8, nblk(units, 256));
    const MdExact &k = c->md_exact;
    if (wide)
        k_moddown_bconv<A, 2><<<grid, 256, 0, st>>>(pcoef, out, items, level, c->N, k, c->d_mod, c->d_dn_pmod, c->d_dn_E, c->L);
    else
        k_moddown_bconv<A, 1><<<grid, 256, 0, st>>>(pcoef, out, items, level, c->N, k, c->d_mod, c->d_dn_pmod, c->d_dn_E, c->L);
}

void launch_moddown_bconv(Ctx *c, const u64 *pcoef, u64 *out, int items, int level, cudaStream_t st) {
    c->n_launch++;
    cudaEvent_t e0;
    c->trace_begin(4, e0);
    switch (c->alpha) {
    case 1: moddown_launch_a<1>(c, pcoef, out, items, level, st); break;
    case 2: moddown_launch_a<2>(c, pcoef, out, items, level, st); break;
    case 3: moddown_launch_a<3>(c, pcoef, out, items, level, st); break;
    default: moddown_launch_a<4>(c, pcoef, out, items, level, st); break;
    }
    c->trace_end(4, e0, 8.0 * items * c->N * (c->alpha + level + 1));
}

// out_r = (u_r - conv_r) P^-1 mod q_r (+ addend_r), NTT domain, r <= level.
__global__ void k_moddown_final(u64 *out, const u64 *u, const u64 *conv, const u64 *add, int items, int level,
                                int N, long us, long os, long as, const ModQ *mods, const ShoupPair *Pinv) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long per = (long)(level + 1) * N;
    if (idx >= (long)items * per) return;
    int it = (int)(idx / per);
    long off = idx - (long)it * per;
    int r = (int)(off / N);
    u64 q = mods[r].q;
    ShoupPair w = Pinv[r];
    u64 v = shoup(submod(u[it * us + off], conv[idx], q), w.w, w.wp, q);
    if (add) v = addmod(v, add[it * as + off], q);
    out[it * os + off] = v;
}
void launch_moddown_final(Ctx *c, u64 *out, const u64 *u, const u64 *conv, const u64 *addend, int items, int level,
                          long us, long os, long as, cudaStream_t st) {
    long n = (long)items * (level + 1) * c->N;
    c->n_launch++;
    k_moddown_final<<<nblk(n, 256), 256, 0, st>>>(out, u, conv, addend, items, level, c->N, us, os, as, c->d_mod,
                                                  c->d_dn_Pinv);
}

// ------------------------------------------------------------- MultSum
// MultSum + Permute (Sec. 3.3.1) for G rotations that share one Decompose
// output (hoisting).  Rotation keys are stored permuted, K'_g[y] = K_g[x]
// with y = pi_g(x) the NTT-domain index of kappa_g, so that
//   out_g[x] = sum_d D[d][pi_g(x)] K_g[d][x] = T_g[pi_g(x)],
//   T_g[y]   = sum_d D[d][y] K'_g[d][y]
// (the same products, summed in the same order, for every output word).
// Each digit word is loaded once and multiplied into all G accumulators; the
// result is written to x = pi_g^{-1}(y), which stays inside the aligned
// 32-word block of y (kappa permutes the low bits of the bit-reversed index
// only), so stores remain coalesced.  Keys in Montgomery form (one REDC per
// output).  With c0 given, P * c0[y] is added on the Q rows of poly 0 (the
// hoisted rotation kept in Q_l P of double hoisting).
// digits: [B][ndig][rows][N]; key_k: [dnum][2][nprimes][N];
// out_k: [B][2][rows][N].
template <int G>
struct MultiKeys {
    const u64 *key[G];
    u64 *out[G];
    u32 ginv[G];   // pi_g^{-1} = pi_{g^{-1} mod 2N}; 1 = identity
};

// Each digit word is loaded once and multiplied into the 2G accumulators of
// the G keys (2G independent accumulation chains per thread).
// With PF > 0 every thread also asks L2 for its digit word PF digits ahead,
// and the threads of the first item for their key words, so that more DRAM
// requests are in flight than the loads themselves keep (no registers held).
__device__ __forceinline__ void l2_prefetch(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// OCC: resident CTAs per SM the launch bound asks for (0: by G).
template <int G, bool STREAM, int PF = 0, int OCC = 0>
__global__ void __launch_bounds__(256, OCC ? OCC : G <= 2 ? 4 : G <= 5 ? 2 : 1) k_multsum_multi(MultiKeys<G> mk, const u64 *digits, int B, int BI, int level,
                                                       int alpha, int L, int ndig, int nprimes, int logN,
                                                       const ModQ *mods, const u64 *c0, long c0s,
                                                       const ShoupPair *Pmod) {
    const int N = 1 << logN;
    const int XW = 256 / BI;
    const int tx = threadIdx.x % XW, ti = threadIdx.x / XW;
    const int y = blockIdx.x * XW + tx;
    const int r = blockIdx.y;
    const int b = blockIdx.z * BI + ti;
    if (b >= B || y >= N) return;
    const int rows = level + 1 + alpha;
    const int kr = r <= level ? r : L + 1 + (r - level - 1);   // the row's global prime
    const ModQ m = mods[kr];
    const long dstride = (long)rows * N;
    const u64 *dp = digits + (long)b * ndig * dstride + (long)r * N + y;
    const long koff = (long)kr * N + y, kd = 2L * nprimes * N, kk = (long)nprimes * N;
    U128 a0[G], a1[G];
    if (m.q < (1ull << 42)) {
        // residues below 2^42 (uniform over the CTA): 96-bit accumulation
        u32 x0[2 * G], x1[2 * G], x2[2 * G];
#pragma unroll
        for (int k = 0; k < 2 * G; k++) x0[k] = 0, x1[k] = 0, x2[k] = 0;
        for (int d = 0; d < ndig; d++) {
            if (PF && d + PF < ndig) {
                l2_prefetch(dp + (long)(d + PF) * dstride);
                if (ti == 0)
#pragma unroll
                    for (int k = 0; k < G; k++) {
                        l2_prefetch(mk.key[k] + (long)(d + PF) * kd + koff);
                        l2_prefetch(mk.key[k] + (long)(d + PF) * kd + koff + kk);
                    }
            }
            const u64 v = STREAM ? __ldcs(dp + (long)d * dstride) : __ldg(dp + (long)d * dstride);
#pragma unroll
            for (int k = 0; k < G; k++) {
                const u64 *kp = mk.key[k] + (long)d * kd + koff;
                mac96(x0[2 * k], x1[2 * k], x2[2 * k], v, __ldg(kp));
                mac96(x0[2 * k + 1], x1[2 * k + 1], x2[2 * k + 1], v, __ldg(kp + kk));
            }
        }
#pragma unroll
        for (int k = 0; k < G; k++) {
            a0[k] = U128{((u64)x1[2 * k] << 32) | x0[2 * k], x2[2 * k]};
            a1[k] = U128{((u64)x1[2 * k + 1] << 32) | x0[2 * k + 1], x2[2 * k + 1]};
        }
    } else {
#pragma unroll
        for (int k = 0; k < G; k++) a0[k] = U128{0, 0}, a1[k] = U128{0, 0};
        for (int d = 0; d < ndig; d++) {
            if (PF && d + PF < ndig) {
                l2_prefetch(dp + (long)(d + PF) * dstride);
                if (ti == 0)
#pragma unroll
                    for (int k = 0; k < G; k++) {
                        l2_prefetch(mk.key[k] + (long)(d + PF) * kd + koff);
                        l2_prefetch(mk.key[k] + (long)(d + PF) * kd + koff + kk);
                    }
            }
            const u64 v = STREAM ? __ldcs(dp + (long)d * dstride) : __ldg(dp + (long)d * dstride);
#pragma unroll
            for (int k = 0; k < G; k++) {
                const u64 *kp = mk.key[k] + (long)d * kd + koff;
                mac128_q(a0[k], v, __ldg(kp), m.q);
                mac128_q(a1[k], v, __ldg(kp + kk), m.q);
            }
        }
    }
    u64 pc0 = 0;
    const bool with_c0 = c0 && r <= level;
    if (with_c0) {
        ShoupPair w = Pmod[r];
        pc0 = shoup(c0[b * c0s + (long)r * N + y], w.w, w.wp, m.q);
    }
#pragma unroll
    for (int k = 0; k < G; k++) {
        u64 o0 = redc(a0[k].lo, a0[k].hi, m), o1 = redc(a1[k].lo, a1[k].hi, m);
        if (with_c0) o0 = addmod(o0, pc0, m.q);
        const int x = mk.ginv[k] == 1u ? y : auto_index(y, mk.ginv[k], logN);
        u64 *ob = mk.out[k] + (long)b * 2 * rows * N;
        ob[(long)r * N + x] = o0;
        ob[(long)(rows + r) * N + x] = o1;
    }
}

// The thread-per-word MultSum with two adjacent coefficients per thread:
// every digit and key load is 16 bytes (ulonglong2), so twice the bytes are
// in flight per load at the same number of resident warps.  For launches of
// at most two rotations (the per-thread accumulators double).
template <int G, bool STREAM, int OCC>
__global__ void __launch_bounds__(256, OCC) k_multsum_vec(MultiKeys<G> mk, const u64 *digits, int B, int BI, int level,
                                                          int alpha, int L, int ndig, int nprimes, int logN,
                                                          const ModQ *mods, const u64 *c0, long c0s,
                                                          const ShoupPair *Pmod) {
    const int N = 1 << logN;
    const int XW = 256 / BI;
    const int tx = threadIdx.x % XW, ti = threadIdx.x / XW;
    const int y = 2 * (blockIdx.x * XW + tx);
    const int r = blockIdx.y;
    const int b = blockIdx.z * BI + ti;
    if (b >= B || y >= N) return;
    const int rows = level + 1 + alpha;
    const int kr = r <= level ? r : L + 1 + (r - level - 1);
    const ModQ m = mods[kr];
    const long dstride = (long)rows * N;
    const ulonglong2 *dp = (const ulonglong2 *)(digits + (long)b * ndig * dstride + (long)r * N + y);
    const long koff = (long)kr * N + y, kd = 2L * nprimes * N, kk = (long)nprimes * N;
    U128 acc[2][2 * G];   // [coefficient][key, polynomial]
    if (m.q < (1ull << 42)) {
        u32 x0[2][2 * G], x1[2][2 * G], x2[2][2 * G];
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
            for (int k = 0; k < 2 * G; k++) x0[c][k] = 0, x1[c][k] = 0, x2[c][k] = 0;
        for (int d = 0; d < ndig; d++) {
            const ulonglong2 v = STREAM ? __ldcs(dp + (long)d * dstride / 2) : __ldg(dp + (long)d * dstride / 2);
#pragma unroll
            for (int k = 0; k < G; k++) {
                const ulonglong2 *kp = (const ulonglong2 *)(mk.key[k] + (long)d * kd + koff);
                const ulonglong2 k0 = __ldg(kp), k1 = __ldg(kp + kk / 2);
                mac96(x0[0][2 * k], x1[0][2 * k], x2[0][2 * k], v.x, k0.x);
                mac96(x0[1][2 * k], x1[1][2 * k], x2[1][2 * k], v.y, k0.y);
                mac96(x0[0][2 * k + 1], x1[0][2 * k + 1], x2[0][2 * k + 1], v.x, k1.x);
                mac96(x0[1][2 * k + 1], x1[1][2 * k + 1], x2[1][2 * k + 1], v.y, k1.y);
            }
        }
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
            for (int k = 0; k < 2 * G; k++) acc[c][k] = U128{((u64)x1[c][k] << 32) | x0[c][k], x2[c][k]};
    } else {
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
            for (int k = 0; k < 2 * G; k++) acc[c][k] = U128{0, 0};
        for (int d = 0; d < ndig; d++) {
            const ulonglong2 v = STREAM ? __ldcs(dp + (long)d * dstride / 2) : __ldg(dp + (long)d * dstride / 2);
#pragma unroll
            for (int k = 0; k < G; k++) {
                const ulonglong2 *kp = (const ulonglong2 *)(mk.key[k] + (long)d * kd + koff);
                const ulonglong2 k0 = __ldg(kp), k1 = __ldg(kp + kk / 2);
                mac128_q(acc[0][2 * k], v.x, k0.x, m.q);
                mac128_q(acc[1][2 * k], v.y, k0.y, m.q);
                mac128_q(acc[0][2 * k + 1], v.x, k1.x, m.q);
                mac128_q(acc[1][2 * k + 1], v.y, k1.y, m.q);
            }
        }
    }
    const bool with_c0 = c0 && r <= level;
    const ShoupPair w = with_c0 ? Pmod[r] : ShoupPair{0, 0};
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const int yc = y + c;
        u64 pc0 = 0;
        if (with_c0) pc0 = shoup(c0[b * c0s + (long)r * N + yc], w.w, w.wp, m.q);
#pragma unroll
        for (int k = 0; k < G; k++) {
            u64 o0 = redc(acc[c][2 * k].lo, acc[c][2 * k].hi, m), o1 = redc(acc[c][2 * k + 1].lo, acc[c][2 * k + 1].hi, m);
            if (with_c0) o0 = addmod(o0, pc0, m.q);
            const int x = mk.ginv[k] == 1u ? yc : auto_index(yc, mk.ginv[k], logN);
            u64 *ob = mk.out[k] + (long)b * 2 * rows * N;
            ob[(long)r * N + x] = o0;
            ob[(long)(rows + r) * N + x] = o1;
        }
    }
}

// The same MultSum with the G keys split over the CTA's warps: 8 warps =
// (G / KG) key groups x BI = 8 KG / G items, 32 coefficients of one row per
// CTA; each thread accumulates KG keys of one item, so its state (2 KG
// accumulators) does not grow with G and more CTAs fit on an SM.  A digit
// word is loaded by the warps of every key group (one DRAM read, L1 for the
// others), a key word by the warps of every item; every output word is
// still the sum over the digits of the same products, reduced once.
template <int G, int KG, int OCC>
__global__ void __launch_bounds__(256, OCC) k_multsum_split(const __grid_constant__ MultiKeys<G> mk, const u64 *digits, int B, int level,
                                                            int alpha, int L, int ndig, int nprimes, int logN,
                                                            const ModQ *mods, const u64 *c0, long c0s,
                                                            const ShoupPair *Pmod) {
    constexpr int NGRP = G / KG, BI = 8 / NGRP;
    const int N = 1 << logN;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int kg0 = (wid / BI) * KG, bi = wid % BI;
    const int y = blockIdx.x * 32 + lane;
    const int r = blockIdx.y;
    const int b = blockIdx.z * BI + bi;
    if (b >= B || y >= N) return;
    const int rows = level + 1 + alpha;
    const int kr = r <= level ? r : L + 1 + (r - level - 1);
    const ModQ m = mods[kr];
    const long dstride = (long)rows * N;
    const u64 *dp = digits + (long)b * ndig * dstride + (long)r * N + y;
    const long koff = (long)kr * N + y, kd = 2L * nprimes * N, kk = (long)nprimes * N;
    U128 a0[KG], a1[KG];
    if (m.q < (1ull << 42)) {
        u32 x0[2 * KG], x1[2 * KG], x2[2 * KG];
#pragma unroll
        for (int k = 0; k < 2 * KG; k++) x0[k] = 0, x1[k] = 0, x2[k] = 0;
        for (int d = 0; d < ndig; d++) {
            const u64 v = __ldg(dp + (long)d * dstride);
#pragma unroll
            for (int k = 0; k < KG; k++) {
                const u64 *kp = mk.key[kg0 + k] + (long)d * kd + koff;
                mac96(x0[2 * k], x1[2 * k], x2[2 * k], v, __ldg(kp));
                mac96(x0[2 * k + 1], x1[2 * k + 1], x2[2 * k + 1], v, __ldg(kp + kk));
            }
        }
#pragma unroll
        for (int k = 0; k < KG; k++) {
            a0[k] = U128{((u64)x1[2 * k] << 32) | x0[2 * k], x2[2 * k]};
            a1[k] = U128{((u64)x1[2 * k + 1] << 32) | x0[2 * k + 1], x2[2 * k + 1]};
        }
    } else {
#pragma unroll
        for (int k = 0; k < KG; k++) a0[k] = U128{0, 0}, a1[k] = U128{0, 0};
        for (int d = 0; d < ndig; d++) {
            const u64 v = __ldg(dp + (long)d * dstride);
#pragma unroll
            for (int k = 0; k < KG; k++) {
                const u64 *kp = mk.key[kg0 + k] + (long)d * kd + koff;
                mac128_q(a0[k], v, __ldg(kp), m.q);
                mac128_q(a1[k], v, __ldg(kp + kk), m.q);
            }
        }
    }
    u64 pc0 = 0;
    const bool with_c0 = c0 && r <= level;
    if (with_c0) {
        ShoupPair w = Pmod[r];
        pc0 = shoup(c0[b * c0s + (long)r * N + y], w.w, w.wp, m.q);
    }
#pragma unroll
    for (int k = 0; k < KG; k++) {
        u64 o0 = redc(a0[k].lo, a0[k].hi, m), o1 = redc(a1[k].lo, a1[k].hi, m);
        if (with_c0) o0 = addmod(o0, pc0, m.q);
        const u32 gi = mk.ginv[kg0 + k];
        const int x = gi == 1u ? y : auto_index(y, gi, logN);
        u64 *ob = mk.out[kg0 + k] + (long)b * 2 * rows * N;
        ob[(long)r * N + x] = o0;
        ob[(long)(rows + r) * N + x] = o1;
    }
}

// The key-split MultSum with two adjacent coefficients per thread and
// 16-byte digit and key loads (each warp covers 64 coefficients).
template <int G, int KG, int OCC>
__global__ void __launch_bounds__(256, OCC) k_multsum_splitv(const __grid_constant__ MultiKeys<G> mk,
                                                             const u64 *digits, int B, int level, int alpha, int L,
                                                             int ndig, int nprimes, int logN, const ModQ *mods,
                                                             const u64 *c0, long c0s, const ShoupPair *Pmod) {
    constexpr int NGRP = G / KG, BI = 8 / NGRP;
    const int N = 1 << logN;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int kg0 = (wid / BI) * KG, bi = wid % BI;
    const int y = 2 * (blockIdx.x * 32 + lane);
    const int r = blockIdx.y;
    const int b = blockIdx.z * BI + bi;
    if (b >= B || y >= N) return;
    const int rows = level + 1 + alpha;
    const int kr = r <= level ? r : L + 1 + (r - level - 1);
    const ModQ m = mods[kr];
    const long dstride = (long)rows * N;
    const ulonglong2 *dp = (const ulonglong2 *)(digits + (long)b * ndig * dstride + (long)r * N + y);
    const long koff = (long)kr * N + y, kd = 2L * nprimes * N, kk = (long)nprimes * N;
    U128 acc[2][2 * KG];
    if (m.q < (1ull << 42)) {
        u32 x0[2][2 * KG], x1[2][2 * KG], x2[2][2 * KG];
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
            for (int k = 0; k < 2 * KG; k++) x0[c][k] = 0, x1[c][k] = 0, x2[c][k] = 0;
        for (int d = 0; d < ndig; d++) {
            const ulonglong2 v = __ldg(dp + (long)d * dstride / 2);
#pragma unroll
            for (int k = 0; k < KG; k++) {
                const ulonglong2 *kp = (const ulonglong2 *)(mk.key[kg0 + k] + (long)d * kd + koff);
                const ulonglong2 k0 = __ldg(kp), k1 = __ldg(kp + kk / 2);
                mac96(x0[0][2 * k], x1[0][2 * k], x2[0][2 * k], v.x, k0.x);
                mac96(x0[1][2 * k], x1[1][2 * k], x2[1][2 * k], v.y, k0.y);
                mac96(x0[0][2 * k + 1], x1[0][2 * k + 1], x2[0][2 * k + 1], v.x, k1.x);
                mac96(x0[1][2 * k + 1], x1[1][2 * k + 1], x2[1][2 * k + 1], v.y, k1.y);
            }
        }
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
            for (int k = 0; k < 2 * KG; k++) acc[c][k] = U128{((u64)x1[c][k] << 32) | x0[c][k], x2[c][k]};
    } else {
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
            for (int k = 0; k < 2 * KG; k++) acc[c][k] = U128{0, 0};
        for (int d = 0; d < ndig; d++) {
            const ulonglong2 v = __ldg(dp + (long)d * dstride / 2);
#pragma unroll
            for (int k = 0; k < KG; k++) {
                const ulonglong2 *kp = (const ulonglong2 *)(mk.key[kg0 + k] + (long)d * kd + koff);
                const ulonglong2 k0 = __ldg(kp), k1 = __ldg(kp + kk / 2);
                mac128_q(acc[0][2 * k], v.x, k0.x, m.q);
                mac128_q(acc[1][2 * k], v.y, k0.y, m.q);
                mac128_q(acc[0][2 * k + 1], v.x, k1.x, m.q);
                mac128_q(acc[1][2 * k + 1], v.y, k1.y, m.q);
            }
        }
    }
    const bool with_c0 = c0 && r <= level;
    const ShoupPair w = with_c0 ? Pmod[r] : ShoupPair{0, 0};
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const int yc = y + c;
        u64 pc0 = 0;
        if (with_c0) pc0 = shoup(c0[b * c0s + (long)r * N + yc], w.w, w.wp, m.q);
#pragma unroll
        for (int k = 0; k < KG; k++) {
            u64 o0 = redc(acc[c][2 * k].lo, acc[c][2 * k].hi, m), o1 = redc(acc[c][2 * k + 1].lo, acc[c][2 * k + 1].hi, m);
            if (with_c0) o0 = addmod(o0, pc0, m.q);
            const u32 gi = mk.ginv[kg0 + k];
            const int x = gi == 1u ? yc : auto_index(yc, gi, logN);
            u64 *ob = mk.out[kg0 + k] + (long)b * 2 * rows * N;
            ob[(long)r * N + x] = o0;
            ob[(long)(rows + r) * N + x] = o1;
        }
    }
}

// Permutes key rows into the layout above: out[row][pi_g(x)] = in[row][x].
__global__ void k_permute_key(u64 *out, const u64 *in, long rows, int logN, u32 g) {
    const int N = 1 << logN;
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * (long)N) return;
    long row = idx / N;
    int x = (int)(idx - row * N);
    out[row * N + auto_index(x, g, logN)] = in[idx];
}
void launch_permute_key(Ctx *c, u64 *out, const u64 *in, long rows, uint32_t g, cudaStream_t st) {
    long n = rows * (long)c->N;
    c->n_launch++;
    k_permute_key<<<nblk(n, 256), 256, 0, st>>>(out, in, rows, c->logN, g);
}

#include "multsum_tma.cuh"

// Launch of the bulk-copy MultSum, persistent: as many CTAs as fit on the
// GPU at once.  Variants: 8: 64-coefficient segments of 8 items, 8 stages;
// 9: 128 of 4, 6 stages; 10: 256 of 2, 4 stages.
template <int G, int S, int TW, int BI>
static void multsum_tma_launch(Ctx *c, const MultiKeys<G> &mk, const u64 *digits, int B, int level, const u64 *c0,
                               long c0s, cudaStream_t st) {
    static_assert(TW * BI == 2 * MST_CONSUMERS, "two items per consumer thread");
    static int occ[64];   // resident CTAs per SM, per device
    const size_t smem = (size_t)S * (BI + 2 * G) * TW * 8;
    const int dev = c->device & 63;
    if (!occ[dev]) {
        cudaFuncSetAttribute(k_multsum_tma<G, S, TW, BI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_multsum_tma<G, S, TW, BI>, MST_THREADS, smem);
        occ[dev] = nb > 0 ? nb : 1;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    MstGeom g;
    g.N = c->N, g.logN = c->logN, g.rows = level + 1 + c->alpha, g.level = level, g.L = c->L;
    g.ndig = c->ndig(level), g.nprimes = c->nprimes, g.ntx = c->N / TW, g.nig = (B + BI - 1) / BI;
    g.B = B;
    g.ntiles = (long)g.ntx * g.rows * g.nig;
    const long grid = std::min<long>(g.ntiles, (long)nsm * occ[dev]);
    k_multsum_tma<G, S, TW, BI><<<(unsigned)grid, MST_THREADS, smem, st>>>(mk, digits, g, c->d_mod, c0, c0s,
                                                                            c->d_Pmod, c->d_err);
}

// MultSum launch variants: items per CTA (BI), streaming digit loads.
static void multsum_variant(int v, int B, int &BI, bool &stream) {
    static const int bis[4] = {8, 4, 2, 1};
    BI = bis[v & 3];
    while (BI > 1 && BI > B) BI >>= 1;
    stream = (v >> 2) & 1;
}

template <int G>
static void multsum_launch_g(Ctx *c, int v, u64 *const *outs, const u64 *digits, const u64 *const *keys,
                             const uint32_t *gs, int B, int level, const u64 *c0, long c0s, cudaStream_t st) {
    MultiKeys<G> mk;
    const u32 M = 2u * (u32)c->N;
    for (int k = 0; k < G; k++) {
        mk.key[k] = keys[k];
        mk.out[k] = outs[k];
        // inverse of the odd g modulo 2N: Newton iteration on 32-bit words
        u32 g = gs[k], inv = g;
        for (int it = 0; it < 5; it++) inv *= 2u - g * inv;
        mk.ginv[k] = inv & (M - 1);
    }
    if ((v == 80 || v == 84) && G <= 2) {
        // two coefficients per thread, 16-byte loads, more resident CTAs
        if constexpr (G <= 2) {
            constexpr int OCCV = G == 1 ? 5 : 3;
            int BI;
            bool stream;
            multsum_variant(0, B, BI, stream);
            stream = v == 84;
            const int rows = level + 1 + c->alpha, XW = 256 / BI;
            dim3 grid((unsigned)((c->N / 2 + XW - 1) / XW), (unsigned)rows, (unsigned)((B + BI - 1) / BI));
            if (stream)
                k_multsum_vec<G, true, OCCV><<<grid, 256, 0, st>>>(mk, digits, B, BI, level, c->alpha, c->L,
                                                                   c->ndig(level), c->nprimes, c->logN, c->d_mod, c0,
                                                                   c0s, c->d_Pmod);
            else
                k_multsum_vec<G, false, OCCV><<<grid, 256, 0, st>>>(mk, digits, B, BI, level, c->alpha, c->L,
                                                                    c->ndig(level), c->nprimes, c->logN, c->d_mod, c0,
                                                                    c0s, c->d_Pmod);
            c->n_launch++;
            return;
        }
    }
    if (v == 80 || v == 84) v = v == 80 ? 32 : 36;   // more than two rotations: the one-coefficient kernel
    if (v == 96 || v == 97) {
        // rotations split over warps (1 or 2 per thread), two coefficients per thread
        const int rows = level + 1 + c->alpha;
        auto go = [&](auto kern, int bi) {
            dim3 grid((unsigned)((c->N / 2 + 31) / 32), (unsigned)rows, (unsigned)((B + bi - 1) / bi));
            kern<<<grid, 256, 0, st>>>(mk, digits, B, level, c->alpha, c->L, c->ndig(level), c->nprimes, c->logN,
                                       c->d_mod, c0, c0s, c->d_Pmod);
        };
        if (v == 97 && G % 2 == 0 && G >= 2) {
            constexpr int KG2 = (G % 2 == 0 && G >= 2) ? 2 : 1;
            constexpr int NG2 = G / KG2;
            if constexpr (8 % NG2 == 0) {
                go(k_multsum_splitv<G, KG2, 3>, 8 / NG2);
                c->n_launch++;
                return;
            }
        }
        if constexpr (8 % G == 0) {
            go(k_multsum_splitv<G, 1, 5>, 8 / G);
            c->n_launch++;
            return;
        }
        v = 80;   // G does not divide the warps
    }
    if ((v == 80 || v == 84) && G > 2) v = v == 80 ? 32 : 36;
    if (v == 64 || v == 65) {
        // keys split over warps: KG = 1 (64) or 2 (65, G even)
        const int rows = level + 1 + c->alpha;
        auto go = [&](auto kern, int bi) {
            dim3 grid((unsigned)((c->N + 31) / 32), (unsigned)rows, (unsigned)((B + bi - 1) / bi));
            kern<<<grid, 256, 0, st>>>(mk, digits, B, level, c->alpha, c->L, c->ndig(level), c->nprimes, c->logN,
                                       c->d_mod, c0, c0s, c->d_Pmod);
        };
        if (v == 65 && G % 2 == 0 && G >= 2) {
            constexpr int KG2 = (G % 2 == 0 && G >= 2) ? 2 : 1;
            constexpr int NG2 = G / KG2;
            if constexpr (8 % NG2 == 0) {
                go(k_multsum_split<G, KG2, 4>, 8 / NG2);
                c->n_launch++;
                return;
            }
        }
        if constexpr (8 % G == 0) {
            go(k_multsum_split<G, 1, 6>, 8 / G);
            c->n_launch++;
            return;
        }
        v = 32;   // G does not divide the warps: the high-occupancy thread-per-word kernel
    }
    if (v >= 8 && v <= 10) {
        if (v == 8) multsum_tma_launch<G, 8, 64, 8>(c, mk, digits, B, level, c0, c0s, st);
        else if (v == 9) multsum_tma_launch<G, 6, 128, 4>(c, mk, digits, B, level, c0, c0s, st);
        else multsum_tma_launch<G, 4, 256, 2>(c, mk, digits, B, level, c0, c0s, st);
        c->n_launch++;
        return;
    }
    int BI;
    bool stream;
    multsum_variant(v & 15, B, BI, stream);
    const bool pf = (v & 16) != 0;
    const int rows = level + 1 + c->alpha, XW = 256 / BI;
    dim3 grid((unsigned)((c->N + XW - 1) / XW), (unsigned)rows, (unsigned)((B + BI - 1) / BI));
    // bit 5: the launch bound asks for more resident CTAs (fewer registers)
    constexpr int OCC_HI = G <= 1 ? 8 : G <= 2 ? 6 : G <= 4 ? 4 : 3;
    const bool hi = (v & 32) != 0;
#define MS_LAUNCH(STR, PFD, OCC)                                                                           \
    k_multsum_multi<G, STR, PFD, OCC><<<grid, 256, 0, st>>>(mk, digits, B, BI, level, c->alpha, c->L,          \
                                                            c->ndig(level), c->nprimes, c->logN, c->d_mod, c0, c0s, \
                                                            c->d_Pmod)
    if (hi) {
        if (pf) MS_LAUNCH(false, 2, OCC_HI);
        else if (stream) MS_LAUNCH(true, 0, OCC_HI);
        else MS_LAUNCH(false, 0, OCC_HI);
    } else if (stream) {
        if (pf) MS_LAUNCH(true, 2, 0); else MS_LAUNCH(true, 0, 0);
    } else {
        if (pf) MS_LAUNCH(false, 2, 0); else MS_LAUNCH(false, 0, 0);
    }
#undef MS_LAUNCH
    c->n_launch++;
}

static void multsum_launch(Ctx *c, int v, int G, u64 *const *outs, const u64 *digits, const u64 *const *keys,
                           const uint32_t *gs, int B, int level, const u64 *c0, long c0s, cudaStream_t st) {
    switch (G) {
    case 1: multsum_launch_g<1>(c, v, outs, digits, keys, gs, B, level, c0, c0s, st); break;
    case 2: multsum_launch_g<2>(c, v, outs, digits, keys, gs, B, level, c0, c0s, st); break;
    case 3: multsum_launch_g<3>(c, v, outs, digits, keys, gs, B, level, c0, c0s, st); break;
    case 4: multsum_launch_g<4>(c, v, outs, digits, keys, gs, B, level, c0, c0s, st); break;
    case 5: multsum_launch_g<5>(c, v, outs, digits, keys, gs, B, level, c0, c0s, st); break;
    case 6: multsum_launch_g<6>(c, v, outs, digits, keys, gs, B, level, c0, c0s, st); break;
    case 7: multsum_launch_g<7>(c, v, outs, digits, keys, gs, B, level, c0, c0s, st); break;
    default: multsum_launch_g<8>(c, v, outs, digits, keys, gs, B, level, c0, c0s, st); break;
    }
}

void launch_multsum_multi(Ctx *c, u64 *const *outs, const u64 *digits, const u64 *const *keys, const uint32_t *gs,
                          int G, int B, int level, const u64 *c0_for_P, long c0s, cudaStream_t st) {
    if (G <= 0) return;
    const int rows = level + 1 + c->alpha;
    // a launch plan: keys per launch (chunk) and the launch variant
    auto run = [&](int chunk, int v, bool traced) {
        for (int k0 = 0; k0 < G; k0 += chunk) {
            const int g = std::min(chunk, G - k0);
            cudaEvent_t e0 = nullptr;
            if (traced) c->trace_begin(0, e0);
            multsum_launch(c, v, g, outs + k0, digits, keys + k0, gs + k0, B, level, c0_for_P, c0s, st);
            if (traced) {
                // algorithmic bytes: every key (2 polys x ndig digits x rows
                // limbs) read once, every item's digits read once for the g
                // keys, both output polys of every (item, key) written, c0
                // read once if fused
                double nd = c->ndig(level), W = (double)c->N * 8.0;
                double bytes = g * 2.0 * nd * rows * W +
                               (double)B * (nd * rows * W + g * 2.0 * rows * W + (c0_for_P ? (level + 1) * W : 0));
                c->trace_end(0, e0, bytes, (double)B * nd * rows * c->N * 2.0 * g);
            }
        }
    };
    int chunk = std::min(G, kMultSumMaxKeys), v = 0;  // default: 8 keys, 8 items per CTA, cached loads
    if (c->force_multsum >= 0) {
        v = c->force_multsum;
    } else if (c->autotune) {
        auto key3 = std::make_tuple(level, B, G);
        auto it = c->tune_multsum.find(key3);
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cap);
        if (it != c->tune_multsum.end()) {
            chunk = it->second >> 8, v = it->second & 255;
        } else if (cap == cudaStreamCaptureStatusNone) {
            // time every (keys per launch, variant) twice on these very
            // launches (the outputs do not depend on the plan); keep the fastest
            cudaEvent_t a = c->ev_get(), b = c->ev_get();
            float best = 1e30f;
            std::set<std::tuple<int, int, bool>> seen;
            for (int ch : {8, 4, 2, 1}) {
                const int cc = std::min(ch, G);
                for (int cand : {0, 1, 2, 3, 4, 5, 6, 7, 16, 20, 32, 36, 48, 64, 65, 80, 84, 96, 97, 8, 9, 10}) {
                    int BI;
                    bool stream;
                    multsum_variant(cand & 15, B, BI, stream);
                    if (cand >= 8) BI = 100 + cand;   // the bulk-copy and prefetching kernels: their own entries
                    if (!seen.insert(std::make_tuple(cc, BI, stream)).second) continue;
                    float t = 1e30f;
                    for (int rep = 0; rep < 2; rep++) {
                        cudaEventRecord(a, st);
                        run(cc, cand, false);
                        cudaEventRecord(b, st);
                        cudaEventSynchronize(b);
                        float ms = 0;
                        cudaEventElapsedTime(&ms, a, b);
                        t = std::min(t, ms);
                    }
                    if (t < best) best = t, chunk = cc, v = cand;
                    char line[128];
                    snprintf(line, sizeof line, "multsum level %d B %d G %d chunk %d BI %d stream %d ms %.4f\n",
                             level, B, G, cc, BI, (int)stream, t);
                    c->tune_log += line;
                }
            }
            c->ev_free.push_back(a);
            c->ev_free.push_back(b);
            c->tune_multsum[key3] = (chunk << 8) | v;
        }
    }
    run(chunk, v, true);
}

void launch_multsum(Ctx *c, u64 *out, const u64 *digits, const u64 *key, uint32_t g, int B, int level,
                    const u64 *c0_for_P, long c0s, cudaStream_t st) {
    launch_multsum_multi(c, &out, digits, &key, &g, 1, B, level, c0_for_P, c0s, st);
}

// ------------------------------------------------- C^k babies with masks
// For k = n1 g + b (b >= 1) the product's C^k step (Sec. 4.1, Table 1
// "Optimized C^k") needs, over Q_l P,
//   S_b = m_k (.) rot_qp(A_g; b) + m'_k (.) rot_qp(A'_g; b),
// rot_qp(X; b) = <kappa_b(digits of X), rtk_b> + (P kappa_b(c0 of X), 0), m_k
// and m'_k the two column masks (Montgomery form).  The two sources use the
// same rotation keys: each key word is loaded once for both, and the two
// hoisted rotations stay in registers, so only S_b reaches memory.  The
// words equal those of two MultSum launches followed by the masked sum
// (every value is a canonical residue).
template <int G>
struct CkArgs {
    const u64 *key[G];
    u64 *out[G];
    const u64 *m1[G], *m2[G];   // masks over Q_l P, [rows][N]
    u32 ginv[G];
};

template <int G>
__global__ void __launch_bounds__(256, G <= 1 ? 4 : G <= 2 ? 3 : 2)
    k_multsum_ck(const __grid_constant__ CkArgs<G> ck, const u64 *dig1, const u64 *dig2, int B, int BI, int level,
                 int alpha, int L, int ndig, int nprimes, int logN, const ModQ *mods, const u64 *c01,
                 const u64 *c02, long c0s, const ShoupPair *Pmod) {
    const int N = 1 << logN;
    const int XW = 256 / BI;
    const int tx = threadIdx.x % XW, ti = threadIdx.x / XW;
    const int y = blockIdx.x * XW + tx;
    const int r = blockIdx.y;
    const int b = blockIdx.z * BI + ti;
    if (b >= B || y >= N) return;
    const int rows = level + 1 + alpha;
    const int kr = r <= level ? r : L + 1 + (r - level - 1);   // the row's global prime
    const ModQ m = mods[kr];
    const long dstride = (long)rows * N;
    const u64 *dp1 = dig1 + (long)b * ndig * dstride + (long)r * N + y;
    const u64 *dp2 = dig2 + (long)b * ndig * dstride + (long)r * N + y;
    const long koff = (long)kr * N + y, kd = 2L * nprimes * N, kk = (long)nprimes * N;
    U128 acc[G][4];   // (source 1: poly 0, poly 1; source 2: poly 0, poly 1) per key
    if (m.q < (1ull << 42)) {
        // residues below 2^42 (uniform over the CTA): 96-bit accumulation
        u32 x0[4 * G], x1[4 * G], x2[4 * G];
#pragma unroll
        for (int k = 0; k < 4 * G; k++) x0[k] = 0, x1[k] = 0, x2[k] = 0;
        for (int d = 0; d < ndig; d++) {
            const u64 v1 = __ldg(dp1 + (long)d * dstride), v2 = __ldg(dp2 + (long)d * dstride);
#pragma unroll
            for (int k = 0; k < G; k++) {
                const u64 *kp = ck.key[k] + (long)d * kd + koff;
                const u64 k0 = __ldg(kp), k1 = __ldg(kp + kk);
                mac96(x0[4 * k], x1[4 * k], x2[4 * k], v1, k0);
                mac96(x0[4 * k + 1], x1[4 * k + 1], x2[4 * k + 1], v1, k1);
                mac96(x0[4 * k + 2], x1[4 * k + 2], x2[4 * k + 2], v2, k0);
                mac96(x0[4 * k + 3], x1[4 * k + 3], x2[4 * k + 3], v2, k1);
            }
        }
#pragma unroll
        for (int k = 0; k < G; k++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[k][j] = U128{((u64)x1[4 * k + j] << 32) | x0[4 * k + j], x2[4 * k + j]};
    } else {
#pragma unroll
        for (int k = 0; k < G; k++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[k][j] = U128{0, 0};
        for (int d = 0; d < ndig; d++) {
            const u64 v1 = __ldg(dp1 + (long)d * dstride), v2 = __ldg(dp2 + (long)d * dstride);
#pragma unroll
            for (int k = 0; k < G; k++) {
                const u64 *kp = ck.key[k] + (long)d * kd + koff;
                const u64 k0 = __ldg(kp), k1 = __ldg(kp + kk);
                mac128_q(acc[k][0], v1, k0, m.q);
                mac128_q(acc[k][1], v1, k1, m.q);
                mac128_q(acc[k][2], v2, k0, m.q);
                mac128_q(acc[k][3], v2, k1, m.q);
            }
        }
    }
    u64 pc1 = 0, pc2 = 0;
    if (r <= level) {
        const ShoupPair w = Pmod[r];
        pc1 = shoup(c01[b * c0s + (long)r * N + y], w.w, w.wp, m.q);
        pc2 = shoup(c02[b * c0s + (long)r * N + y], w.w, w.wp, m.q);
    }
#pragma unroll
    for (int k = 0; k < G; k++) {
        const u64 a10 = addmod(redc(acc[k][0].lo, acc[k][0].hi, m), pc1, m.q);
        const u64 a11 = redc(acc[k][1].lo, acc[k][1].hi, m);
        const u64 a20 = addmod(redc(acc[k][2].lo, acc[k][2].hi, m), pc2, m.q);
        const u64 a21 = redc(acc[k][3].lo, acc[k][3].hi, m);
        const int x = ck.ginv[k] == 1u ? y : auto_index(y, ck.ginv[k], logN);
        const u64 w1 = __ldg(ck.m1[k] + (long)r * N + x), w2 = __ldg(ck.m2[k] + (long)r * N + x);
        U128 s0 = {0, 0}, s1 = {0, 0};   // two products below q^2: below q 2^64
        mac128(s0, w1, a10);
        mac128(s0, w2, a20);
        mac128(s1, w1, a11);
        mac128(s1, w2, a21);
        u64 *ob = ck.out[k] + (long)b * 2 * rows * N;
        ob[(long)r * N + x] = redc(s0.lo, s0.hi, m);
        ob[(long)(rows + r) * N + x] = redc(s1.lo, s1.hi, m);
    }
}

// The same with the rotations split over the warps: warp w takes rotation
// w / BI of items blockIdx.z BI + w % BI (BI = 8 / G), two adjacent
// coefficients per thread with 16-byte digit, key and store accesses, so a
// thread holds 8 accumulators whatever G is (more resident warps than
// k_multsum_ck at G >= 2).
template <int G>
__global__ void __launch_bounds__(256, 3)
    k_multsum_cks(const __grid_constant__ CkArgs<G> ck, const u64 *dig1, const u64 *dig2, int B, int level,
                  int alpha, int L, int ndig, int nprimes, int logN, const ModQ *mods, const u64 *c01,
                  const u64 *c02, long c0s, const ShoupPair *Pmod) {
    constexpr int BI = 8 / G;
    const int N = 1 << logN;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int kq = wid / BI, bi = wid % BI;
    // one item per CTA (G = 8): the items are the fastest grid index, so the
    // CTAs of the B items that read the same key words run together
    const int xb = BI == 1 ? (int)(blockIdx.x / B) : (int)blockIdx.x;
    const int y = 2 * (xb * 32 + lane);
    const int r = blockIdx.y;
    const int b = BI == 1 ? (int)(blockIdx.x % B) : (int)blockIdx.z * BI + bi;
    if (b >= B || y >= N) return;
    const int rows = level + 1 + alpha;
    const int kr = r <= level ? r : L + 1 + (r - level - 1);
    const ModQ m = mods[kr];
    const long dstride = (long)rows * N;
    const ulonglong2 *dp1 = (const ulonglong2 *)(dig1 + (long)b * ndig * dstride + (long)r * N + y);
    const ulonglong2 *dp2 = (const ulonglong2 *)(dig2 + (long)b * ndig * dstride + (long)r * N + y);
    const long koff = (long)kr * N + y, kd = 2L * nprimes * N, kk = (long)nprimes * N;
    const u64 *key = ck.key[kq];
    U128 acc[2][4];   // [coefficient][source 1 poly 0, poly 1, source 2 poly 0, poly 1]
    if (m.q < (1ull << 42)) {
        u32 x0[2][4], x1[2][4], x2[2][4];
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
            for (int j = 0; j < 4; j++) x0[c][j] = 0, x1[c][j] = 0, x2[c][j] = 0;
        for (int d = 0; d < ndig; d++) {
            const ulonglong2 v1 = __ldg(dp1 + (long)d * dstride / 2), v2 = __ldg(dp2 + (long)d * dstride / 2);
            const ulonglong2 *kp = (const ulonglong2 *)(key + (long)d * kd + koff);
            const ulonglong2 k0 = __ldg(kp), k1 = __ldg(kp + kk / 2);
            mac96(x0[0][0], x1[0][0], x2[0][0], v1.x, k0.x);
            mac96(x0[1][0], x1[1][0], x2[1][0], v1.y, k0.y);
            mac96(x0[0][1], x1[0][1], x2[0][1], v1.x, k1.x);
            mac96(x0[1][1], x1[1][1], x2[1][1], v1.y, k1.y);
            mac96(x0[0][2], x1[0][2], x2[0][2], v2.x, k0.x);
            mac96(x0[1][2], x1[1][2], x2[1][2], v2.y, k0.y);
            mac96(x0[0][3], x1[0][3], x2[0][3], v2.x, k1.x);
            mac96(x0[1][3], x1[1][3], x2[1][3], v2.y, k1.y);
        }
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[c][j] = U128{((u64)x1[c][j] << 32) | x0[c][j], x2[c][j]};
    } else {
#pragma unroll
        for (int c = 0; c < 2; c++)
#pragma unroll
            for (int j = 0; j < 4; j++) acc[c][j] = U128{0, 0};
        for (int d = 0; d < ndig; d++) {
            const ulonglong2 v1 = __ldg(dp1 + (long)d * dstride / 2), v2 = __ldg(dp2 + (long)d * dstride / 2);
            const ulonglong2 *kp = (const ulonglong2 *)(key + (long)d * kd + koff);
            const ulonglong2 k0 = __ldg(kp), k1 = __ldg(kp + kk / 2);
            mac128_q(acc[0][0], v1.x, k0.x, m.q);
            mac128_q(acc[1][0], v1.y, k0.y, m.q);
            mac128_q(acc[0][1], v1.x, k1.x, m.q);
            mac128_q(acc[1][1], v1.y, k1.y, m.q);
            mac128_q(acc[0][2], v2.x, k0.x, m.q);
            mac128_q(acc[1][2], v2.y, k0.y, m.q);
            mac128_q(acc[0][3], v2.x, k1.x, m.q);
            mac128_q(acc[1][3], v2.y, k1.y, m.q);
        }
    }
    const ShoupPair wP = r <= level ? Pmod[r] : ShoupPair{0, 0};
    u64 *ob = ck.out[kq] + (long)b * 2 * rows * N;
    const u32 gi = ck.ginv[kq];
#pragma unroll
    for (int c = 0; c < 2; c++) {
        const int yc = y + c;
        u64 pc1 = 0, pc2 = 0;
        if (r <= level) {
            pc1 = shoup(c01[b * c0s + (long)r * N + yc], wP.w, wP.wp, m.q);
            pc2 = shoup(c02[b * c0s + (long)r * N + yc], wP.w, wP.wp, m.q);
        }
        const u64 a10 = addmod(redc(acc[c][0].lo, acc[c][0].hi, m), pc1, m.q);
        const u64 a11 = redc(acc[c][1].lo, acc[c][1].hi, m);
        const u64 a20 = addmod(redc(acc[c][2].lo, acc[c][2].hi, m), pc2, m.q);
        const u64 a21 = redc(acc[c][3].lo, acc[c][3].hi, m);
        const int x = gi == 1u ? yc : auto_index(yc, gi, logN);
        const u64 w1 = __ldg(ck.m1[kq] + (long)r * N + x), w2 = __ldg(ck.m2[kq] + (long)r * N + x);
        U128 s0 = {0, 0}, s1 = {0, 0};
        mac128(s0, w1, a10);
        mac128(s0, w2, a20);
        mac128(s1, w1, a11);
        mac128(s1, w2, a21);
        ob[(long)r * N + x] = redc(s0.lo, s0.hi, m);
        ob[(long)(rows + r) * N + x] = redc(s1.lo, s1.hi, m);
    }
}

template <int G>
static void multsum_ck_launch_g(Ctx *c, int BI, u64 *const *outs, const u64 *dig1, const u64 *dig2,
                                const u64 *const *keys, const uint32_t *gs, const u64 *const *m1,
                                const u64 *const *m2, int B, int level, const u64 *c01, const u64 *c02, long c0s,
                                cudaStream_t st) {
    CkArgs<G> ck;
    const u32 M = 2u * (u32)c->N;
    for (int k = 0; k < G; k++) {
        ck.key[k] = keys[k];
        ck.out[k] = outs[k];
        ck.m1[k] = m1[k];
        ck.m2[k] = m2[k];
        u32 g = gs[k], inv = g;   // inverse of the odd g modulo 2N (Newton on 32-bit words)
        for (int it = 0; it < 5; it++) inv *= 2u - g * inv;
        ck.ginv[k] = inv & (M - 1);
    }
    const int rows = level + 1 + c->alpha;
    if constexpr (G > 4) BI = 0;   // eight rotations: the split form only
    if constexpr (8 % G == 0) {
        if (BI == 0) {   // rotations split over the warps
            constexpr int SBI = 8 / G;
            const unsigned xblocks = (unsigned)((c->N / 2 + 31) / 32);
            const dim3 grid = SBI == 1 ? dim3(xblocks * (unsigned)B, (unsigned)rows, 1)
                                       : dim3(xblocks, (unsigned)rows, (unsigned)((B + SBI - 1) / SBI));
            k_multsum_cks<G><<<grid, 256, 0, st>>>(ck, dig1, dig2, B, level, c->alpha, c->L, c->ndig(level),
                                                   c->nprimes, c->logN, c->d_mod, c01, c02, c0s, c->d_Pmod);
            c->n_launch++;
            return;
        }
    }
    if constexpr (G <= 4) {
        if (BI == 0) BI = 8;   // G does not divide the warps
        const int XW = 256 / BI;
        dim3 grid((unsigned)((c->N + XW - 1) / XW), (unsigned)rows, (unsigned)((B + BI - 1) / BI));
        k_multsum_ck<G><<<grid, 256, 0, st>>>(ck, dig1, dig2, B, BI, level, c->alpha, c->L, c->ndig(level),
                                              c->nprimes, c->logN, c->d_mod, c01, c02, c0s, c->d_Pmod);
        c->n_launch++;
    }
}

void launch_multsum_ck(Ctx *c, u64 *const *outs, const u64 *dig1, const u64 *dig2, const u64 *const *keys,
                       const uint32_t *gs, const u64 *const *m1, const u64 *const *m2, int G, int B, int level,
                       const u64 *c01, const u64 *c02, long c0s, cudaStream_t st) {
    if (G <= 0) return;
    const int rows = level + 1 + c->alpha;
    auto run = [&](int chunk, int BI, bool traced) {
        for (int k0 = 0, g = 0; k0 < G; k0 += g) {
            g = std::min(chunk, G - k0);
            if (g > 4 && g != 8) g = 4;   // launches of 1..4 or 8 rotations
            cudaEvent_t e0 = nullptr;
            if (traced) c->trace_begin(0, e0);
            switch (g) {
            case 8: multsum_ck_launch_g<8>(c, 0, outs + k0, dig1, dig2, keys + k0, gs + k0, m1 + k0, m2 + k0, B, level, c01, c02, c0s, st); break;
            case 1: multsum_ck_launch_g<1>(c, BI, outs + k0, dig1, dig2, keys + k0, gs + k0, m1 + k0, m2 + k0, B, level, c01, c02, c0s, st); break;
            case 2: multsum_ck_launch_g<2>(c, BI, outs + k0, dig1, dig2, keys + k0, gs + k0, m1 + k0, m2 + k0, B, level, c01, c02, c0s, st); break;
            case 3: multsum_ck_launch_g<3>(c, BI, outs + k0, dig1, dig2, keys + k0, gs + k0, m1 + k0, m2 + k0, B, level, c01, c02, c0s, st); break;
            default: multsum_ck_launch_g<4>(c, BI, outs + k0, dig1, dig2, keys + k0, gs + k0, m1 + k0, m2 + k0, B, level, c01, c02, c0s, st); break;
            }
            if (traced) {
                // algorithmic bytes: every key and every mask read once, both
                // sources' digits and c0 read once per item, one output per
                // (item, key)
                const double nd = c->ndig(level), W = (double)c->N * 8.0;
                const double bytes = g * (2.0 * nd * rows + 2.0 * rows) * W +
                                     (double)B * (2.0 * nd * rows * W + 2.0 * (level + 1) * W + g * 2.0 * rows * W);
                c->trace_end(0, e0, bytes, (double)B * nd * rows * c->N * 4.0 * g);
            }
        }
    };
    int chunk = std::min(G, 4), BI = std::min(B, 8);
    while (BI > 1 && BI > B) BI >>= 1;
    if (c->force_multsum >= 0) {
        // a pinned MultSum variant: 96 / 97 (rotations split over the warps)
        // select the split form here too (97: launches of 8 rotations where 8
        // remain), every other one the thread-per-word form
        if (c->force_multsum == 96 || c->force_multsum == 97) BI = 0;
        if (c->force_multsum == 97) chunk = std::min(G, 8);
    } else if (c->autotune) {
        auto key3 = std::make_tuple(level, B, G);
        auto it = c->tune_ck.find(key3);
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cap);
        if (it != c->tune_ck.end()) {
            chunk = it->second >> 8, BI = it->second & 255;
        } else if (cap == cudaStreamCaptureStatusNone) {
            // time every (keys per launch, items per CTA) twice on these very
            // launches (the outputs do not depend on the plan); keep the fastest
            cudaEvent_t a = c->ev_get(), b = c->ev_get();
            float best = 1e30f;
            std::set<std::pair<int, int>> seen;
            for (int ch : {8, 4, 2, 1}) {
                for (int bi : {8, 4, 2, 1, 0}) {   // 0: rotations split over the warps
                    const int cc = std::min(ch, G);
                    int bb = bi;
                    while (bb > 1 && bb > B) bb >>= 1;
                    if (bi == 0 && (8 % cc) && cc <= 4) continue;
                    if (cc > 4 && bi != 0) continue;   // more than 4 rotations: the split form only
                    if (!seen.insert(std::make_pair(cc, bb)).second) continue;
                    float t = 1e30f;
                    for (int rep = 0; rep < 2; rep++) {
                        cudaEventRecord(a, st);
                        run(cc, bb, false);
                        cudaEventRecord(b, st);
                        cudaEventSynchronize(b);
                        float ms = 0;
                        cudaEventElapsedTime(&ms, a, b);
                        t = std::min(t, ms);
                    }
                    if (t < best) best = t, chunk = cc, BI = bb;
                    char line[128];
                    snprintf(line, sizeof line, "multsum_ck level %d B %d G %d chunk %d BI %d ms %.4f\n", level, B,
                             G, cc, bb, t);
                    c->tune_log += line;
                }
            }
            c->ev_free.push_back(a);
            c->ev_free.push_back(b);
            c->tune_ck[key3] = (chunk << 8) | BI;
        }
    }
    run(chunk, BI, true);
}

// ------------------------------------------------------ double hoisting
// S[b][k][r][x] = sum_t ptM_t[r][x] * R_t[b][k][r][x] over Q_l P (one REDC).
struct PtrList {
    const u64 *p[32];
};
// One REDC per output word: up to 32 products below q^2 stay below q 2^64
// for q < 2^59; on wider rows (q_0, the special primes) the sum is kept
// below it term by term (mac128_q).
__global__ void k_pmul_acc(u64 *out, PtrList pts, PtrList R, int nterms, int B, int rows, int N, long Rs,
                           RowMap qp, const ModQ *mods) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long per = (long)rows * N;
    if (idx >= per) return;
    int r = (int)(idx / N);
    const ModQ m = mods[qp.at(r)];
    const bool wide = m.q >= (1ull << 59);   // uniform over the CTA (128 | N)
    for (int b = 0; b < B; b++) {
        U128 a0 = {0, 0}, a1 = {0, 0};
        for (int t = 0; t < nterms; t++) {
            const u64 pv = pts.p[t][idx];
            const u64 *rb = R.p[t] + b * Rs;
            if (wide) {
                mac128_q(a0, pv, rb[idx], m.q);
                mac128_q(a1, pv, rb[per + idx], m.q);
            } else {
                mac128(a0, pv, rb[idx]);
                mac128(a1, pv, rb[per + idx]);
            }
        }
        u64 *ob = out + (long)b * 2 * per;
        ob[idx] = redc(a0.lo, a0.hi, m);
        ob[per + idx] = redc(a1.lo, a1.hi, m);
    }
}
void launch_pmul_acc(Ctx *c, u64 *out, const u64 *const *pts, const u64 *const *R, int nterms, int B, int level,
                     long Rs, cudaStream_t st) {
    PtrList a, b;
    for (int t = 0; t < nterms; t++) { a.p[t] = pts[t]; b.p[t] = R[t]; }
    int rows = level + 1 + c->alpha;
    long n = (long)rows * c->N;
    c->n_launch++;
    k_pmul_acc<<<nblk(n, 128), 128, 0, st>>>(out, a, b, nterms, B, rows, c->N, Rs, c->map_qp(level), c->d_mod);
}

// P * a over Q_l P: rows q_r get (P mod q_r) a_r, the p rows are zero.
// in: [items][l+1][N] (stride in_s), out: [items][l+1+alpha][N] (stride out_s)
__global__ void k_lift_P(u64 *out, const u64 *in, int items, int level, int alpha, int N, long is, long os,
                         const ModQ *mods, const ShoupPair *Pmod) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    int rows = level + 1 + alpha;
    long per = (long)rows * N;
    if (idx >= (long)items * per) return;
    int it = (int)(idx / per);
    long off = idx - (long)it * per;
    int r = (int)(off / N);
    u64 v = 0;
    if (r <= level) {
        ShoupPair w = Pmod[r];
        v = shoup(in[it * is + off], w.w, w.wp, mods[r].q);
    }
    out[it * os + off] = v;
}
void launch_lift_P(Ctx *c, u64 *out_qp, const u64 *in_q, int items, int level, long is, long os, cudaStream_t st) {
    long n = (long)items * (level + 1 + c->alpha) * c->N;
    c->n_launch++;
    k_lift_P<<<nblk(n, 256), 256, 0, st>>>(out_qp, in_q, items, level, c->alpha, c->N, is, os, c->d_mod,
                                           c->d_Pmod);
}

// ------------------------------------------------------------- Rescale
// t_i = [c_l]_{q_l} mod q_i for i < l (coefficient form): the centred residue
// of the last limb (reading of App. A Rescaling: round(c / q_l)).
// last: [items][N]; out: [items][l][N]
__global__ void k_rescale_prep(const u64 *last, u64 *out, int items, int level, int N, const ModQ *mods,
                               const u64 *qlmod) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long)items * N) return;
    int x = (int)(idx % N);
    int it = (int)(idx / N);
    u64 ql = mods[level].q;
    u64 v = last[idx];
    bool neg = v > (ql >> 1);
    for (int i = 0; i < level; i++) {
        u64 q = mods[i].q;
        u64 r = v % q;
        if (neg) r = submod(r, qlmod[i], q);  // v - q_l
        out[((long)it * level + i) * N + x] = r;
    }
}
void launch_rescale_prep(Ctx *c, const u64 *lastcoef, u64 *out, int items, int level, cudaStream_t st) {
    const LevelConsts &L = c->lc(level);
    long n = (long)items * c->N;
    c->n_launch++;
    k_rescale_prep<<<nblk(n, 256), 256, 0, st>>>(lastcoef, out, items, level, c->N, c->d_mod, L.d_rs_qlmod);
}

// out_i = (c_i - t_i) q_l^-1 mod q_i (NTT domain), i < l.
// in: [items][l+1][N] stride is; t: [items][l][N]; out: [items][l][N] stride os
__global__ void k_rescale_final(u64 *out, const u64 *in, const u64 *t, int items, int level, int N, long is, long os,
                                const ModQ *mods, const ShoupPair *inv) {
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long per = (long)level * N;
    if (idx >= (long)items * per) return;
    int it = (int)(idx / per);
    long off = idx - (long)it * per;
    int i = (int)(off / N);
    u64 q = mods[i].q;
    ShoupPair w = inv[i];
    out[it * os + off] = shoup(submod(in[it * is + off], t[idx], q), w.w, w.wp, q);
}
void launch_rescale_final(Ctx *c, u64 *out, const u64 *in, const u64 *t, int items, int level, long is, long os,
                          cudaStream_t st) {
    const LevelConsts &L = c->lc(level);
    long n = (long)items * level * c->N;
    c->n_launch++;
    k_rescale_final<<<nblk(n, 256), 256, 0, st>>>(out, in, t, items, level, c->N, is, os, c->d_mod, L.d_rs_inv);
}

// ------------------------------------------------------------- decrypt
// m = c0 + c1 s on limb q_0 (NTT domain), written into out (u64 view).
__global__ void k_dec_q0(const u64 *c0, const u64 *c1, const u64 *skM, u64 *out, int N, const ModQ *mods) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    const ModQ &m = mods[0];
    out[x] = addmod(c0[x], mulmont(c1[x], skM[x], m), m.q);
}
__global__ void k_centre_q0(const u64 *a, double *out, int N, const ModQ *mods) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= N) return;
    u64 q = mods[0].q, v = a[x];
    out[x] = v > (q >> 1) ? -(double)(q - v) : (double)v;
}

// -------------------------------------------------------------- diagonals
// Slot vector (length S, period n^2) of a permutation-matrix diagonal,
// rotated left by `rot` (mod n^2) and multiplied by `value`:
//   kind 0  Z (sigma), eq. 5, index t in (-n, n)
//   kind 1  T (tau), eq. 6, index t = k n
//   kind 2  G (transpose), index t = (n-1) k, ones where column - row = k
//   kind 3  C^k mask 1 (columns j < n-k); kind 4  C^k mask 2 (j >= n-k)
//   kind 5  all ones (constant)
//   kind 6  first column (j == 0); kind 7  identity (i == j)
//   kind 10 row k (i == k); kind 11 column k (j == k)
__global__ void k_diag_fill(double *out, int S, int kind, int n, long t, long rot, double value, int k) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= S) return;
    long n2 = (long)n * n;
    long l = ((long)(p % n2) + rot) % n2;
    long i = l / n, j = l % n;
    bool one = false;
    switch (kind) {
    case 0:
        if (t >= 0) one = (l - n * t >= 0) && (l - n * t < n - t);
        else one = (l - (n + t) * n >= -t) && (l - (n + t) * n < n);
        break;
    case 1: one = (j == t / n); break;
    case 2: one = ((j - i) * (n - 1) == t); break;
    case 3: one = j < n - k; break;
    case 4: one = j >= n - k; break;
    case 5: one = true; break;
    case 6: one = (j == 0); break;
    case 7: one = (i == j); break;
    case 10: one = (i == k); break;
    case 11: one = (j == k); break;
    }
    out[p] = one ? value : 0.0;
}
void launch_diag_fill(Ctx *c, double *out, int kind, int n, long t, long rot, double value, int k, cudaStream_t st) {
    c->n_launch++;
    k_diag_fill<<<nblk(c->S, 256), 256, 0, st>>>(out, c->S, kind, n, t, rot, value, k);
}

void launch_copy_rows(u64 *dst, long dst_stride, const u64 *src, long src_stride, int items, long words,
                      cudaStream_t st) {
    cudaMemcpy2DAsync(dst, dst_stride * 8, src, src_stride * 8, words * 8, items, cudaMemcpyDeviceToDevice, st);
}

}  // namespace he

// exported for decrypt
namespace he {
void launch_dec_q0(Ctx *c, const u64 *c0, const u64 *c1, u64 *out, cudaStream_t st) {
    c->n_launch++;
    k_dec_q0<<<nblk(c->N, 256), 256, 0, st>>>(c0, c1, c->d_skM, out, c->N, c->d_mod);
}
void launch_centre_q0(Ctx *c, const u64 *a, double *out, cudaStream_t st) {
    c->n_launch++;
    k_centre_q0<<<nblk(c->N, 256), 256, 0, st>>>(a, out, c->N, c->d_mod);
}
}  // namespace he
