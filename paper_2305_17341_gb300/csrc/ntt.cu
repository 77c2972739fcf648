// ntt.cu -- batched negacyclic number-theoretic transforms over RNS limbs.
//
// The polynomial products of full-RNS CKKS (App. A; "RNS and NTT domains",
// Sec. 3.2) are evaluated pointwise after a negacyclic NTT of every limb.
// Decompose and ModDown (Sec. 3.3) spend most of their time here.
//
// Forward: Cooley-Tukey with the 2N-th root psi merged in (twiddle psi^brv(k)),
// natural order in, bit-reversed order out; evaluation point of output j is
// psi^(2 brv(j) + 1).  Inverse: Gentleman-Sande with psi^-brv(k), bit-reversed
// in, natural out, times N^-1.  Harvey's lazy butterflies keep values in
// [0, 4q) (forward) / [0, 2q) (inverse) between stages; the output is in [0, q).
// The register-blocked kernels for logN 14..16 go lazier: the forward skips
// the per-stage reduction on primes below 2^57 and the inverse keeps values
// in [0, 4q), both with a truncated-quotient Shoup product.
//
// Each limb of N = N1 * N2 coefficients is transformed in two passes: pass 1
// runs the stages whose butterfly span is >= N2 on column tiles (elements with
// equal index mod N2, C columns per CTA, staged in shared memory); pass 2 runs
// the remaining log2(N2) stages on rows of N2 contiguous coefficients.  Both
// passes read and write HBM once.
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <stdexcept>

#include "bulkcopy.cuh"
#include "he_internal.h"

namespace he {

__device__ __forceinline__ void bf_fwd(u64 &x, u64 &y, u64 w, u64 wp, u64 q) {
    u64 tq = 2 * q;
    u64 a = x >= tq ? x - tq : x;
    u64 t = shoup_lazy(y, w, wp, q);
    x = a + t;
    y = a - t + tq;
}

__device__ __forceinline__ void bf_inv(u64 &x, u64 &y, u64 w, u64 wp, u64 q) {
    u64 tq = 2 * q;
    u64 s = x + y;
    s = s >= tq ? s - tq : s;
    u64 d = x - y + tq;
    x = s;
    y = shoup_lazy(d, w, wp, q);
}

// Inverse butterfly on values in [0, 4q): s = x + y reduced below 4q,
// y' = w (x - y + 4q) with the truncated-quotient Shoup product, in [0, 4q)
// (8q < 2^64 for every prime below 2^61).
__device__ __forceinline__ void bf_inv4(u64 &x, u64 &y, u64 w, u64 wp, u64 q) {
    const u64 fq = 4 * q;
    u64 s = x + y;
    s = s >= fq ? s - fq : s;
    const u64 d = x - y + fq;
    x = s;
    y = shoup_lazy4(d, w, wp, q);
}

// ---------------------------------------------------------------- forward
__global__ void k_ntt_fwd_p1(u64 *data, RowMap rm, const ModQ *mods, const u64 *tw, const u64 *twp,
                             int logN, int logN1, int C) {
    extern __shared__ u64 sm[];
    const int N = 1 << logN, N1 = 1 << logN1, N2 = N >> logN1;
    const long row = blockIdx.y;
    const int pidx = rm.at(row);
    const u64 q = mods[pidx].q;
    u64 *base = data + row * (long)N + (long)blockIdx.x * C;
    const u64 *w = tw + (long)pidx * N, *wp = twp + (long)pidx * N;
    for (int e = threadIdx.x; e < N1 * C; e += blockDim.x) {
        int r = e / C, c = e - r * C;
        sm[e] = base[(long)r * N2 + c];
    }
    __syncthreads();
    for (int m = 1, t1 = N1 >> 1; m < N1; m <<= 1, t1 >>= 1) {
        for (int e = threadIdx.x; e < (N1 >> 1) * C; e += blockDim.x) {
            int b = e / C, c = e - b * C;
            int i = b / t1, k = b - i * t1;
            int hi = 2 * i * t1 + k;
            u64 x = sm[hi * C + c], y = sm[(hi + t1) * C + c];
            bf_fwd(x, y, w[m + i], wp[m + i], q);
            sm[hi * C + c] = x;
            sm[(hi + t1) * C + c] = y;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < N1 * C; e += blockDim.x) {
        int r = e / C, c = e - r * C;
        base[(long)r * N2 + c] = sm[e];
    }
}

__global__ void k_ntt_fwd_p2(u64 *data, RowMap rm, const ModQ *mods, const u64 *tw, const u64 *twp,
                             int logN, int logN1, int R) {
    extern __shared__ u64 sm[];
    const int N = 1 << logN, N1 = 1 << logN1, N2 = N >> logN1;
    const long row = blockIdx.y;
    const int pidx = rm.at(row);
    const u64 q = mods[pidx].q;
    const int hi0 = blockIdx.x * R;
    u64 *base = data + row * (long)N + (long)hi0 * N2;
    const u64 *w = tw + (long)pidx * N, *wp = twp + (long)pidx * N;
    for (int e = threadIdx.x; e < R * N2; e += blockDim.x) sm[e] = base[e];
    __syncthreads();
    const int half = N2 >> 1;
    for (int m = N1, t = N2 >> 1; t >= 1; m <<= 1, t >>= 1) {
        for (int e = threadIdx.x; e < R * half; e += blockDim.x) {
            int rr = e / half, b = e - rr * half;
            int il = b / t, k = b - il * t;
            int j = 2 * il * t + k;
            int gi = (hi0 + rr) * (N2 / (2 * t)) + il;
            u64 *s = sm + rr * N2;
            u64 x = s[j], y = s[j + t];
            bf_fwd(x, y, w[m + gi], wp[m + gi], q);
            s[j] = x;
            s[j + t] = y;
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < R * N2; e += blockDim.x) base[e] = reduce4q(sm[e], q);
}

// ---------------------------------------------------------------- inverse
__global__ void k_ntt_inv_p2(u64 *data, RowMap rm, const ModQ *mods, const u64 *tw, const u64 *twp,
                             int logN, int logN1, int R) {
    extern __shared__ u64 sm[];
    const int N = 1 << logN, N1 = 1 << logN1, N2 = N >> logN1;
    const long row = blockIdx.y;
    const int pidx = rm.at(row);
    const u64 q = mods[pidx].q;
    const int hi0 = blockIdx.x * R;
    u64 *base = data + row * (long)N + (long)hi0 * N2;
    const u64 *w = tw + (long)pidx * N, *wp = twp + (long)pidx * N;
    for (int e = threadIdx.x; e < R * N2; e += blockDim.x) sm[e] = base[e];
    __syncthreads();
    const int half = N2 >> 1;
    for (int t = 1; t < N2; t <<= 1) {
        int m = N / (2 * t);
        for (int e = threadIdx.x; e < R * half; e += blockDim.x) {
            int rr = e / half, b = e - rr * half;
            int il = b / t, k = b - il * t;
            int j = 2 * il * t + k;
            int gi = (hi0 + rr) * (N2 / (2 * t)) + il;
            u64 *s = sm + rr * N2;
            u64 x = s[j], y = s[j + t];
            bf_inv(x, y, w[m + gi], wp[m + gi], q);
            s[j] = x;
            s[j + t] = y;
        }
        __syncthreads();
    }
    (void)N1;
    for (int e = threadIdx.x; e < R * N2; e += blockDim.x) base[e] = sm[e];
}

__global__ void k_ntt_inv_p1(u64 *data, RowMap rm, const ModQ *mods, const u64 *tw, const u64 *twp,
                             const u64 *ninv, int logN, int logN1, int C) {
    extern __shared__ u64 sm[];
    const int N = 1 << logN, N1 = 1 << logN1, N2 = N >> logN1;
    const long row = blockIdx.y;
    const int pidx = rm.at(row);
    const u64 q = mods[pidx].q;
    u64 *base = data + row * (long)N + (long)blockIdx.x * C;
    const u64 *w = tw + (long)pidx * N, *wp = twp + (long)pidx * N;
    for (int e = threadIdx.x; e < N1 * C; e += blockDim.x) {
        int r = e / C, c = e - r * C;
        sm[e] = base[(long)r * N2 + c];
    }
    __syncthreads();
    for (int t1 = 1; t1 < N1; t1 <<= 1) {
        int m = N1 / (2 * t1);
        for (int e = threadIdx.x; e < (N1 >> 1) * C; e += blockDim.x) {
            int b = e / C, c = e - b * C;
            int i = b / t1, k = b - i * t1;
            int hi = 2 * i * t1 + k;
            u64 x = sm[hi * C + c], y = sm[(hi + t1) * C + c];
            bf_inv(x, y, w[m + i], wp[m + i], q);
            sm[hi * C + c] = x;
            sm[(hi + t1) * C + c] = y;
        }
        __syncthreads();
    }
    const u64 ni = ninv[2 * pidx], nip = ninv[2 * pidx + 1];
    for (int e = threadIdx.x; e < N1 * C; e += blockDim.x) {
        int r = e / C, c = e - r * C;
        base[(long)r * N2 + c] = shoup(sm[e], ni, nip, q);
    }
}

// ------------------------------------------------- register-blocked passes
// One pass transforms W independent length-M sequences per CTA (M = 2^LM,
// 128 or 256).  Each of the T = M/16 threads of a sequence holds 16 elements:
// layout A = elements t + T k (k < 16), which covers the 4 stages with spans
// M/2 .. T in registers; a shared-memory transpose gives layout B = elements
// 16 t + k, which covers spans T/2 .. 1.  ROWS: sequences are rows of M
// contiguous coefficients (the last stages of a limb); otherwise columns
// with stride N/M (the first stages).  The twiddle of the butterfly at local
// span sp and local group i is psi^brv((M / 2sp) G + i), G = 1 for columns
// and G = N/M + row for rows.  Global loads and stores are always in layout A
// (coalesced across the W sequences for columns, along the row for rows).
// Rows keep each sequence contiguous in shared memory with one pad word per
// 16 (element r at r + r/16): both layouts are free of bank conflicts, and
// every access is a compile-time offset from a per-thread base (17 t + k in
// layout B, t + T k + k T/16 in layout A).
template <int LM, bool ROWS>
struct PassGeom {
    static constexpr int M = 1 << LM, T = M / 16, W = 256 / T;
    static constexpr int SM = ROWS ? W * (M + M / 16) : W * M;
    __device__ static __forceinline__ int sidx(int r, int w) {
        if (ROWS) return w * (M + M / 16) + r + (r >> 4);
        return r * W + w;
    }
};

// Forward butterfly without the reduction of x: x' = x + t, y' = x - t + 4q
// (t = w y mod q in [0, 4q), Shoup's product with the truncated quotient).
// Both outputs grow by less than 4q per stage, so from inputs below 4q the
// 16 stages of a limb stay below 68q < 2^64 for every prime below 2^57 (all
// the 40-bit levels); larger primes use bf_fwd.
__device__ __forceinline__ void bf_fwd_nored(u64 &x, u64 &y, u64 w, u64 wp, u64 q) {
    u64 t = shoup_lazy4(y, w, wp, q);
    u64 a = x;
    x = a + t;
    y = a - t + 4 * q;
}

// Barrier of the threads that run the butterflies: the whole CTA, or the
// 256 consumer threads (named barrier 1) of a CTA that also has a producer warp.
template <bool CONS>
__device__ __forceinline__ void pass_sync() {
    if (CONS) asm volatile("bar.sync 1, 256;" ::: "memory");
    else __syncthreads();
}

// The 8 stages of one pass (4 in registers in layout A, a shared-memory
// transpose, 4 in layout B), leaving the result in shared memory (layout B).
template <int LM, bool ROWS, bool RED, bool CONS = false>
__device__ __forceinline__ void fwd_pass_body(u64 (&x)[16], u64 *sm, const ulonglong2 *w2_, long G, int t, int w,
                                              u64 q) {
    typedef PassGeom<LM, ROWS> G_;
    constexpr int M = G_::M, T = G_::T;
#pragma unroll
    for (int s = 8; s >= 1; s >>= 1) {
        const long mb = (long)(M / (2 * T * s)) * G;
#pragma unroll
        for (int k = 0; k < 16; k++)
            if (!(k & s)) {
                const ulonglong2 wv = __ldg(w2_ + mb + k / (2 * s));
                if (RED) bf_fwd(x[k], x[k + s], wv.x, wv.y, q);
                else bf_fwd_nored(x[k], x[k + s], wv.x, wv.y, q);
            }
    }
#pragma unroll
    for (int k = 0; k < 16; k++) sm[G_::sidx(t + T * k, w)] = x[k];
    pass_sync<CONS>();
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = sm[G_::sidx(16 * t + k, w)];
#pragma unroll
    for (int sp = T / 2; sp >= 1; sp >>= 1) {
        const long mb = (long)(M / (2 * sp)) * G + (long)t * (8 / sp);
#pragma unroll
        for (int k = 0; k < 16; k++)
            if (!(k & sp)) {
                const ulonglong2 wv = __ldg(w2_ + mb + k / (2 * sp));
                if (RED) bf_fwd(x[k], x[k + sp], wv.x, wv.y, q);
                else bf_fwd_nored(x[k], x[k + sp], wv.x, wv.y, q);
            }
    }
#pragma unroll
    for (int k = 0; k < 16; k++) sm[G_::sidx(16 * t + k, w)] = x[k];
    pass_sync<CONS>();
}

template <int LM, bool ROWS, int MINB, bool SUBSC>
__global__ void __launch_bounds__(256, MINB) k_ntt_fwd_fast(u64 *data, RowMap rm, const ModQ *mods,
                                                            const ulonglong2 *tw2, int logN, RowSkip skip,
                                                            SubScale ep) {
    typedef PassGeom<LM, ROWS> G_;
    constexpr int M = G_::M, T = G_::T, W = G_::W;
    __shared__ u64 sm[G_::SM];
    const int N = 1 << logN;
    const long row = blockIdx.y;
    if (skip.skip(row)) return;  // uniform over the CTA
    const int pidx = rm.at(row);
    const u64 q = mods[pidx].q;
    const ulonglong2 *w2_ = tw2 + (long)pidx * N;
    int t, w;
    if (ROWS) { w = threadIdx.x / T; t = threadIdx.x % T; }
    else { t = threadIdx.x / W; w = threadIdx.x % W; }
    const long stride = ROWS ? 1 : (N >> LM);
    const long seq = (long)blockIdx.x * W + w;
    u64 *p = data + row * (long)N + (ROWS ? seq * M : seq);
    const long G = ROWS ? ((long)(N >> LM) + seq) : 1;
    if (ROWS && SUBSC && threadIdx.x == 0) {
        // the epilogue's operands (this CTA's W sequences of u, and of the
        // addend) are contiguous: have the copy engine bring them into L2
        // while the butterflies run, so the epilogue does not wait on DRAM
        const long arow = ep.row0 + row, it = arow / ep.rows_per_item;
        const long off = (arow - it * ep.rows_per_item) * (long)N + (long)blockIdx.x * W * M;
        bc_prefetch_l2(ep.u + it * ep.us + off, W * M * 8);
        if (ep.add) bc_prefetch_l2(ep.add + it * ep.as + off, W * M * 8);
    }
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = p[(long)(t + T * k) * stride];
    const bool red = q >= (1ull << 57);   // uniform over the CTA
    if (red) fwd_pass_body<LM, ROWS, true>(x, sm, w2_, G, t, w, q);
    else fwd_pass_body<LM, ROWS, false>(x, sm, w2_, G, t, w, q);
    // the row pass ends with exact residues: [0, 4q) after reducing
    // butterflies, below 68q after the others
    const u64 wone = mods[pidx].wone;
    if (ROWS && SUBSC) {
        const long arow = ep.row0 + row;
        const long it = arow / ep.rows_per_item;
        const int r = (int)(arow - it * ep.rows_per_item);
        const ShoupPair wr = ep.w[r];
        const long off = (long)r * N + seq * M;
        const u64 *up = ep.u + it * ep.us + off;
        u64 *op = ep.out + it * ep.os + off;
        const u64 *ap = ep.add ? ep.add + it * ep.as + off : nullptr;
#pragma unroll
        for (int k = 0; k < 16; k++) {
            const u64 s = sm[G_::sidx(t + T * k, w)];
            const u64 v = red ? reduce4q(s, q) : reduce_any(s, q, wone);
            u64 o = shoup(submod(up[t + T * k], v, q), wr.w, wr.wp, q);
            if (ap) o = addmod(o, ap[t + T * k], q);
            op[t + T * k] = o;
        }
        return;
    }
    // the store addresses are formed again here from an opaque copy of the
    // base, so that the 16 strided load addresses of the columns are not
    // kept live through the butterflies
    u64 *ps = p;
    asm volatile("" : "+l"(ps));
#pragma unroll
    for (int k = 0; k < 16; k++) {
        u64 v = sm[G_::sidx(t + T * k, w)];
        if (ROWS) v = red ? reduce4q(v, q) : reduce_any(v, q, wone);
        ps[(long)(t + T * k) * stride] = v;
    }
}

template <int LM, bool ROWS, int MINB>
__global__ void __launch_bounds__(256, MINB) k_ntt_inv_fast(u64 *data, RowMap rm, const ModQ *mods,
                                                            const ulonglong2 *tw2, const u64 *ninv, int logN) {
    typedef PassGeom<LM, ROWS> G_;
    constexpr int M = G_::M, T = G_::T, W = G_::W;
    __shared__ u64 sm[G_::SM];
    const int N = 1 << logN;
    const long row = blockIdx.y;
    const int pidx = rm.at(row);
    const u64 q = mods[pidx].q;
    const ulonglong2 *w2_ = tw2 + (long)pidx * N;
    int t, w;
    if (ROWS) { w = threadIdx.x / T; t = threadIdx.x % T; }
    else { t = threadIdx.x / W; w = threadIdx.x % W; }
    const long stride = ROWS ? 1 : (N >> LM);
    const long seq = (long)blockIdx.x * W + w;
    u64 *p = data + row * (long)N + (ROWS ? seq * M : seq);
    const long G = ROWS ? ((long)(N >> LM) + seq) : 1;
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) sm[G_::sidx(t + T * k, w)] = p[(long)(t + T * k) * stride];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = sm[G_::sidx(16 * t + k, w)];
#pragma unroll
    for (int sp = 1; sp <= T / 2; sp <<= 1) {
        const long mb = (long)(M / (2 * sp)) * G + (long)t * (8 / sp);
#pragma unroll
        for (int k = 0; k < 16; k++)
            if (!(k & sp)) {
                const ulonglong2 w = __ldg(w2_ + mb + k / (2 * sp));
                bf_inv4(x[k], x[k + sp], w.x, w.y, q);
            }
    }
#pragma unroll
    for (int k = 0; k < 16; k++) sm[G_::sidx(16 * t + k, w)] = x[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = sm[G_::sidx(t + T * k, w)];
#pragma unroll
    for (int s = 1; s <= 8; s <<= 1) {
        const long mb = (long)(M / (2 * T * s)) * G;
#pragma unroll
        for (int k = 0; k < 16; k++)
            if (!(k & s)) {
                const ulonglong2 w = __ldg(w2_ + mb + k / (2 * s));
                bf_inv4(x[k], x[k + s], w.x, w.y, q);
            }
    }
    if (!ROWS) {
        const u64 ni = ninv[2 * pidx], nip = ninv[2 * pidx + 1];
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = shoup(x[k], ni, nip, q);
    }
#pragma unroll
    for (int k = 0; k < 16; k++) p[(long)(t + T * k) * stride] = x[k];
}

// ------------------------------------------ persistent passes, bulk copies
// The same passes (butterflies, stages and lazy reductions as k_ntt_fwd_fast,
// so the same words) on persistent CTAs whose input tiles arrive through the
// copy engine: a producer warp loads tile i + 1 (a 32 KiB contiguous run of
// W sequences for the row pass; a W-column x M-row box of a 2-D tensor map
// for the column pass) into one of two shared buffers while the 256 consumer
// threads transform tile i, so the load latency that stalls the one-tile
// CTAs is off the critical path.  Rows that a RowSkip excludes are not in the
// tile sequence at all.  Waits are bounded (see bulkcopy.cuh); a wait that
// runs out sets *err, and the consumers stop together after a vote taken on
// their own barrier, so no consumer is left at a barrier.
constexpr int NTC_CONS = 256, NTC_THREADS = NTC_CONS + 32, NTC_STAGES = 2, NTC_TILE = 4096;

// The tiles of a launch: every transformed row, in order, tpr tiles each.
struct NttTiles {
    long rows = 0;   // rows transformed (those a RowSkip keeps)
    int tpr = 0;     // tiles per row
    RowSkip sk;      // rows_per_digit == 0: no row is skipped
    // Absolute row (within the launch) of the ridx-th transformed row: in
    // Decompose output [item][digit][rows_per_digit], digit d skips its own
    // rows [d alpha, min(d alpha + alpha, nq)).
    __device__ __forceinline__ long row_of(long ridx) const {
        if (!sk.rows_per_digit) return ridx;
        const int rpd = sk.rows_per_digit, nd = sk.ndig, a = sk.alpha;
        const long per_item = (long)nd * rpd - sk.nq;
        const long item = ridx / per_item;
        const long rem = ridx - item * per_item, first = (long)(nd - 1) * (rpd - a);
        int d;
        long j;
        if (rem < first) {
            d = (int)(rem / (rpd - a));
            j = rem - (long)d * (rpd - a);
        } else {
            d = nd - 1;
            j = rem - first;
        }
        const int i0 = d * a, kd = d < nd - 1 ? a : sk.nq - i0;
        return (item * nd + d) * rpd + (j < i0 ? j : j + kd);
    }
};

template <int LM, bool ROWS, bool SUBSC>
__global__ void __launch_bounds__(NTC_THREADS, 2)
    k_ntt_fwd_tma(u64 *data, const __grid_constant__ CUtensorMap tmap, RowMap rm, const ModQ *mods,
                  const ulonglong2 *tw2, int logN, NttTiles tl, SubScale ep, int *err) {
    typedef PassGeom<LM, ROWS> G_;
    constexpr int M = G_::M, T = G_::T, W = G_::W;
    static_assert(W * M == NTC_TILE, "a tile is 4096 words");
    extern __shared__ __align__(128) u64 ntc_dyn[];
    u64 *stage = ntc_dyn;                       // [NTC_STAGES][NTC_TILE], dense
    u64 *sm = ntc_dyn + NTC_STAGES * NTC_TILE;  // transpose scratch, G_::SM words
    __shared__ __align__(8) u64 full[NTC_STAGES], empty[NTC_STAGES];
    __shared__ volatile int stop, cons_fail;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < NTC_STAGES; s++) {
            bc_bar_init(&full[s], 1);
            bc_bar_init(&empty[s], NTC_CONS / 32);
        }
        stop = 0;
        cons_fail = 0;
        bc_init_fence();
    }
    __syncthreads();
    const int N = 1 << logN;
    const long ntiles = tl.rows * tl.tpr;
    const long per_cta = ntiles > (long)blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    if (tid >= NTC_CONS) {
        // producer warp: one lane loads each tile once its buffer is free
        if (tid != NTC_CONS) return;
        long jj = 0;
        for (; jj < per_cta; jj++) {
            const int s = (int)(jj % NTC_STAGES);
            if (jj >= NTC_STAGES && !bc_wait(&empty[s], (u32)(((jj / NTC_STAGES) - 1) & 1))) {
                stop = 1;
                atomicExch(err, 1);
                break;
            }
            if (stop) break;
            const long u = (long)blockIdx.x + jj * (long)gridDim.x;
            const long row = tl.row_of(u / tl.tpr);
            const int tr = (int)(u % tl.tpr);
            u64 *dst = stage + (long)s * NTC_TILE;
            bc_expect_tx(&full[s], NTC_TILE * 8);
            if (ROWS) {
                const u64 *src = data + row * (long)N + (long)tr * NTC_TILE;
#pragma unroll
                for (int k = 0; k < 4; k++) bc_bulk(dst + k * 1024, src + k * 1024, 8192, &full[s]);
            } else {
                bc_tensor2d(dst, &tmap, tr * W, (int)(row * M), &full[s]);
            }
        }
        // copies still in flight land before the CTA's shared memory goes
        for (long k = (jj > NTC_STAGES ? jj - NTC_STAGES : 0); k < jj; k++)
            bc_wait(&full[k % NTC_STAGES], (u32)((k / NTC_STAGES) & 1));
        return;
    }
    int t, w;
    if (ROWS) {
        w = tid / T;
        t = tid % T;
    } else {
        t = tid / W;
        w = tid % W;
    }
    const long stride = ROWS ? 1 : (N >> LM);
    for (long jj = 0; jj < per_cta; jj++) {
        const int s = (int)(jj % NTC_STAGES);
        if (!bc_wait(&full[s], (u32)((jj / NTC_STAGES) & 1))) {
            cons_fail = 1;
            atomicExch(err, 1);
        }
        if (stop) cons_fail = 1;
        // every consumer reads the vote after the barrier: a uniform exit
        pass_sync<true>();
        if (cons_fail) return;
        const long u = (long)blockIdx.x + jj * (long)gridDim.x;
        const long row = tl.row_of(u / tl.tpr);
        const int tr = (int)(u % tl.tpr);
        const u64 *sg = stage + (long)s * NTC_TILE;
        u64 x[16];
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = ROWS ? sg[w * M + t + T * k] : sg[(t + T * k) * W + w];
        __syncwarp();
        if ((tid & 31) == 0) bc_arrive(&empty[s]);
        const int pidx = rm.at(row);
        const u64 q = mods[pidx].q;
        const ulonglong2 *w2_ = tw2 + (long)pidx * N;
        const long seq = (long)tr * W + w;
        u64 *p = data + row * (long)N + (ROWS ? seq * M : seq);
        const long G = ROWS ? ((long)(N >> LM) + seq) : 1;
        const bool red = q >= (1ull << 57);   // uniform over the CTA
        if (red) fwd_pass_body<LM, ROWS, true, true>(x, sm, w2_, G, t, w, q);
        else fwd_pass_body<LM, ROWS, false, true>(x, sm, w2_, G, t, w, q);
        const u64 wone = mods[pidx].wone;
        if (ROWS && SUBSC) {
            const long arow = ep.row0 + row;
            const long it = arow / ep.rows_per_item;
            const int r = (int)(arow - it * ep.rows_per_item);
            const ShoupPair wr = ep.w[r];
            const long off = (long)r * N + seq * M;
            const u64 *up = ep.u + it * ep.us + off;
            u64 *op = ep.out + it * ep.os + off;
            const u64 *ap = ep.add ? ep.add + it * ep.as + off : nullptr;
#pragma unroll
            for (int k = 0; k < 16; k++) {
                const u64 sv = sm[G_::sidx(t + T * k, w)];
                const u64 v = red ? reduce4q(sv, q) : reduce_any(sv, q, wone);
                u64 o = shoup(submod(up[t + T * k], v, q), wr.w, wr.wp, q);
                if (ap) o = addmod(o, ap[t + T * k], q);
                op[t + T * k] = o;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 16; k++) {
                u64 v = sm[G_::sidx(t + T * k, w)];
                if (ROWS) v = red ? reduce4q(v, q) : reduce_any(v, q, wone);
                p[(long)(t + T * k) * stride] = v;
            }
        }
        // the scratch is rewritten by the next tile
        pass_sync<true>();
    }
}

// ---------------------------------------- one pass per limb, 8-CTA clusters
// N = 2^16: the 8 CTAs of a cluster transform one limb with a single read
// and a single write of it.  CTA c loads, from each eighth e of the limb,
// the 1024 words [e 8192 + 1024 c, + 1024) (8 bulk copies of 8 KiB) and
// runs the first three stages (spans N/2, N/4, N/8: the eighths of one
// position) in registers; element (e, p) then belongs to eighth e and is
// stored straight into CTA e's shared memory (distributed shared memory)
// at index 1024 c + p.  After a cluster barrier CTA r holds eighth r and runs
// its 13 remaining stages: 5 in registers on elements t + 256 k, 5 on
// a + 8 k + 256 b, 3 on 32 t + i, each round a shared-memory transpose;
// eighth r's stage-s group g uses twiddle psi^brv(2^s (8 + r) + g).  The
// words are those of the two-pass kernels (same butterflies in the same
// stage order, same lazy bounds: 16 stages from inputs below 4q).  Shared
// rows hold one pad word per 32.  Every CTA passes both cluster barriers on
// every path (a bounded load wait that runs out only flags the error).
constexpr int NCL = 8, NCL_EIGHTH = 8192, NCL_SMEM_WORDS = NCL_EIGHTH + NCL_EIGHTH / 32;

__device__ __forceinline__ int ncl_pad(int l) { return l + (l >> 5); }

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ u32 cluster_rank() {
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Address of `local` (a shared address of this CTA) in CTA `rank`'s shared memory.
__device__ __forceinline__ u32 cluster_map(u32 local, u32 rank) {
    u32 r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_cluster_u64(u32 addr, u64 v) {
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

template <bool RED>
__device__ __forceinline__ void ncl_bf(u64 &x, u64 &y, const ulonglong2 w, u64 q) {
    if (RED) bf_fwd(x, y, w.x, w.y, q);
    else bf_fwd_nored(x, y, w.x, w.y, q);
}

template <bool RED>
__device__ __forceinline__ void ncl_local(u64 *buf, const ulonglong2 *w2_, int r, int t, u64 q) {
    u64 x[32];
    // round A: l = t + 256 k, spans 4096 .. 256 (stages s = 0 .. 4 of the eighth)
#pragma unroll
    for (int k = 0; k < 32; k++) x[k] = buf[ncl_pad(t + 256 * k)];
#pragma unroll
    for (int s = 0; s < 5; s++) {
        const int h = 16 >> s;
#pragma unroll
        for (int k = 0; k < 32; k++)
            if (!(k & h)) ncl_bf<RED>(x[k], x[k + h], __ldg(w2_ + ((8 + r) << s) + (k >> (5 - s))), q);
    }
#pragma unroll
    for (int k = 0; k < 32; k++) buf[ncl_pad(t + 256 * k)] = x[k];
    __syncthreads();
    // round B: l = a + 8 k + 256 b, spans 128 .. 8 (stages 5 .. 9)
    const int a = t & 7, b = t >> 3;
#pragma unroll
    for (int k = 0; k < 32; k++) x[k] = buf[ncl_pad(a + 8 * k + 256 * b)];
#pragma unroll
    for (int sp = 0; sp < 5; sp++) {
        const int h = 16 >> sp;
        const long base = ((long)(8 + r) << (5 + sp)) + ((long)b << sp);
#pragma unroll
        for (int k = 0; k < 32; k++)
            if (!(k & h)) ncl_bf<RED>(x[k], x[k + h], __ldg(w2_ + base + (k >> (5 - sp))), q);
    }
#pragma unroll
    for (int k = 0; k < 32; k++) buf[ncl_pad(a + 8 * k + 256 * b)] = x[k];
    __syncthreads();
    // round C: l = 32 t + i, spans 4, 2, 1 (stages 10 .. 12)
#pragma unroll
    for (int i = 0; i < 32; i++) x[i] = buf[ncl_pad(32 * t + i)];
#pragma unroll
    for (int s = 10; s < 13; s++) {
        const int span = 1 << (12 - s);
        const long base = (long)(8 + r) << s;
#pragma unroll
        for (int i = 0; i < 32; i++)
            if (!(i & span)) ncl_bf<RED>(x[i], x[i + span], __ldg(w2_ + base + ((32 * t + i) >> (13 - s))), q);
    }
#pragma unroll
    for (int i = 0; i < 32; i++) buf[ncl_pad(32 * t + i)] = x[i];
    __syncthreads();
}

template <bool SUBSC>
__global__ void __launch_bounds__(256, 2) k_ntt_fwd_cluster(u64 *data, RowMap rm, const ModQ *mods,
                                                            const ulonglong2 *tw2, RowSkip skip, SubScale ep,
                                                            int *err) {
    constexpr int N = 1 << 16;
    extern __shared__ __align__(128) u64 ncl_buf[];   // NCL_SMEM_WORDS
    __shared__ __align__(8) u64 full;
    const long row = blockIdx.y;
    if (skip.skip(row)) return;   // uniform over the cluster: no cluster barrier is taken
    const int t = threadIdx.x;
    const u32 c = cluster_rank();
    const int pidx = rm.at(row);
    const u64 q = mods[pidx].q, wone = mods[pidx].wone;
    const ulonglong2 *w2_ = tw2 + (long)pidx * N;
    u64 *rowp = data + row * (long)N;
    if (t == 0) {
        bc_bar_init(&full, 1);
        bc_init_fence();
    }
    __syncthreads();
    if (t == 0) {
        bc_expect_tx(&full, 8 * 1024 * 8);
        for (int e = 0; e < 8; e++) bc_bulk(ncl_buf + e * 1024, rowp + e * NCL_EIGHTH + c * 1024, 8192, &full);
    }
    const bool loaded = bc_wait(&full, 0);
    if (!loaded) atomicExch(err, 1);   // the words are garbage then; every barrier is still taken
    const bool red = q >= (1ull << 57);   // uniform over the cluster
    // stages 1-3 on the eighths of positions p = t + 256 j
    u64 x[4][8];
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int e = 0; e < 8; e++) x[j][e] = ncl_buf[e * 1024 + t + 256 * j];
    const ulonglong2 w1 = __ldg(w2_ + 1), w2 = __ldg(w2_ + 2), w3 = __ldg(w2_ + 3), w4 = __ldg(w2_ + 4),
                     w5 = __ldg(w2_ + 5), w6 = __ldg(w2_ + 6), w7 = __ldg(w2_ + 7);
#pragma unroll
    for (int j = 0; j < 4; j++) {
        if (red) {
#pragma unroll
            for (int e = 0; e < 4; e++) ncl_bf<true>(x[j][e], x[j][e + 4], w1, q);
            ncl_bf<true>(x[j][0], x[j][2], w2, q), ncl_bf<true>(x[j][1], x[j][3], w2, q);
            ncl_bf<true>(x[j][4], x[j][6], w3, q), ncl_bf<true>(x[j][5], x[j][7], w3, q);
            ncl_bf<true>(x[j][0], x[j][1], w4, q), ncl_bf<true>(x[j][2], x[j][3], w5, q);
            ncl_bf<true>(x[j][4], x[j][5], w6, q), ncl_bf<true>(x[j][6], x[j][7], w7, q);
        } else {
#pragma unroll
            for (int e = 0; e < 4; e++) ncl_bf<false>(x[j][e], x[j][e + 4], w1, q);
            ncl_bf<false>(x[j][0], x[j][2], w2, q), ncl_bf<false>(x[j][1], x[j][3], w2, q);
            ncl_bf<false>(x[j][4], x[j][6], w3, q), ncl_bf<false>(x[j][5], x[j][7], w3, q);
            ncl_bf<false>(x[j][0], x[j][1], w4, q), ncl_bf<false>(x[j][2], x[j][3], w5, q);
            ncl_bf<false>(x[j][4], x[j][5], w6, q), ncl_bf<false>(x[j][6], x[j][7], w7, q);
        }
    }
    // every CTA has its words in registers before anyone writes into its buffer
    cluster_sync_all();
    const u32 base = bc_smem(ncl_buf);
#pragma unroll
    for (int e = 0; e < 8; e++) {
        const u32 rb = cluster_map(base, (u32)e);
#pragma unroll
        for (int j = 0; j < 4; j++) st_cluster_u64(rb + 8u * (u32)ncl_pad((int)c * 1024 + t + 256 * j), x[j][e]);
    }
    // every CTA's eighth has arrived
    cluster_sync_all();
    if (red) ncl_local<true>(ncl_buf, w2_, (int)c, t, q);
    else ncl_local<false>(ncl_buf, w2_, (int)c, t, q);
    // exact residues, coalesced stores of eighth c (or the fused epilogue)
    const long off0 = (long)c * NCL_EIGHTH;
    if (SUBSC) {
        const long arow = ep.row0 + row;
        const long it = arow / ep.rows_per_item;
        const int rr = (int)(arow - it * ep.rows_per_item);
        const ShoupPair wr = ep.w[rr];
        const long off = (long)rr * N + off0;
        const u64 *up = ep.u + it * ep.us + off;
        u64 *op = ep.out + it * ep.os + off;
        const u64 *ap = ep.add ? ep.add + it * ep.as + off : nullptr;
#pragma unroll 8
        for (int k = 0; k < 32; k++) {
            const int l = t + 256 * k;
            const u64 sv = ncl_buf[ncl_pad(l)];
            const u64 v = red ? reduce4q(sv, q) : reduce_any(sv, q, wone);
            u64 o = shoup(submod(up[l], v, q), wr.w, wr.wp, q);
            if (ap) o = addmod(o, ap[l], q);
            op[l] = o;
        }
    } else {
#pragma unroll 8
        for (int k = 0; k < 32; k++) {
            const int l = t + 256 * k;
            const u64 sv = ncl_buf[ncl_pad(l)];
            rowp[off0 + l] = red ? reduce4q(sv, q) : reduce_any(sv, q, wone);
        }
    }
    // a load that ran out of its wait may still land: wait for it (bounded)
    // before this CTA's shared memory is given back
    if (!loaded && t == 0) bc_wait(&full, 0);
}

// Launches the cluster kernel over nr rows (nr <= 65535); false if no
// cluster of 8 such CTAs fits on the device.
template <bool SUBSC>
static bool ntt_cluster_launch(Ctx *ctx, u64 *d, long nr, const RowMap &m, cudaStream_t st, const RowSkip &sk,
                               const SubScale &e) {
    static int ok[64];   // 0 unknown, 1 fits, -1 does not
    const int dev = ctx->device & 63;
    const size_t smem = (size_t)NCL_SMEM_WORDS * 8;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = NCL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(NCL, (unsigned)nr, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (!ok[dev]) {
        cudaFuncSetAttribute(k_ntt_fwd_cluster<SUBSC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, k_ntt_fwd_cluster<SUBSC>, &cfg) != cudaSuccess) cudaGetLastError();
        ok[dev] = nc > 0 ? 1 : -1;
    }
    if (ok[dev] < 0) return false;
    cudaLaunchKernelEx(&cfg, k_ntt_fwd_cluster<SUBSC>, d, m, (const ModQ *)ctx->d_mod,
                       (const ulonglong2 *)ctx->d_psi2, sk, e, ctx->d_err);
    return true;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !p)
            throw std::runtime_error("cuTensorMapEncodeTiled is not available");
        fn = (EncodeTiledFn)p;
    }
    return fn;
}

// Launch of one persistent pass kernel: its shared-memory attribute and
// occupancy are set up once per device for this very instantiation.
template <int LM, bool ROWS, bool SUBSC>
static void ntt_tma_launch(Ctx *ctx, u64 *d, const CUtensorMap &map, const RowMap &m, cudaStream_t st,
                           const NttTiles &tl, const SubScale &e) {
    typedef PassGeom<LM, ROWS> G_;
    const size_t smem = ((size_t)NTC_STAGES * NTC_TILE + G_::SM) * 8;
    static int occ[64];
    const int dev = ctx->device & 63;
    if (!occ[dev]) {
        cudaFuncSetAttribute(k_ntt_fwd_tma<LM, ROWS, SUBSC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_ntt_fwd_tma<LM, ROWS, SUBSC>, NTC_THREADS, smem);
        occ[dev] = nb > 0 ? nb : 1;
    }
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    const long grid = std::min<long>(tl.rows * tl.tpr, (long)nsm * occ[dev]);
    k_ntt_fwd_tma<LM, ROWS, SUBSC><<<(unsigned)grid, NTC_THREADS, smem, st>>>(
        d, map, m, ctx->d_mod, (const ulonglong2 *)ctx->d_psi2, ctx->logN, tl, e, ctx->d_err);
}

// One pass over all `nr` rows of `d` (no 65535-row split: the grid is
// persistent).  skip: rows left out; ep: the row pass's fused epilogue.
template <int LM, bool ROWS>
static void fwd_pass_tma(Ctx *ctx, u64 *d, long nr, const RowMap &m, cudaStream_t st, const RowSkip &sk,
                         const SubScale *ep) {
    typedef PassGeom<LM, ROWS> G_;
    const int N = ctx->N;
    NttTiles tl;
    tl.sk = sk;
    tl.sk.row0 = 0;
    tl.tpr = (N >> LM) / G_::W;
    tl.rows = nr;
    if (sk.rows_per_digit) {
        const long per_item = (long)sk.ndig * sk.rows_per_digit;
        tl.rows = (nr / per_item) * (per_item - sk.nq);
    }
    if (tl.rows <= 0) return;
    CUtensorMap map;
    std::memset(&map, 0, sizeof map);
    if (!ROWS) {
        // the rows as a (N / M) x (M nr) matrix; a box is W columns x M rows
        const cuuint64_t dims[2] = {(cuuint64_t)(N >> LM), (cuuint64_t)G_::M * (cuuint64_t)nr};
        const cuuint64_t strides[1] = {(cuuint64_t)(N >> LM) * 8};
        const cuuint32_t box[2] = {(cuuint32_t)G_::W, (cuuint32_t)G_::M}, es[2] = {1, 1};
        if (encode_tiled()(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, d, dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            throw std::runtime_error("tensor map encoding failed");
    }
    const SubScale e = ep ? *ep : SubScale();
    if (ROWS && ep) ntt_tma_launch<LM, ROWS, true>(ctx, d, map, m, st, tl, e);
    else ntt_tma_launch<LM, ROWS, false>(ctx, d, map, m, st, tl, e);
}

template <int LM, bool ROWS>
static void fwd_pass(Ctx *ctx, u64 *d, long nr, const RowMap &m, cudaStream_t st, const RowSkip &sk,
                     const SubScale *ep = nullptr) {
    typedef PassGeom<LM, ROWS> G_;
    dim3 grid((unsigned)((ctx->N >> LM) / G_::W), (unsigned)nr);
    const ulonglong2 *t2 = (const ulonglong2 *)ctx->d_psi2;
    const SubScale e = ep ? *ep : SubScale();
    // ntt_minb: 2 or 3 CTAs per SM; 5: 4 CTAs per SM
    if (ROWS && ep) {
        if (ctx->ntt_minb == 3)
            k_ntt_fwd_fast<LM, ROWS, 3, true><<<grid, 256, 0, st>>>(d, m, ctx->d_mod, t2, ctx->logN, sk, e);
        else if (ctx->ntt_minb == 5)
            k_ntt_fwd_fast<LM, ROWS, 4, true><<<grid, 256, 0, st>>>(d, m, ctx->d_mod, t2, ctx->logN, sk, e);
        else
            k_ntt_fwd_fast<LM, ROWS, 2, true><<<grid, 256, 0, st>>>(d, m, ctx->d_mod, t2, ctx->logN, sk, e);
    } else if (ctx->ntt_minb == 3) {
        k_ntt_fwd_fast<LM, ROWS, 3, false><<<grid, 256, 0, st>>>(d, m, ctx->d_mod, t2, ctx->logN, sk, e);
    } else if (ctx->ntt_minb == 5) {
        k_ntt_fwd_fast<LM, ROWS, 4, false><<<grid, 256, 0, st>>>(d, m, ctx->d_mod, t2, ctx->logN, sk, e);
    } else {
        k_ntt_fwd_fast<LM, ROWS, 2, false><<<grid, 256, 0, st>>>(d, m, ctx->d_mod, t2, ctx->logN, sk, e);
    }
}

template <int LM, bool ROWS>
static void inv_pass(Ctx *ctx, u64 *d, long nr, const RowMap &m, cudaStream_t st) {
    typedef PassGeom<LM, ROWS> G_;
    dim3 grid((unsigned)((ctx->N >> LM) / G_::W), (unsigned)nr);
    const ulonglong2 *t2 = (const ulonglong2 *)ctx->d_ipsi2;
    if (ctx->ntt_minb_inv == 3)
        k_ntt_inv_fast<LM, ROWS, 3><<<grid, 256, 0, st>>>(d, m, ctx->d_mod, t2, ctx->d_ninv, ctx->logN);
    else if (ctx->ntt_minb_inv == 5)
        k_ntt_inv_fast<LM, ROWS, 4><<<grid, 256, 0, st>>>(d, m, ctx->d_mod, t2, ctx->d_ninv, ctx->logN);
    else
        k_ntt_inv_fast<LM, ROWS, 2><<<grid, 256, 0, st>>>(d, m, ctx->d_mod, t2, ctx->d_ninv, ctx->logN);
}

// ------------------------------------------------------ integer roofline
// Peak rate of the forward butterfly that the NTT runs on the limbs of every
// prime below 2^57 (one lazy Shoup product with the truncated quotient and
// two lazy add/sub, bf_fwd_nored) with operands in registers: 16 independent
// chains per thread, `iters` rounds, every SM filled.  The values wrap
// modulo 2^64 after a few rounds; only the instruction stream matters.  The
// result is the denominator of the NTT's "alu" roofline.
__global__ void k_bfly_peak(u64 *sink, int iters, u64 q, u64 w, u64 wp) {
    u64 x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = (threadIdx.x * 16 + k) % q;
    for (int it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < 16; k += 2) bf_fwd_nored(x[k], x[k + 1], w, wp, q);
#pragma unroll
        for (int k = 0; k < 16; k += 4) {
            bf_fwd_nored(x[k], x[k + 2], w, wp, q);
            bf_fwd_nored(x[k + 1], x[k + 3], w, wp, q);
        }
    }
    u64 acc = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) acc ^= x[k];
    if (acc == 0x1234567ull) sink[0] = acc;  // keeps the work alive
}

double bfly_peak(int iters) {
    const u64 q = 1099510054913ull;  // a 40-bit prime = 1 mod 2^17
    const u64 w = 123456789012345ull % q;
    ShoupPair sp = h_shoup(w, q);
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    u64 *sink;
    cudaMalloc(&sink, 8);
    const int blocks = nsm * 8, threads = 256;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_bfly_peak<<<blocks, threads>>>(sink, 16, q, sp.w, sp.wp);  // warm-up
    cudaEventRecord(a);
    k_bfly_peak<<<blocks, threads>>>(sink, iters, q, sp.w, sp.wp);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    double bfly = (double)blocks * threads * iters * 16.0;  // 8 + 8 butterflies per round
    return bfly / (ms * 1e-3);
}

// Integer roofline of MultSum: the rate of its inner step on the 40-bit
// limbs, one digit-key product accumulated into 96 bits (mac96: eight 32-bit
// multiply-adds with carries), operands in registers, 16 independent
// accumulators per thread, 8 CTAs of 256 threads per SM.  Only the
// instruction stream matters; the sums are kept alive through a store that
// never happens.
__global__ void k_mac_peak(u64 *sink, int iters, u64 seed) {
    u32 x0[16], x1[16], x2[16];
    u64 kk[16];
    u64 v = (seed ^ threadIdx.x) & ((1ull << 42) - 1);
#pragma unroll
    for (int k = 0; k < 16; k++) x0[k] = x1[k] = x2[k] = 0, kk[k] = (seed * (k + 3)) & ((1ull << 42) - 1);
    for (int it = 0; it < iters; it++) {
        v = (v + 0x9E3779B97F4A7C15ull) & ((1ull << 42) - 1);
#pragma unroll
        for (int k = 0; k < 16; k++) mac96(x0[k], x1[k], x2[k], v, kk[k]);
    }
    u32 acc = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) acc ^= x0[k] ^ x1[k] ^ x2[k];
    if (acc == 0x1234567u) sink[0] = acc;
}

double mac_peak(int iters) {
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    u64 *sink;
    cudaMalloc(&sink, 8);
    const int blocks = nsm * 8, threads = 256;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    k_mac_peak<<<blocks, threads>>>(sink, 16, 12345);   // warm-up
    cudaEventRecord(a);
    k_mac_peak<<<blocks, threads>>>(sink, iters, 12345);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    return (double)blocks * threads * iters * 16.0 / (ms * 1e-3);
}

// ----------------------------------------------------------------- launch
static void split(int logN, int &logN1, int &C, int &R) {
    logN1 = logN / 2;
    int N1 = 1 << logN1, N2 = 1 << (logN - logN1);
    C = 2048 / N1;
    if (C < 1) C = 1;
    if (C > N2) C = N2;
    R = 2048 / N2;
    if (R < 1) R = 1;
    if (R > N1) R = N1;
}

// Both forward passes over nr rows (at most 65535 for the one-tile CTAs
// and the clusters; any number for the persistent ones), with the variant
// the context picked: ntt_minb 2, 3 or 5 (4 CTAs per SM) for one-tile CTAs,
// 4 the persistent passes fed by bulk copies, 6 one pass per limb over
// 8-CTA clusters (N = 2^16).
static void fwd_both(Ctx *ctx, u64 *d, long nr, const RowMap &m, cudaStream_t st, const RowSkip &sk,
                     const SubScale *ep) {
    int logN1, C, R;
    split(ctx->logN, logN1, C, R);
    if (ctx->ntt_minb == 6 && ctx->logN == 16) {
        // one pass per limb over 8-CTA clusters (N = 2^16)
        const SubScale e = ep ? *ep : SubScale();
        const bool done = ep ? ntt_cluster_launch<true>(ctx, d, nr, m, st, sk, e)
                             : ntt_cluster_launch<false>(ctx, d, nr, m, st, sk, e);
        if (done) return;
        ctx->ntt_minb = 3;   // no cluster fits: the one-tile passes from now on
    }
    const bool rows8 = ctx->logN - logN1 == 8;
    if (ctx->ntt_minb == 4) {
        if (logN1 == 8) fwd_pass_tma<8, false>(ctx, d, nr, m, st, sk, nullptr);
        else fwd_pass_tma<7, false>(ctx, d, nr, m, st, sk, nullptr);
        if (rows8) fwd_pass_tma<8, true>(ctx, d, nr, m, st, sk, ep);
        else fwd_pass_tma<7, true>(ctx, d, nr, m, st, sk, ep);
        return;
    }
    if (logN1 == 8) fwd_pass<8, false>(ctx, d, nr, m, st, sk); else fwd_pass<7, false>(ctx, d, nr, m, st, sk);
    if (rows8) fwd_pass<8, true>(ctx, d, nr, m, st, sk, ep); else fwd_pass<7, true>(ctx, d, nr, m, st, sk, ep);
}

// Picks the register budget of the register-blocked passes (2 or 3 CTAs per
// SM) by timing a forward and an inverse transform of 256 scratch rows with
// each; runs once per context, outside stream capture.
// Picks the CTAs per SM (2 or 3) of the register-blocked passes, forward
// and inverse separately: each variant transforms 1024 rows over the
// context's whole chain (the 40-bit limbs run the non-reducing butterflies,
// as in Decompose), 3 repetitions, fastest kept.
static void tune_ntt(Ctx *ctx, cudaStream_t st) {
    ctx->ntt_tuned = true;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    if (cap != cudaStreamCaptureStatusNone) {
        ctx->ntt_tuned = false;
        return;
    }
    const long R = 1024;
    Buf scratch(&ctx->pool, (size_t)R * ctx->N);
    // any words do for timing; 0x15.. keeps them below the 60-bit primes
    cudaMemsetAsync(scratch.p, 0x15, (size_t)R * ctx->N * 8, st);
    int logN1, C, Rr;
    split(ctx->logN, logN1, C, Rr);
    RowMap m = ctx->map_qp(ctx->L);
    RowSkip none;
    cudaEvent_t a = ctx->ev_get(), b = ctx->ev_get();
    for (int dir = 0; dir < 2; dir++) {
        float best = 1e30f;
        int pick = 2;
        for (int minb : {2, 3, 5, 4, 6}) {
            if (dir == 1 && (minb == 4 || minb == 6)) continue;   // 4, 6: forward only
            if (minb == 6 && ctx->logN != 16) continue;            // the cluster pass is for N = 2^16
            (dir == 0 ? ctx->ntt_minb : ctx->ntt_minb_inv) = minb;
            float t = 1e30f;
            for (int rep = 0; rep < 3; rep++) {
                cudaEventRecord(a, st);
                if (dir == 0) {
                    fwd_both(ctx, scratch.p, R, m, st, none, nullptr);
                } else {
                    if (ctx->logN - logN1 == 8) inv_pass<8, true>(ctx, scratch.p, R, m, st); else inv_pass<7, true>(ctx, scratch.p, R, m, st);
                    if (logN1 == 8) inv_pass<8, false>(ctx, scratch.p, R, m, st); else inv_pass<7, false>(ctx, scratch.p, R, m, st);
                }
                cudaEventRecord(b, st);
                cudaEventSynchronize(b);
                float ms = 0;
                cudaEventElapsedTime(&ms, a, b);
                t = std::min(t, ms);
                ctx->n_launch += 2;
            }
            char line[112];
            snprintf(line, sizeof line, "ntt %s logN %d rows %ld %s %d ms %.4f\n", dir ? "inverse" : "forward",
                     ctx->logN, R,
                     minb == 4 ? "bulk-copy persistent, ctas_per_sm"
                               : minb == 6 ? "one pass, 8-CTA clusters, ctas_per_sm" : "ctas_per_sm",
                     minb == 4 ? 2 : minb == 5 ? 4 : minb == 6 ? 2 : minb, t);
            ctx->tune_log += line;
            if (t < best) best = t, pick = minb;
        }
        (dir == 0 ? ctx->ntt_minb : ctx->ntt_minb_inv) = pick;
        if (pick == 4 || pick == 6) {   // these take every row in one launch (no chunks)
            ctx->ntt_chunk = 0;
            continue;
        }
        // then the rows per launch pair: all, or chunks of 96 or 48 MiB
        // whose pass-0 output pass 1 still finds in L2
        int &chunk = dir == 0 ? ctx->ntt_chunk : ctx->ntt_chunk_inv;
        int cpick = 0;
        for (long mb : {0L, 96L, 48L}) {
            const int c = mb ? (int)std::max(1L, (mb << 20) / (8L * ctx->N)) : 0;
            if (c >= R) continue;
            chunk = c;
            float t = 1e30f;
            for (int rep = 0; rep < 3; rep++) {
                cudaEventRecord(a, st);
                const long step = c ? c : R;
                for (long r0 = 0; r0 < R; r0 += step) {
                    const long nr = std::min(step, R - r0);
                    u64 *d = scratch.p + r0 * (long)ctx->N;
                    RowMap mm = m.shifted(r0);
                    if (dir == 0) {
                        fwd_both(ctx, d, nr, mm, st, none, nullptr);
                    } else {
                        if (ctx->logN - logN1 == 8) inv_pass<8, true>(ctx, d, nr, mm, st); else inv_pass<7, true>(ctx, d, nr, mm, st);
                        if (logN1 == 8) inv_pass<8, false>(ctx, d, nr, mm, st); else inv_pass<7, false>(ctx, d, nr, mm, st);
                    }
                }
                cudaEventRecord(b, st);
                cudaEventSynchronize(b);
                float ms = 0;
                cudaEventElapsedTime(&ms, a, b);
                t = std::min(t, ms);
            }
            char line[112];
            snprintf(line, sizeof line, "ntt %s logN %d rows %ld rows_per_launch %d ms %.4f\n",
                     dir ? "inverse" : "forward", ctx->logN, R, c ? c : (int)R, t);
            ctx->tune_log += line;
            if (mb == 0 || t < best) best = t, cpick = c;
        }
        chunk = cpick;
    }
    ctx->ev_free.push_back(a);
    ctx->ev_free.push_back(b);
}

void ntt_fwd(Ctx *ctx, u64 *data, long rows, const RowMap &rm, cudaStream_t st, const RowSkip *skip) {
    if (rows <= 0) return;
    if (ctx->autotune && !ctx->ntt_tuned && ctx->logN >= 14 && ctx->logN <= 16) tune_ntt(ctx, st);
    int logN = ctx->logN, logN1, C, R;
    split(logN, logN1, C, R);
    int N1 = 1 << logN1, N2 = 1 << (logN - logN1);
    if (logN >= 14 && logN <= 16 && ctx->ntt_minb == 4) {
        // persistent passes: one launch each over every row
        RowSkip sk;
        long done = rows;
        if (skip) {
            sk = *skip;
            sk.row0 = 0;
            const long per_item = (long)sk.ndig * sk.rows_per_digit;
            done = (rows / per_item) * (per_item - sk.nq);
        }
        ctx->n_launch += 2;
        cudaEvent_t e0;
        ctx->trace_begin(1, e0);
        fwd_both(ctx, data, rows, rm, st, sk, nullptr);
        ctx->trace_end(1, e0, 2.0 * done * ctx->N * 8.0);
        return;
    }
    const long chunk = ctx->ntt_chunk > 0 && ctx->ntt_chunk < 65535 ? ctx->ntt_chunk : 65535;
    for (long r0 = 0; r0 < rows; r0 += chunk) {
        long nr = rows - r0 < chunk ? rows - r0 : chunk;
        u64 *d = data + r0 * (long)ctx->N;
        RowMap m = rm.shifted(r0);
        ctx->n_launch += 2;
        cudaEvent_t e0;
        ctx->trace_begin(1, e0);
        if (logN >= 14 && logN <= 16) {
            RowSkip sk;
            long done = nr;
            if (skip) {
                sk = *skip;
                sk.row0 = r0;
                done = 0;
                for (long r = 0; r < nr; r++) done += !sk.skip(r);
            }
            fwd_both(ctx, d, nr, m, st, sk, nullptr);
            // algorithmic bytes: every transformed word read and written once
            // (the two passes move twice that)
            ctx->trace_end(1, e0, 2.0 * done * ctx->N * 8.0);
            continue;
        }
        if (skip) throw std::logic_error("row skipping needs the register-blocked NTT (logN 14..16)");
        k_ntt_fwd_p1<<<dim3(N2 / C, (unsigned)nr), 256, N1 * C * 8, st>>>(d, m, ctx->d_mod, ctx->d_psi,
                                                                       ctx->d_psip, logN, logN1, C);
        k_ntt_fwd_p2<<<dim3(N1 / R, (unsigned)nr), 256, R * N2 * 8, st>>>(d, m, ctx->d_mod, ctx->d_psi,
                                                                       ctx->d_psip, logN, logN1, R);
    }
}

void ntt_fwd_subscale(Ctx *ctx, u64 *data, long rows, const RowMap &rm, cudaStream_t st, const SubScale &ep) {
    if (rows <= 0) return;
    if (ctx->autotune && !ctx->ntt_tuned && ctx->logN >= 14 && ctx->logN <= 16) tune_ntt(ctx, st);
    int logN = ctx->logN, logN1, C, R;
    split(logN, logN1, C, R);
    if (logN < 14 || logN > 16) throw std::logic_error("the fused NTT epilogue needs the register-blocked NTT");
    if (ctx->ntt_minb == 4) {
        ctx->n_launch += 2;
        cudaEvent_t e0;
        ctx->trace_begin(1, e0);
        RowSkip none;
        fwd_both(ctx, data, rows, rm, st, none, &ep);
        ctx->trace_end(1, e0, 2.0 * rows * ctx->N * 8.0);
        return;
    }
    const long chunk = ctx->ntt_chunk > 0 && ctx->ntt_chunk < 65535 ? ctx->ntt_chunk : 65535;
    for (long r0 = 0; r0 < rows; r0 += chunk) {
        long nr = rows - r0 < chunk ? rows - r0 : chunk;
        u64 *d = data + r0 * (long)ctx->N;
        RowMap m = rm.shifted(r0);
        SubScale e = ep;
        e.row0 = ep.row0 + r0;
        ctx->n_launch += 2;
        cudaEvent_t e0;
        ctx->trace_begin(1, e0);
        RowSkip none;
        fwd_both(ctx, d, nr, m, st, none, &e);
        // algorithmic bytes of the transform: every word read and written once
        // (the fused epilogue's read of u is not counted, so butterflies per
        // traced byte stay those of a plain transform)
        ctx->trace_end(1, e0, 2.0 * nr * ctx->N * 8.0);
    }
}

void ntt_inv(Ctx *ctx, u64 *data, long rows, const RowMap &rm, cudaStream_t st) {
    if (rows <= 0) return;
    if (ctx->autotune && !ctx->ntt_tuned && ctx->logN >= 14 && ctx->logN <= 16) tune_ntt(ctx, st);
    int logN = ctx->logN, logN1, C, R;
    split(logN, logN1, C, R);
    int N1 = 1 << logN1, N2 = 1 << (logN - logN1);
    const long chunk = ctx->ntt_chunk_inv > 0 && ctx->ntt_chunk_inv < 65535 ? ctx->ntt_chunk_inv : 65535;
    for (long r0 = 0; r0 < rows; r0 += chunk) {
        long nr = rows - r0 < chunk ? rows - r0 : chunk;
        u64 *d = data + r0 * (long)ctx->N;
        RowMap m = rm.shifted(r0);
        ctx->n_launch += 2;
        cudaEvent_t e0;
        ctx->trace_begin(2, e0);
        if (logN >= 14 && logN <= 16) {
            if (logN - logN1 == 8) inv_pass<8, true>(ctx, d, nr, m, st); else inv_pass<7, true>(ctx, d, nr, m, st);
            if (logN1 == 8) inv_pass<8, false>(ctx, d, nr, m, st); else inv_pass<7, false>(ctx, d, nr, m, st);
            ctx->trace_end(2, e0, 2.0 * nr * ctx->N * 8.0);
            continue;
        }
        k_ntt_inv_p2<<<dim3(N1 / R, (unsigned)nr), 256, R * N2 * 8, st>>>(d, m, ctx->d_mod, ctx->d_ipsi,
                                                                       ctx->d_ipsip, logN, logN1, R);
        k_ntt_inv_p1<<<dim3(N2 / C, (unsigned)nr), 256, N1 * C * 8, st>>>(d, m, ctx->d_mod, ctx->d_ipsi,
                                                                       ctx->d_ipsip, ctx->d_ninv, logN,
                                                                       logN1, C);
    }
}

}  // namespace he
