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
//
// Each limb of N = N1 * N2 coefficients is transformed in two passes: pass 1
// runs the stages whose butterfly span is >= N2 on column tiles (elements with
// equal index mod N2, C columns per CTA, staged in shared memory); pass 2 runs
// the remaining log2(N2) stages on rows of N2 contiguous coefficients.  Both
// passes read and write HBM once.
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

// ---------------------------------------------------------------- forward
__global__ void k_ntt_fwd_p1(u64 *data, RowMap rm, const ModQ *mods, const u64 *tw, const u64 *twp,
                             int logN, int logN1, int C) {
    extern __shared__ u64 sm[];
    const int N = 1 << logN, N1 = 1 << logN1, N2 = N >> logN1;
    const long row = blockIdx.y;
    const int pidx = rm.p[row % rm.n];
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
    const int pidx = rm.p[row % rm.n];
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
    const int pidx = rm.p[row % rm.n];
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
    const int pidx = rm.p[row % rm.n];
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

void ntt_fwd(Ctx *ctx, u64 *data, long rows, const RowMap &rm, cudaStream_t st) {
    if (rows <= 0) return;
    int logN = ctx->logN, logN1, C, R;
    split(logN, logN1, C, R);
    int N1 = 1 << logN1, N2 = 1 << (logN - logN1);
    for (long r0 = 0; r0 < rows; r0 += 65535) {
        long nr = rows - r0 < 65535 ? rows - r0 : 65535;
        u64 *d = data + r0 * (long)ctx->N;
        RowMap m = rm.shifted(r0);
        k_ntt_fwd_p1<<<dim3(N2 / C, (unsigned)nr), 256, N1 * C * 8, st>>>(d, m, ctx->d_mod, ctx->d_psi,
                                                                       ctx->d_psip, logN, logN1, C);
        k_ntt_fwd_p2<<<dim3(N1 / R, (unsigned)nr), 256, R * N2 * 8, st>>>(d, m, ctx->d_mod, ctx->d_psi,
                                                                       ctx->d_psip, logN, logN1, R);
    }
}

void ntt_inv(Ctx *ctx, u64 *data, long rows, const RowMap &rm, cudaStream_t st) {
    if (rows <= 0) return;
    int logN = ctx->logN, logN1, C, R;
    split(logN, logN1, C, R);
    int N1 = 1 << logN1, N2 = 1 << (logN - logN1);
    for (long r0 = 0; r0 < rows; r0 += 65535) {
        long nr = rows - r0 < 65535 ? rows - r0 : 65535;
        u64 *d = data + r0 * (long)ctx->N;
        RowMap m = rm.shifted(r0);
        k_ntt_inv_p2<<<dim3(N1 / R, (unsigned)nr), 256, R * N2 * 8, st>>>(d, m, ctx->d_mod, ctx->d_ipsi,
                                                                       ctx->d_ipsip, logN, logN1, R);
        k_ntt_inv_p1<<<dim3(N2 / C, (unsigned)nr), 256, N1 * C * 8, st>>>(d, m, ctx->d_mod, ctx->d_ipsi,
                                                                       ctx->d_ipsip, ctx->d_ninv, logN,
                                                                       logN1, C);
    }
}

}  // namespace he
