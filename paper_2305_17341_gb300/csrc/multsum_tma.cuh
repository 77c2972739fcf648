// multsum_tma.cuh -- MultSum + Permute (Sec. 3.3.1) fed by bulk asynchronous
// copies.  Included by kernels.cu, after MultiKeys and auto_index.
//
// The inner product of the hoisted key switch reads every digit word once
// and every key word once per launch; the work per byte is a few 32-bit
// multiply-adds, so the kernel lives on memory throughput.  Here each CTA is
// persistent and walks a sequence of (tile, digit) stages: a tile is TW
// coefficients of one row of Q_l P for up to BI items, a stage the digit-d
// words of those items plus the digit-d words of the G keys (2 polynomials
// each).  One thread issues every segment of a stage as a `cp.async.bulk`
// global->shared copy (contiguous TW words) that completes on the stage's
// "full" mbarrier.  The copies are issued by a producer warp of its own,
// which refills a buffer as soon as the eight consumer warps have released
// it on the buffer's "empty" mbarrier, so S stages stay in flight while the
// consumers multiply-accumulate the oldest: the copies run back to back
// across digits and tiles, no register holds a load in flight and no
// CTA-wide barrier is taken in the loop.  Each consumer thread owns one
// coefficient of two items and the 2G accumulators of each: the key words
// it reads from shared memory serve both items, the digit words all G keys.
//
// Segments of 8 TW bytes: the copy engine's cost per request, not the bytes,
// limits small segments, so wider tiles with fewer items (keys then come
// from L2 for the other item groups of a tile) are launch variants.
//
// Waits are bounded: a wait that does not complete within the iteration
// limit sets *err (a flag the host checks after synchronising) and a shared
// stop flag; every thread then leaves its loop, and the producer waits (again
// bounded) for the copies it still has in flight before the CTA exits.
#pragma once
// (bulkcopy.cuh is included by the including file, outside its namespace)

// A tile is TW coefficients (segments of 8 TW bytes) of BI items; 256
// consumer threads, each with one coefficient of two items (TW * BI = 512),
// and one producer warp.
constexpr int MST_CONSUMERS = 256;
constexpr int MST_THREADS = MST_CONSUMERS + 32;

struct MstGeom {
    int N, logN, rows, level, L, ndig, nprimes, ntx, nig, B;   // ntx = N / TW, nig = ceil(B / BI)
    long ntiles;
    __device__ __forceinline__ void tile(long t, int &ig, int &xt, int &r) const {
        ig = (int)(t % nig);
        const long rest = t / nig;
        xt = (int)(rest % ntx);
        r = (int)(rest / ntx);
    }
    __device__ __forceinline__ int prime_of_row(int r) const { return r <= level ? r : L + 1 + (r - level - 1); }
};

// Issues the copies of stage jj of this CTA's sequence (tile jj / ndig of
// the CTA, digit jj % ndig) into buffer jj % S; false past the last tile.
template <int G, int S, int TW, int BI>
__device__ __forceinline__ bool mst_issue(const MstGeom &g, const MultiKeys<G> &mk, const u64 *digits, u64 *stage,
                                          u64 *full, long jj) {
    constexpr int SEG = BI + 2 * G;
    const long ti = jj / g.ndig;
    const int d = (int)(jj - ti * g.ndig);
    const long t = (long)blockIdx.x + ti * (long)gridDim.x;
    if (t >= g.ntiles) return false;
    int ig, xt, r;
    g.tile(t, ig, xt, r);
    const int kr = g.prime_of_row(r);
    const int s = (int)(jj % S);
    const int b0 = ig * BI, nb = min(BI, g.B - b0);
    u64 *dst = stage + (long)s * SEG * TW;
    const long y0 = (long)xt * TW, N = g.N;
    // the buffer's previous contents were read by the consumers before they
    // arrived on its "empty" barrier, which the producer waited on: that
    // ordering covers the copy engine's writes (no proxy fence per stage)
    u64 *bar = full;
    bc_expect_tx(&bar[s], (u32)((nb + 2 * G) * TW * 8));
    const long dstride = (long)g.rows * N;
    for (int b = 0; b < nb; b++)
        bc_bulk(dst + b * TW, digits + ((long)(b0 + b) * g.ndig + d) * dstride + (long)r * N + y0, TW * 8, &bar[s]);
    const long kd = 2L * g.nprimes * N, kk = (long)g.nprimes * N;
#pragma unroll
    for (int k = 0; k < G; k++) {
        const u64 *kp = mk.key[k] + (long)d * kd + (long)kr * N + y0;
        bc_bulk(dst + (BI + 2 * k) * TW, kp, TW * 8, &bar[s]);
        bc_bulk(dst + (BI + 2 * k + 1) * TW, kp + kk, TW * 8, &bar[s]);
    }
    return true;
}

// Accumulators of one thread: per (item, key, polynomial) 96 bits (three
// 32-bit words) for rows below 2^42, 128 bits for the 60-bit rows.
template <int G, bool W96>
struct MstAcc;
template <int G>
struct MstAcc<G, true> {
    u32 x0[2][2 * G], x1[2][2 * G], x2[2][2 * G];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int k = 0; k < 2 * G; k++) x0[i][k] = 0, x1[i][k] = 0, x2[i][k] = 0;
    }
    __device__ __forceinline__ void mac(int i, int k, u64 v, u64 key, u64) { mac96(x0[i][k], x1[i][k], x2[i][k], v, key); }
    __device__ __forceinline__ u64 out(int i, int k, const ModQ &m) const {
        return redc(((u64)x1[i][k] << 32) | x0[i][k], x2[i][k], m);
    }
};
template <int G>
struct MstAcc<G, false> {
    U128 w[2][2 * G];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < 2; i++)
#pragma unroll
            for (int k = 0; k < 2 * G; k++) w[i][k] = U128{0, 0};
    }
    __device__ __forceinline__ void mac(int i, int k, u64 v, u64 key, u64 q) { mac128_q(w[i][k], v, key, q); }
    __device__ __forceinline__ u64 out(int i, int k, const ModQ &m) const { return redc(w[i][k].lo, w[i][k].hi, m); }
};

// One tile on a consumer thread: its ndig stages (wait until the buffer is
// full, accumulate, release it to the producer), then the epilogue.
// Returns false when a wait ran out or another thread stopped the CTA.
template <int G, int S, int TW, int BI, bool W96>
__device__ __forceinline__ bool mst_tile(const MultiKeys<G> &mk, const MstGeom &geo, const u64 *stage, u64 *full,
                                         u64 *empty, volatile int &stop, int *err, long &jj, int r, int y, int b0,
                                         const ModQ &m, const u64 *c0, long c0s, const ShoupPair *Pmod) {
    constexpr int SEG = BI + 2 * G;
    const int tid = threadIdx.x, c = tid % TW, ip = tid / TW, lane = tid & 31;
    MstAcc<G, W96> acc;
    acc.zero();
    for (int d = 0; d < geo.ndig; d++, jj++) {
        const int s = (int)(jj % S);
        if (stop) return false;
        if (!bc_wait(&full[s], (u32)((jj / S) & 1))) {
            stop = 1;
            atomicExch(err, 1);
            return false;
        }
        const u64 *sg = stage + (long)s * SEG * TW;
        u64 kv[2 * G];
#pragma unroll
        for (int k = 0; k < 2 * G; k++) kv[k] = sg[(BI + k) * TW + c];
        const u64 v0 = sg[(2 * ip) * TW + c], v1 = sg[(2 * ip + 1) * TW + c];
        // every word of the buffer this warp needs is in registers: release it
        __syncwarp();
        if (lane == 0) bc_arrive(&empty[s]);
#pragma unroll
        for (int k = 0; k < 2 * G; k++) {
            acc.mac(0, k, v0, kv[k], m.q);
            acc.mac(1, k, v1, kv[k], m.q);
        }
    }
    // epilogue: one Montgomery reduction per output word, P c0 on the Q rows
    // of polynomial 0, store at the permuted position
    const int N = geo.N, rows = geo.rows;
    const bool with_c0 = c0 && r <= geo.level;
    const ShoupPair wP = with_c0 ? Pmod[r] : ShoupPair{0, 0};
#pragma unroll
    for (int i = 0; i < 2; i++) {
        const int b = b0 + i;
        if (b >= geo.B) continue;
        u64 pc0 = 0;
        if (with_c0) pc0 = shoup(c0[(long)b * c0s + (long)r * N + y], wP.w, wP.wp, m.q);
#pragma unroll
        for (int k = 0; k < G; k++) {
            u64 o0 = acc.out(i, 2 * k, m);
            const u64 o1 = acc.out(i, 2 * k + 1, m);
            if (with_c0) o0 = addmod(o0, pc0, m.q);
            const int x = mk.ginv[k] == 1u ? y : auto_index(y, mk.ginv[k], geo.logN);
            u64 *ob = mk.out[k] + (long)b * 2 * rows * N;
            ob[(long)r * N + x] = o0;
            ob[(long)(rows + r) * N + x] = o1;
        }
    }
    return true;
}

template <int G, int S, int TW, int BI>
__global__ void __launch_bounds__(MST_THREADS, 1)
    k_multsum_tma(MultiKeys<G> mk, const u64 *digits, MstGeom geo, const ModQ *mods, const u64 *c0, long c0s,
                  const ShoupPair *Pmod, int *err) {
    extern __shared__ __align__(128) u64 mst_stage[];
    __shared__ __align__(8) u64 full[S], empty[S];
    __shared__ volatile int stop;
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int s = 0; s < S; s++) {
            bc_bar_init(&full[s], 1);
            bc_bar_init(&empty[s], MST_CONSUMERS / 32);
        }
        stop = 0;
        bc_init_fence();
    }
    __syncthreads();
    const long per_cta = geo.ntiles > blockIdx.x ? (geo.ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const long nstages = per_cta * geo.ndig;
    if (tid >= MST_CONSUMERS) {
        // producer warp: one lane refills each buffer once the consumers
        // have released it
        if (tid != MST_CONSUMERS) return;
        long jj = 0;
        for (; jj < nstages; jj++) {
            const int s = (int)(jj % S);
            if (jj >= S && !bc_wait(&empty[s], (u32)(((jj / S) - 1) & 1))) {
                stop = 1;
                atomicExch(err, 1);
                break;
            }
            if (stop) break;
            mst_issue<G, S, TW, BI>(geo, mk, digits, mst_stage, full, jj);
        }
        // copies still in flight land before the CTA's shared memory is
        // given back: wait (bounded) for every issued stage that no consumer
        // consumed, or simply the last S of them
        for (long k = (jj > S ? jj - S : 0); k < jj; k++) bc_wait(&full[k % S], (u32)((k / S) & 1));
        return;
    }
    const int c = tid % TW, ip = tid / TW;   // coefficient; item pair
    long jj = 0;
    for (long ti = 0; ti < per_cta; ti++) {
        const long t = (long)blockIdx.x + ti * (long)gridDim.x;
        int ig, xt, r;
        geo.tile(t, ig, xt, r);
        const ModQ m = mods[geo.prime_of_row(r)];
        const int y = xt * TW + c, b0 = ig * BI + 2 * ip;
        // 96-bit accumulation on the rows below 2^42 (uniform over the tile)
        const bool ok = m.q < (1ull << 42)
                            ? mst_tile<G, S, TW, BI, true>(mk, geo, mst_stage, full, empty, stop, err, jj, r, y, b0,
                                                           m, c0, c0s, Pmod)
                            : mst_tile<G, S, TW, BI, false>(mk, geo, mst_stage, full, empty, stop, err, jj, r, y, b0,
                                                            m, c0, c0s, Pmod);
        if (!ok) return;
    }
}
