// noalloc.cu -- a slot rotation that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need a
// rotation: code that runs while the device memory of the process is owned
// and budgeted by another runtime (an inference server's arena, a framework
// allocator that must see every byte), code on a latency-critical thread
// that must not block in the driver's allocator, or code that must not risk
// an out-of-memory failure halfway through a pipeline.  he_rotate_noalloc
// serves them: the caller passes the input and output in device memory it
// owns, and every temporary the rotation needs lives in one fixed array
// that this library reserves in device memory when it is loaded.
//
// The array is shared by every call on the same device and keeps whatever
// the last call left in it; the rotation overwrites every word it reads, so
// nothing has to start at zero.  Calls whose work overlaps on the GPU (two
// host threads, or several contexts on one device) race on the array and
// must be serialised by the caller.
//
// The work runs on the context's stream, which is not ordered after any
// stream of the caller: the caller finishes its own writes to the input and
// output buffers (for instance by synchronising the stream that made them)
// before the call, and the call returns only when its work is done.
#include <cstring>
#include <mutex>
#include <new>

#include "eval.h"

using namespace he;

namespace he {
void launch_modup_bconv_with(Ctx *c, const u64 *coef, u64 *out, int B, int level, const ShoupPair *up_inv,
                             const ShoupPair *up_mod, cudaStream_t st);
}

struct he_ctx {
    Ctx c;
};

// 32 MiB of device scratch per device that loads the library, held until exit.
#define HE_NOALLOC_SCRATCH_WORDS (4ull << 20)
static __device__ __align__(256) unsigned long long g_noalloc_scratch[HE_NOALLOC_SCRATCH_WORDS];

static std::mutex g_noalloc_mu;
static u64 *g_noalloc_addr[64];                       // device address of the array, per device
static ShoupPair g_noalloc_consts[48 * 4 * 53 + 48 * 4];  // host staging of the ModUp constants

// The host-side name of the array is only a stand-in: its device address is
// asked from the runtime once per device, with that device current.
static int noalloc_scratch(int dev, u64 **out) {
    if (dev < 0 || dev >= 64) {
        set_error("device index out of range");
        return HE_ERR_ARG;
    }
    if (!g_noalloc_addr[dev]) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != dev && cudaSetDevice(dev) != cudaSuccess) {
            set_error("cannot select the context's device");
            return HE_ERR_CUDA;
        }
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (cur != dev && cur >= 0) cudaSetDevice(cur);
        if (e != cudaSuccess || !p) {
            set_error(std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return HE_ERR_CUDA;
        }
        g_noalloc_addr[dev] = (u64 *)p;
    }
    *out = g_noalloc_addr[dev];
    return HE_OK;
}

// Turns the context's tracing and launch tuner off for the duration of a
// call (both would create CUDA events) and restores them on every exit path.
struct QuietCtx {
    Ctx &c;
    bool tr, at;
    explicit QuietCtx(Ctx &cc) : c(cc), tr(cc.trace), at(cc.autotune) {
        c.trace = false;
        c.autotune = false;
    }
    ~QuietCtx() {
        c.trace = tr;
        c.autotune = at;
    }
};

static int rotate_noalloc(he_ctx *ctx, const uint64_t *in_dev, int level, int step, uint64_t *out_dev);

extern "C" int he_rotate_noalloc(he_ctx *ctx, const uint64_t *in_dev, int level, int step, uint64_t *out_dev) {
    // nothing may cross the C boundary as a C++ exception
    try {
        return rotate_noalloc(ctx, in_dev, level, step, out_dev);
    } catch (const HeError &e) {
        set_error(e.what());
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return HE_ERR_OOM;
    } catch (const std::exception &e) {
        set_error(e.what());
        return HE_ERR_ARG;
    }
}

static int rotate_noalloc(he_ctx *ctx, const uint64_t *in_dev, int level, int step, uint64_t *out_dev) {
    if (!ctx || !in_dev || !out_dev) {
        set_error("null argument");
        return HE_ERR_ARG;
    }
    Ctx &c = ctx->c;
    if (level < 0 || level > c.L) {
        set_error("level out of range");
        return HE_ERR_LEVEL;
    }
    const int N = c.N, nq = level + 1, rows = c.qp_rows(level), nd = c.ndig(level), a = c.alpha;
    if (nd * a * rows + nd * a > (int)(sizeof(g_noalloc_consts) / sizeof(ShoupPair))) {
        set_error("level too deep for the no-allocation rotation");
        return HE_ERR_ARG;
    }
    // scratch layout (words): constants | ct | digits | u | P rows | conversion
    const size_t wc = ((size_t)2 * (nd * a + (size_t)nd * a * rows) + 31) / 32 * 32;
    const size_t wct = (size_t)2 * nq * N, wdig = (size_t)nd * rows * N, wu = (size_t)2 * rows * N;
    const size_t wpc = (size_t)2 * a * N, wconv = (size_t)2 * nq * N;
    const size_t need = wc + wct + wdig + wu + wpc + wconv;
    if (need > HE_NOALLOC_SCRATCH_WORDS) {
        set_error("rotation at this ring degree and level needs " + std::to_string(need * 8) +
                  " bytes of scratch, more than the " + std::to_string(HE_NOALLOC_SCRATCH_WORDS * 8) +
                  " bytes reserved");
        return HE_ERR_ARG;
    }
    uint32_t g = galois_of_step(&c, step);
    auto kit = c.rtk.find(g);
    if (kit == c.rtk.end()) {
        set_error("rotation key for this step missing");
        return HE_ERR_KEY_MISSING;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    u64 *base = nullptr;
    if (int rc = noalloc_scratch(c.device, &base)) return rc;
    ShoupPair *d_inv = (ShoupPair *)base, *d_mod = d_inv + nd * a;
    u64 *S_ct = base + wc, *S_dig = S_ct + wct, *S_u = S_dig + wdig, *S_pc = S_u + wu, *S_conv = S_pc + wpc;

    // ModUp constants of this level: (Q_d/q_i)^-1 mod q_i and Q_d/q_i mod r
    ShoupPair *h_inv = g_noalloc_consts, *h_mod = g_noalloc_consts + nd * a;
    for (int d = 0; d < nd; d++) {
        int i0 = d * a, ns = std::min(a, level + 1 - i0);
        for (int s = 0; s < ns; s++) {
            u64 qi = c.primes[i0 + s], prod = 1;
            for (int t = 0; t < ns; t++)
                if (t != s) prod = h_mulmod(prod, c.primes[i0 + t] % qi, qi);
            h_inv[d * a + s] = h_shoup(h_invmod(prod, qi), qi);
            for (int r = 0; r < rows; r++) {
                u64 pr = r <= level ? c.primes[r] : c.primes[c.L + 1 + (r - level - 1)], v = 1;
                for (int t = 0; t < ns; t++)
                    if (t != s) v = h_mulmod(v, c.primes[i0 + t] % pr, pr);
                h_mod[((size_t)d * a + s) * rows + r] = h_shoup(v, pr);
            }
        }
    }
    cudaStream_t st = c.stream;
    QuietCtx quiet(c);
    cudaMemcpyAsync(d_inv, h_inv, sizeof(ShoupPair) * (nd * a + (size_t)nd * a * rows), cudaMemcpyHostToDevice, st);
    // Decompose c1 (the input is in coefficient form already), extend, NTT
    const u64 *in = (const u64 *)in_dev;
    launch_modup_bconv_with(&c, in + (size_t)nq * N, S_dig, 1, level, d_inv, d_mod, st);
    ntt_fwd(&c, S_dig, (long)nd * rows, c.map_qp(level), st);
    // the ciphertext in the NTT domain (c0 enters MultSum as P kappa(c0))
    cudaMemcpyAsync(S_ct, in_dev, wct * 8, cudaMemcpyDeviceToDevice, st);
    ntt_fwd(&c, S_ct, 2L * nq, c.map_q(level), st);
    launch_multsum(&c, S_u, S_dig, kit->second, g, 1, level, S_ct, (long)wct, st);
    // rounding ModDown of both polynomials into the ct region, back to coefficients
    launch_copy_rows(S_pc, (long)a * N, S_u + (size_t)nq * N, (long)rows * N, 2, (long)a * N, st);
    ntt_inv(&c, S_pc, 2L * a, c.map_p(), st);
    launch_moddown_bconv(&c, S_pc, S_conv, 2, level, st);
    ntt_fwd(&c, S_conv, 2L * nq, c.map_q(level), st);
    launch_moddown_final(&c, S_ct, S_u, S_conv, nullptr, 2, level, (long)rows * N, (long)nq * N, 0, st);
    ntt_inv(&c, S_ct, 2L * nq, c.map_q(level), st);
    cudaMemcpyAsync(out_dev, S_ct, wct * 8, cudaMemcpyDeviceToDevice, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error(std::string("CUDA error: ") + cudaGetErrorString(e));
        return HE_ERR_CUDA;
    }
    return HE_OK;
}
