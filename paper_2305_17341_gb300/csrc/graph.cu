// graph.cu -- captured batched products (he_mm_plan_*): the gather, the
// replication and every kernel of the batched JKLS product (Sec. 3.3.2 with
// the hoisted schedule of Sec. 4.1) for a fixed set of jobs, recorded once as
// a CUDA graph on the context's stream and replayed per run, so that the
// thousands of launches of a batched step cost one graph launch on the host.
//
// The graph's temporaries live in a pool owned by the plan (never handed to
// anything else), filled by one uncaptured recording run before capture;
// outputs are copied from plan memory into fresh ciphertexts after each
// replay, outside the graph.
#include <algorithm>
#include <map>
#include <tuple>

#include "ctapi.h"

using namespace he;

namespace {

struct Group {
    std::vector<int> idx;        // job indices
    int level = 0, n = 0, n1z = 0, n1t = 0;
    bool repA = false, repB = false, relin_once = false;
    int dcd_z = 0, dcd_t = 0, depth = 3;
    u64 *O = nullptr;            // [items][2][level-2][N], plan memory
    size_t wo = 0;
};

}  // namespace

struct he_mm_plan {
    Ctx *c = nullptr;
    std::vector<he_mm_job> jobs;
    std::vector<Group> groups;
    DevicePool pool;             // the graph's private scratch and outputs
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;      // kernel launches one replay performs
};

static int plan_fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

// Enqueues the whole batched step on c->stream with scratch from the ctx pool
// (redirected to the plan's pool by the caller).
static void record(he_mm_plan *P) {
    Ctx &c = *P->c;
    for (Group &g : P->groups) {
        const int Bn = (int)g.idx.size();
        const size_t w = ct_words(&c, g.level);
        Buf A(&c.pool, Bn * w), B(&c.pool, Bn * w);
        for (int t = 0; t < Bn; t++) {
            const he_mm_job &j = P->jobs[g.idx[t]];
            const size_t pitch = (size_t)(g.level + 1) * c.N * 8;
            cudaMemcpy2DAsync(A.p + t * w, pitch, j.A->d, (size_t)(j.A->level + 1) * c.N * 8, pitch, 2,
                              cudaMemcpyDeviceToDevice, c.stream);
            cudaMemcpy2DAsync(B.p + t * w, pitch, j.B->d, (size_t)(j.B->level + 1) * c.N * 8, pitch, 2,
                              cudaMemcpyDeviceToDevice, c.stream);
        }
        if (g.repA) replicate(&c, A.p, Bn, g.level, g.n);
        if (g.repB) replicate(&c, B.p, Bn, g.level, g.n);
        hmatmul(&c, A.p, B.p, Bn, g.level, g.n, g.n1z, g.n1t, g.O, g.relin_once, g.dcd_z, g.dcd_t);
    }
}

extern "C" {

int he_mm_plan_create(const he_mm_job *jobs, int n_jobs, he_mm_plan **out) {
    if (!jobs || n_jobs < 1 || !out) return plan_fail(HE_ERR_ARG, "bad arguments");
    Ctx *c = nullptr;
    for (int i = 0; i < n_jobs; i++) {
        const he_mm_job &j = jobs[i];
        if (!j.A || !j.B || j.A->ctx != j.B->ctx) return plan_fail(HE_ERR_ARG, "bad job operands");
        if (c && j.A->ctx != c) return plan_fail(HE_ERR_ARG, "a plan serves one context");
        c = j.A->ctx;
        const int n = j.n;
        auto pow2 = [](int x) { return x > 0 && (x & (x - 1)) == 0; };
        if (!pow2(n) || (long)n * n > c->S || !pow2(j.sched.n1_z) || !pow2(j.sched.n1_t) || j.sched.n1_z > n ||
            j.sched.n1_t > n || j.sched.n1_z > 32 || j.sched.n1_t > 32)
            return plan_fail(HE_ERR_ARG, "bad block size or schedule");
        if ((j.sched.dcd_z && (j.sched.dcd_z >= n || j.sched.dcd_z % j.sched.n1_z)) ||
            (j.sched.dcd_t && (j.sched.dcd_t >= n || j.sched.dcd_t % j.sched.n1_t)))
            return plan_fail(HE_ERR_ARG, "a decomposition needs n' < n with the baby steps dividing n'");
        if (std::min(j.A->level, j.B->level) < hmatmul_depth(n, j.sched.dcd_z, j.sched.dcd_t))
            return plan_fail(HE_ERR_LEVEL, "not enough levels for the product");
        if (long miss = first_missing_key(c, matmul_steps(n, j.sched.n1_z, j.sched.n1_t, c->S, j.sched.dcd_z,
                                                          j.sched.dcd_t),
                                          (j.A->period == n * n && j.B->period == n * n) ? (long)n * n : c->S))
            return plan_fail(HE_ERR_KEY_MISSING, "rotation key for step " + std::to_string(miss) + " missing");
        if (!c->rlk) return plan_fail(HE_ERR_KEY_MISSING, "relinearisation key missing");
    }
    he_mm_plan *P = new (std::nothrow) he_mm_plan;
    if (!P) return plan_fail(HE_ERR_OOM, "host allocation failed");
    P->c = c;
    P->jobs.assign(jobs, jobs + n_jobs);
    typedef std::tuple<int, int, int, int, bool, bool, bool, int, int> Key;
    std::map<Key, int> gi;
    for (int i = 0; i < n_jobs; i++) {
        const he_mm_job &j = jobs[i];
        const int n = j.n, lv = std::min(j.A->level, j.B->level);
        Key k(lv, n, j.sched.n1_z, j.sched.n1_t, j.A->period != n * n, j.B->period != n * n,
              j.sched.relin_once != 0, j.sched.dcd_z, j.sched.dcd_t);
        auto it = gi.find(k);
        if (it == gi.end()) {
            Group g;
            g.level = lv, g.n = n, g.n1z = j.sched.n1_z, g.n1t = j.sched.n1_t;
            g.repA = std::get<4>(k), g.repB = std::get<5>(k), g.relin_once = std::get<6>(k);
            g.dcd_z = j.sched.dcd_z, g.dcd_t = j.sched.dcd_t, g.depth = hmatmul_depth(n, g.dcd_z, g.dcd_t);
            it = gi.emplace(k, (int)P->groups.size()).first;
            P->groups.push_back(g);
        }
        P->groups[it->second].idx.push_back(i);
    }
    const bool trace = c->trace;
    c->trace = false;
    int rc = HE_OK;
    try {
        for (Group &g : P->groups) {
            g.wo = ct_words(c, g.level - g.depth);
            g.O = (u64 *)P->pool.get(g.idx.size() * g.wo * 8);
        }
        // 1. recording run: fills the plan's pool and the context's caches
        c->pool.set_redirect(&P->pool);
        record(P);
        c->pool.set_redirect(nullptr);
        if (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
            throw HeError(HE_ERR_CUDA, "recording run failed");
        // 2. capture (relaxed: a pool miss may still allocate)
        const long long n0 = c->n_launch;
        c->pool.set_redirect(&P->pool);
        if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
            c->pool.set_redirect(nullptr);
            throw HeError(HE_ERR_CUDA, "stream capture could not start");
        }
        try {
            record(P);
        } catch (...) {
            cudaGraph_t g = nullptr;
            cudaStreamEndCapture(c->stream, &g);
            if (g) cudaGraphDestroy(g);
            c->pool.set_redirect(nullptr);
            throw;
        }
        c->pool.set_redirect(nullptr);
        P->launches = c->n_launch - n0;
        c->n_launch = n0;
        if (cudaStreamEndCapture(c->stream, &P->graph) != cudaSuccess || !P->graph)
            throw HeError(HE_ERR_CUDA, "stream capture failed");
        if (cudaGraphInstantiate(&P->exec, P->graph, 0) != cudaSuccess)
            throw HeError(HE_ERR_CUDA, "graph instantiation failed");
    } catch (const HeError &e) {
        set_error(e.what());
        rc = e.code;
    } catch (const std::bad_alloc &) {
        set_error("device or host allocation failed");
        rc = HE_ERR_OOM;
    } catch (const std::exception &e) {
        set_error(e.what());
        rc = HE_ERR_ARG;
    }
    c->trace = trace;
    cudaGetLastError();
    if (rc != HE_OK) {
        if (P->exec) cudaGraphExecDestroy(P->exec);
        if (P->graph) cudaGraphDestroy(P->graph);
        delete P;
        return rc;
    }
    *out = P;
    return HE_OK;
}

int he_mm_plan_run(he_mm_plan *P, he_ct **outs) {
    if (!P || !outs) return plan_fail(HE_ERR_ARG, "bad arguments");
    Ctx &c = *P->c;
    std::vector<he_ct *> res(P->jobs.size(), nullptr);
    try {
        if (cudaGraphLaunch(P->exec, c.stream) != cudaSuccess) throw HeError(HE_ERR_CUDA, "graph launch failed");
        c.n_launch += P->launches;
        for (const Group &g : P->groups) {
            const double q2 = (double)c.primes[g.level - g.depth + 1];
            for (size_t t = 0; t < g.idx.size(); t++) {
                const he_mm_job &j = P->jobs[g.idx[t]];
                he_ct *o = new_ct(&c, g.level - g.depth, (j.A->scale * j.B->scale) / q2, j.n * j.n);
                res[g.idx[t]] = o;
                cudaMemcpyAsync(o->d, g.O + t * g.wo, g.wo * 8, cudaMemcpyDeviceToDevice, c.stream);
            }
        }
        cudaError_t e = cudaStreamSynchronize(c.stream);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) throw HeError(HE_ERR_CUDA, std::string("CUDA error: ") + cudaGetErrorString(e));
        if (device_status(&c)) throw HeError(HE_ERR_TIMEOUT, last_error());
    } catch (const HeError &e) {
        for (he_ct *o : res) free_ct(o);
        set_error(e.what());
        return e.code;
    } catch (const std::bad_alloc &) {
        for (he_ct *o : res) free_ct(o);
        set_error("device or host allocation failed");
        return HE_ERR_OOM;
    }
    for (size_t i = 0; i < res.size(); i++) outs[i] = res[i];
    return HE_OK;
}

int he_mm_plan_info(const he_mm_plan *P, long long *launches, double *scratch_bytes) {
    if (!P) return plan_fail(HE_ERR_ARG, "bad arguments");
    if (launches) *launches = P->launches;
    if (scratch_bytes) *scratch_bytes = (double)(const_cast<he_mm_plan *>(P)->pool.bytes_in_use() +
                                                 const_cast<he_mm_plan *>(P)->pool.bytes_cached());
    return HE_OK;
}

int he_mm_plan_destroy(he_mm_plan *P) {
    if (!P) return HE_OK;
    cudaStreamSynchronize(P->c->stream);
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->graph) cudaGraphDestroy(P->graph);
    delete P;  // the pool's destructor frees the scratch
    return HE_OK;
}

}  // extern "C"
