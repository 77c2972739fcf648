// graph.cu -- captured batched products (he_mm_plan_*): the gather, the
// replication and every kernel of the batched JKLS product (Sec. 3.3.2 with
// the hoisted schedule of Sec. 4.1) for a fixed set of jobs, recorded once as
// a CUDA graph and replayed per run, so that the thousands of launches of a
// batched step cost one graph launch on the host.
//
// Jobs are grouped as he_hmatmul_batch groups them (context, level, block
// size, schedule); every group is one branch of the graph, recorded on a
// stream of its own and forked from / joined to the plan's stream, so at
// replay the groups -- of different sizes, levels and ring degrees -- run
// concurrently on the GPU and small groups fill what large ones leave idle
// (the paper's parallel matrix products of Sec. 4.1.2 as concurrent branches
// of one launch).  Each branch's temporaries live in a pool of its own,
// owned by the plan and filled by one uncaptured recording run before
// capture, so concurrent branches never share scratch; outputs are copied
// from plan memory into fresh ciphertexts after each replay, outside the
// graph.
#include <algorithm>
#include <map>
#include <memory>
#include <tuple>

#include "ctapi.h"

using namespace he;

namespace {

struct Group {
    Ctx *c = nullptr;
    std::vector<int> idx;        // job indices
    int level = 0, n = 0, n1z = 0, n1t = 0;
    bool repA = false, repB = false, relin_once = false;
    int dcd_z = 0, dcd_t = 0, depth = 3;
    u64 *O = nullptr;            // [items][2][level-2][N], plan memory
    size_t wo = 0;
    std::unique_ptr<DevicePool> pool;   // the branch's private scratch
    cudaStream_t st = nullptr;          // the branch's stream during capture
    cudaEvent_t join = nullptr;
};

}  // namespace

struct he_mm_plan {
    std::vector<he_mm_job> jobs;
    std::vector<Group> groups;
    std::vector<Ctx *> ctxs;     // distinct contexts of the jobs
    std::vector<long long> ctx_launches;   // kernel launches of one replay, per context
    std::vector<cudaEvent_t> ctx_ev;       // inputs ready on each context's stream
    DevicePool pool;             // the outputs
    cudaStream_t st = nullptr;   // the plan's stream: replays and output copies
    cudaEvent_t fork = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;      // kernel launches one replay performs
    ~he_mm_plan() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (Group &g : groups) {
            if (g.st) cudaStreamDestroy(g.st);
            if (g.join) cudaEventDestroy(g.join);
        }
        if (fork) cudaEventDestroy(fork);
        for (cudaEvent_t e : ctx_ev) cudaEventDestroy(e);
        if (st) cudaStreamDestroy(st);
    }
};

static int plan_fail(int code, const std::string &msg) {
    set_error(msg);
    return code;
}

// Enqueues one group's batched products on its context's current stream
// with scratch from the context's pool (redirected by the caller).
static void record_group(he_mm_plan *P, Group &g) {
    Ctx &c = *g.c;
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

// Runs fn(group) with the group's context launching on `st` (if given) and
// allocating from the group's pool; restores both afterwards.
template <class F>
static void on_branch(Group &g, cudaStream_t st, F fn) {
    Ctx &c = *g.c;
    cudaStream_t keep = c.stream;
    if (st) c.stream = st;
    c.pool.set_redirect(g.pool.get());
    try {
        fn();
    } catch (...) {
        c.pool.set_redirect(nullptr);
        c.stream = keep;
        throw;
    }
    c.pool.set_redirect(nullptr);
    c.stream = keep;
}

extern "C" {

int he_mm_plan_create(const he_mm_job *jobs, int n_jobs, he_mm_plan **out) {
    if (!jobs || n_jobs < 1 || !out) return plan_fail(HE_ERR_ARG, "bad arguments");
    int device = -1;
    for (int i = 0; i < n_jobs; i++) {
        const he_mm_job &j = jobs[i];
        if (!j.A || !j.B || j.A->ctx != j.B->ctx) return plan_fail(HE_ERR_ARG, "bad job operands");
        Ctx *c = j.A->ctx;
        if (device >= 0 && c->device != device) return plan_fail(HE_ERR_ARG, "a plan serves contexts of one device");
        device = c->device;
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
    P->jobs.assign(jobs, jobs + n_jobs);
    typedef std::tuple<Ctx *, int, int, int, int, bool, bool, bool, int, int> Key;
    std::map<Key, int> gi;
    for (int i = 0; i < n_jobs; i++) {
        const he_mm_job &j = jobs[i];
        Ctx *c = j.A->ctx;
        const int n = j.n, lv = std::min(j.A->level, j.B->level);
        Key k(c, lv, n, j.sched.n1_z, j.sched.n1_t, j.A->period != n * n, j.B->period != n * n,
              j.sched.relin_once != 0, j.sched.dcd_z, j.sched.dcd_t);
        auto it = gi.find(k);
        if (it == gi.end()) {
            Group g;
            g.c = c;
            g.level = lv, g.n = n, g.n1z = j.sched.n1_z, g.n1t = j.sched.n1_t;
            g.repA = std::get<5>(k), g.repB = std::get<6>(k), g.relin_once = std::get<7>(k);
            g.dcd_z = j.sched.dcd_z, g.dcd_t = j.sched.dcd_t, g.depth = hmatmul_depth(n, g.dcd_z, g.dcd_t);
            it = gi.emplace(k, (int)P->groups.size()).first;
            P->groups.push_back(std::move(g));
        }
        P->groups[it->second].idx.push_back(i);
        if (std::find(P->ctxs.begin(), P->ctxs.end(), c) == P->ctxs.end()) P->ctxs.push_back(c);
    }
    std::vector<bool> trace;
    for (Ctx *c : P->ctxs) trace.push_back(c->trace), c->trace = false;
    int rc = HE_OK;
    try {
        if (cudaStreamCreateWithFlags(&P->st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming) != cudaSuccess)
            throw HeError(HE_ERR_CUDA, "stream or event creation failed");
        for (Group &g : P->groups) {
            g.pool.reset(new DevicePool);
            g.wo = ct_words(g.c, g.level - g.depth);
            g.O = (u64 *)P->pool.get(g.idx.size() * g.wo * 8);
            if (cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming) != cudaSuccess)
                throw HeError(HE_ERR_CUDA, "stream or event creation failed");
        }
        // 1. recording run, group after group on each context's own stream:
        //    fills every branch pool and the contexts' caches (plaintext
        //    diagonals, launch tuning)
        for (Group &g : P->groups) on_branch(g, nullptr, [&] { record_group(P, g); });
        for (Ctx *c : P->ctxs)
            if (cudaStreamSynchronize(c->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess)
                throw HeError(HE_ERR_CUDA, "recording run failed");
        for (size_t i = 0; i < P->ctxs.size(); i++) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
                throw HeError(HE_ERR_CUDA, "event creation failed");
            P->ctx_ev.push_back(e);
        }
        // 2. capture: every group a branch forked from the plan's stream
        std::vector<long long> n0;
        for (Ctx *c : P->ctxs) n0.push_back(c->n_launch);
        if (cudaStreamBeginCapture(P->st, cudaStreamCaptureModeRelaxed) != cudaSuccess)
            throw HeError(HE_ERR_CUDA, "stream capture could not start");
        try {
            cudaEventRecord(P->fork, P->st);
            for (Group &g : P->groups) {
                cudaStreamWaitEvent(g.st, P->fork, 0);
                on_branch(g, g.st, [&] { record_group(P, g); });
                cudaEventRecord(g.join, g.st);
                cudaStreamWaitEvent(P->st, g.join, 0);
            }
        } catch (...) {
            cudaGraph_t gr = nullptr;
            cudaStreamEndCapture(P->st, &gr);
            if (gr) cudaGraphDestroy(gr);
            throw;
        }
        // the captured launches did not run: count them per replay instead
        P->launches = 0;
        for (size_t i = 0; i < P->ctxs.size(); i++) {
            P->ctx_launches.push_back(P->ctxs[i]->n_launch - n0[i]);
            P->launches += P->ctx_launches.back();
            P->ctxs[i]->n_launch = n0[i];
        }
        if (cudaStreamEndCapture(P->st, &P->graph) != cudaSuccess || !P->graph)
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
    for (size_t i = 0; i < P->ctxs.size(); i++) P->ctxs[i]->trace = trace[i];
    cudaGetLastError();
    if (rc != HE_OK) {
        delete P;
        return rc;
    }
    *out = P;
    return HE_OK;
}

int he_mm_plan_run(he_mm_plan *P, he_ct **outs) {
    if (!P || !outs) return plan_fail(HE_ERR_ARG, "bad arguments");
    std::vector<he_ct *> res(P->jobs.size(), nullptr);
    try {
        // the inputs were written on their contexts' streams
        for (size_t i = 0; i < P->ctxs.size(); i++) {
            cudaEventRecord(P->ctx_ev[i], P->ctxs[i]->stream);
            cudaStreamWaitEvent(P->st, P->ctx_ev[i], 0);
        }
        if (cudaGraphLaunch(P->exec, P->st) != cudaSuccess) throw HeError(HE_ERR_CUDA, "graph launch failed");
        for (size_t i = 0; i < P->ctxs.size(); i++) P->ctxs[i]->n_launch += P->ctx_launches[i];
        for (const Group &g : P->groups) {
            Ctx &c = *g.c;
            const double q2 = (double)c.primes[g.level - g.depth + 1];
            for (size_t t = 0; t < g.idx.size(); t++) {
                const he_mm_job &j = P->jobs[g.idx[t]];
                he_ct *o = new_ct(&c, g.level - g.depth, (j.A->scale * j.B->scale) / q2, j.n * j.n);
                res[g.idx[t]] = o;
                cudaMemcpyAsync(o->d, g.O + t * g.wo, g.wo * 8, cudaMemcpyDeviceToDevice, P->st);
            }
        }
        cudaError_t e = cudaStreamSynchronize(P->st);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) throw HeError(HE_ERR_CUDA, std::string("CUDA error: ") + cudaGetErrorString(e));
        for (Ctx *c : P->ctxs)
            if (device_status(c)) throw HeError(HE_ERR_TIMEOUT, last_error());
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
    if (scratch_bytes) {
        he_mm_plan *Q = const_cast<he_mm_plan *>(P);
        double b = (double)(Q->pool.bytes_in_use() + Q->pool.bytes_cached());
        for (Group &g : Q->groups) b += (double)(g.pool->bytes_in_use() + g.pool->bytes_cached());
        *scratch_bytes = b;
    }
    return HE_OK;
}

int he_mm_plan_destroy(he_mm_plan *P) {
    if (!P) return HE_OK;
    cudaStreamSynchronize(P->st);
    delete P;  // the pools' destructors free the scratch
    return HE_OK;
}

}  // extern "C"
