// server.cu -- the serving loop of include/he.h (he_server_*): per-context
// worker threads that merge the block products of every queued job into
// batched passes over resident keys, with admission against a device-memory
// budget.  The paper keeps the evaluation keys on the server before any
// computation (Sec. 2) and finds its parallel throughput limited by device
// memory (Sec. 7); this file is the scheduler around the circuits of
// eval.cu / pca.cu, which stay the only code that touches ciphertext data.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>

#include "stages.h"

using namespace he;

namespace {

typedef std::chrono::steady_clock Clock;

struct Job {
    uint64_t id = 0;
    he_job spec{};
    std::vector<he_ct *> in;
    std::vector<int> counts;      // PCA Newton counts (copied)
    Ctx *c = nullptr;
    int status = HE_JOB_QUEUED;
    int err = 0;
    std::string msg;
    double t_submit = 0, t_done = 0;
    double charge = 0;            // released when the results are taken
    std::vector<he_ct *> out;
    std::vector<int> aux;
    // per-tick state
    size_t p0 = 0, p1 = 0;        // range in the tick's product list
    CovStage *stage = nullptr;
};

struct Accum {
    int k = 0, n = 0, n1z = 0, n1t = 0, s = 0, level = -1, relin_once = 0;
    CovStage *stage = nullptr;    // plan of the first row block (used for the final mirror)
    std::vector<he_ct *> upper;   // k*k, entries a <= b
};

struct Worker {
    Ctx *c = nullptr;
    std::deque<Job *> q;
    std::map<uint64_t, Accum> acc;
    std::thread th;
};

double ct_bytes(const Ctx *c, int level) { return 16.0 * c->N * (level + 1); }

// Device bytes of one item in a batched product pass at `level`: the n1
// hoisted rotations over Q_l P (two polynomials each), the Decompose digits,
// and about a dozen ciphertexts of intermediates.
double prod_bytes(const Ctx *c, int level, int n1) {
    const double row = 8.0 * c->N;
    return row * ((2.0 * n1 + c->ndig(level)) * c->qp_rows(level) + 24.0 * (level + 1));
}

double key_bytes(const Ctx *c) {
    double b = (double)c->rtk.size() * c->key_words() * 8.0;
    if (c->rlk) b += c->key_words() * 8.0;
    return b;
}

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

bool finished(const Job *J) { return J->status == HE_JOB_DONE || J->status == HE_JOB_FAILED; }

}  // namespace

struct he_server {
    he_server_cfg cfg{};
    std::mutex m;
    std::condition_variable cv_work, cv_done;
    std::vector<std::unique_ptr<Worker>> workers;
    std::unordered_map<uint64_t, Job *> jobs;
    std::deque<Job *> waiting;                          // accepted, not yet admitted (FIFO)
    std::set<std::pair<Ctx *, uint64_t>> acc_charged;   // accumulators already charged
    std::map<std::pair<Ctx *, uint64_t>, double> acc_bytes;
    uint64_t next_id = 1;
    double charged = 0;
    bool stop = false;
    Clock::time_point t0 = Clock::now();
    // statistics, per kind (index 0: all)
    long long submitted[6] = {}, admitted[6] = {}, rejected[6] = {}, completed[6] = {}, failed[6] = {},
              waited[6] = {};
    std::vector<double> lat[6];
    double first_submit[6], last_done[6];
    long long ticks = 0, products = 0, max_tick_products = 0;

    he_server() {
        for (int i = 0; i < 6; i++) first_submit[i] = -1, last_done[i] = -1;
    }
    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
    Worker *worker_of(const Ctx *c) {
        for (auto &w : workers)
            if (w->c == c) return w.get();
        return nullptr;
    }
    void run(Worker *w);
    void tick(Worker *w, std::vector<Job *> &batch);
    // accumulator bytes a row-block job adds when it is admitted (caller holds m)
    double acc_extra(const Job *J) const {
        if (J->spec.kind != HE_JOB_XTX_BLOCK || acc_charged.count(std::make_pair(J->c, J->spec.acc_id))) return 0;
        return (double)J->spec.k * (J->spec.k + 1) / 2 * ct_bytes(J->c, J->in[0]->level - 4);
    }
    // charges the job and queues it on its context's worker (caller holds m)
    void admit(Job *J) {
        const double extra = acc_extra(J);
        charged += J->charge;
        if (extra > 0) {
            auto key = std::make_pair(J->c, J->spec.acc_id);
            acc_charged.insert(key);
            acc_bytes[key] = extra;
            charged += extra;
        }
        const int kd = J->spec.kind;
        for (int x : {0, kd}) admitted[x]++;
        J->status = HE_JOB_QUEUED;
        worker_of(J->c)->q.push_back(J);
        cv_work.notify_all();
    }
    // admits waiting jobs, in order, while they fit (caller holds m)
    void admit_waiting() {
        while (!waiting.empty()) {
            Job *J = waiting.front();
            if (charged + J->charge + acc_extra(J) > cfg.hbm_budget_bytes) break;
            waiting.pop_front();
            admit(J);
        }
    }
};

// --------------------------------------------------------------- one tick
// All jobs of the tick prepare their products; the products run as batched
// passes; then every job finishes in queue order.  A failure inside one job's
// own steps fails only that job; a failure of the shared passes or of the
// stream fails every job of the tick.
void he_server::tick(Worker *w, std::vector<Job *> &batch) {
    Ctx *c = w->c;
    std::vector<ProdSpec> prods;
    auto fail_job = [](Job *j, int code, const std::string &msg) {
        if (j->status == HE_JOB_FAILED) return;
        j->status = HE_JOB_FAILED;
        j->err = code;
        j->msg = msg;
        for (he_ct *o : j->out) free_ct(o);
        j->out.clear();
    };
    auto guarded = [&](Job *j, auto &&fn) {
        try {
            fn();
        } catch (const HeError &e) {
            fail_job(j, e.code, e.what());
        } catch (const std::bad_alloc &) {
            fail_job(j, HE_ERR_OOM, "device or host allocation failed");
        } catch (const std::exception &e) {
            fail_job(j, HE_ERR_ARG, e.what());
        }
    };
    // 1. prepare
    for (Job *j : batch) {
        const he_job &s = j->spec;
        j->p0 = prods.size();
        guarded(j, [&] {
            if (s.kind == HE_JOB_MATMUL) {
                prods.push_back({j->in[0], j->in[1], s.n, s.sched.n1_z, s.sched.n1_t, s.sched.relin_once != 0,
                                 s.sched.dcd_z, s.sched.dcd_t});
            } else if (s.kind == HE_JOB_COVARIANCE) {
                j->stage = cov_begin(c, j->in.data(), s.n_row_blocks, s.k, s.n, s.s, s.centered != 0, s.sched.n1_z,
                                     s.sched.n1_t, prods, s.sched.relin_once != 0, s.sched.dcd_z, s.sched.dcd_t);
            } else if (s.kind == HE_JOB_XTX_BLOCK) {
                j->stage = cov_begin(c, j->in.data(), 1, s.k, s.n, s.s, true, s.sched.n1_z, s.sched.n1_t, prods,
                                     s.sched.relin_once != 0, s.sched.dcd_z, s.sched.dcd_t);
            }
        });
        if (j->status == HE_JOB_FAILED) prods.resize(j->p0);
        j->p1 = prods.size();
    }
    // 2. the shared batched passes
    std::vector<he_ct *> outs;
    bool pass_ok = true;
    std::string pass_msg;
    int pass_code = HE_OK;
    if (!prods.empty()) {
        try {
            run_products(prods, outs, cfg.max_batch);
        } catch (const HeError &e) {
            pass_ok = false, pass_code = e.code, pass_msg = e.what();
        } catch (const std::bad_alloc &) {
            pass_ok = false, pass_code = HE_ERR_OOM, pass_msg = "device allocation failed in a batched pass";
        } catch (const std::exception &e) {
            pass_ok = false, pass_code = HE_ERR_ARG, pass_msg = e.what();
        }
    }
    {
        std::lock_guard<std::mutex> lk(m);
        ticks++;
        products += (long long)prods.size();
        max_tick_products = std::max(max_tick_products, (long long)prods.size());
    }
    // 3. each job's own steps, in queue order
    for (Job *j : batch) {
        const he_job &s = j->spec;
        if (j->status == HE_JOB_FAILED) continue;
        if (j->p1 > j->p0 && !pass_ok) {
            fail_job(j, pass_code, pass_msg);
            continue;
        }
        guarded(j, [&] {
            if (s.kind == HE_JOB_MATMUL) {
                j->out.push_back(outs[j->p0]);
                outs[j->p0] = nullptr;
            } else if (s.kind == HE_JOB_COVARIANCE) {
                std::vector<he_ct *> C;
                std::vector<he_ct *> mine(outs.begin() + j->p0, outs.begin() + j->p1);
                for (size_t t = j->p0; t < j->p1; t++) outs[t] = nullptr;
                cov_upper(c, j->stage, mine.data(), C);
                cov_finish(c, j->stage, C);
                j->out = C;
            } else if (s.kind == HE_JOB_XTX_BLOCK) {
                std::vector<he_ct *> U;
                std::vector<he_ct *> mine(outs.begin() + j->p0, outs.begin() + j->p1);
                for (size_t t = j->p0; t < j->p1; t++) outs[t] = nullptr;
                cov_upper(c, j->stage, mine.data(), U);
                auto it = w->acc.find(s.acc_id);
                if (it == w->acc.end()) {
                    Accum a;
                    a.k = s.k, a.n = s.n, a.n1z = s.sched.n1_z, a.n1t = s.sched.n1_t, a.s = s.s;
                    a.relin_once = s.sched.relin_once != 0;
                    a.level = U[0]->level;
                    a.stage = j->stage;
                    j->stage = nullptr;
                    a.upper = U;
                    w->acc[s.acc_id] = a;
                } else {
                    Accum &a = it->second;
                    bool same = a.k == s.k && a.n == s.n && a.n1z == s.sched.n1_z && a.n1t == s.sched.n1_t &&
                                a.s == s.s && a.level == U[0]->level && a.relin_once == (s.sched.relin_once != 0);
                    if (!same) {
                        for (he_ct *u : U) free_ct(u);
                        throw HeError(HE_ERR_ARG, "row block does not match its accumulator (shape, rows or level)");
                    }
                    for (int t = 0; t < s.k * s.k; t++)
                        if (U[t]) {
                            add(c, a.upper[t]->d, U[t]->d, 1, a.upper[t]->level, a.upper[t]->d);
                            free_ct(U[t]);
                        }
                }
            } else if (s.kind == HE_JOB_XTX_FINAL) {
                auto it = w->acc.find(s.acc_id);
                if (it == w->acc.end()) throw HeError(HE_ERR_ARG, "no accumulator with this id");
                Accum a = it->second;
                w->acc.erase(it);
                std::vector<he_ct *> C = a.upper;
                try {
                    cov_finish(c, a.stage, C);
                } catch (...) {
                    for (he_ct *x : C) free_ct(x);
                    cov_free(a.stage);
                    throw;
                }
                cov_free(a.stage);
                j->out = C;
            } else if (s.kind == HE_JOB_PCA) {
                const int k = s.k;
                uint32_t next = s.refresh_obj;
                int count = 0;
                std::vector<he_ct *> lams, V;
                std::vector<int> axes;
                pca_run(c, j->in.data(), k, s.n, s.l_E, j->in.data() + k * k, s.axis, s.l_P, j->counts.data(), s.B2,
                        next, count, lams, V, axes);
                j->out = lams;
                j->out.insert(j->out.end(), V.begin(), V.end());
                j->aux = axes;
                j->aux.push_back(count);
            }
        });
        if (j->stage) cov_free(j->stage), j->stage = nullptr;
    }
    for (he_ct *o : outs) free_ct(o);
    // 4. the stream decides whether anything of the tick failed on the device
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    const int dev_rc = e == cudaSuccess ? device_status(c) : HE_OK;
    std::lock_guard<std::mutex> lk(m);
    const double t = now();
    for (Job *j : batch) {
        if (e != cudaSuccess) fail_job(j, HE_ERR_CUDA, std::string("CUDA error: ") + cudaGetErrorString(e));
        else if (dev_rc) fail_job(j, dev_rc, "a device-side wait ran out of its iteration limit");
        if (j->status != HE_JOB_FAILED) j->status = HE_JOB_DONE;
        j->t_done = t;
        const int kd = j->spec.kind;
        if (j->status == HE_JOB_DONE) {
            for (int x : {0, kd}) {
                completed[x]++;
                lat[x].push_back(1000.0 * (t - j->t_submit));
                last_done[x] = t;
            }
        } else {
            for (int x : {0, kd}) failed[x]++;
        }
        // jobs without outputs give their charge back now
        if (j->out.empty()) {
            charged -= j->charge;
            j->charge = 0;
        }
        if (kd == HE_JOB_XTX_FINAL) {
            auto key = std::make_pair(c, j->spec.acc_id);
            auto it = acc_bytes.find(key);
            if (it != acc_bytes.end()) {
                charged -= it->second;
                acc_bytes.erase(it);
            }
            acc_charged.erase(key);
        }
    }
    admit_waiting();
    cv_done.notify_all();
}

void he_server::run(Worker *w) {
    cudaSetDevice(w->c->device);
    for (;;) {
        std::vector<Job *> batch;
        {
            std::unique_lock<std::mutex> lk(m);
            cv_work.wait(lk, [&] { return stop || !w->q.empty(); });
            if (w->q.empty()) return;  // stop requested and nothing left
            // a tick takes every queued job up to and including the first
            // X^T X final, so that a final sees exactly the row blocks queued
            // before it
            while (!w->q.empty()) {
                Job *j = w->q.front();
                w->q.pop_front();
                j->status = HE_JOB_RUNNING;
                batch.push_back(j);
                if (j->spec.kind == HE_JOB_XTX_FINAL) break;
            }
        }
        tick(w, batch);
    }
}

// ----------------------------------------------------------------- checks
static int reject(const char *msg, int code) {
    set_error(msg);
    return code;
}

// Validates a job and computes its charge.  Returns HE_OK or an error code.
static int check_job(he_server *S, const he_job *j, Ctx **ctx_out, double *charge, std::vector<long> *steps,
                     bool *need_rlk, long *skip_from) {
    if (!j || (j->n_in > 0 && !j->in)) return reject("null job or inputs", HE_ERR_ARG);
    Ctx *c = nullptr;
    for (int i = 0; i < j->n_in; i++) {
        if (!j->in[i]) return reject("null input ciphertext", HE_ERR_ARG);
        if (c && j->in[i]->ctx != c) return reject("inputs of different contexts", HE_ERR_ARG);
        c = j->in[i]->ctx;
    }
    const int kind = j->kind;
    if (j->ctx) {
        if (c && c != &j->ctx->c) return reject("inputs not of the job's context", HE_ERR_ARG);
        c = &j->ctx->c;
    }
    if (!c || !S->worker_of(c)) return reject("the job's context is not served here", HE_ERR_ARG);
    *ctx_out = c;
    *need_rlk = false;
    *skip_from = c->S;
    const int n = j->n;
    auto sched_ok = [&] {
        return pow2(j->sched.n1_z) && pow2(j->sched.n1_t) && j->sched.n1_z <= n && j->sched.n1_t <= n &&
               j->sched.n1_z <= 32 && j->sched.n1_t <= 32;
    };
    if (!pow2(n) || (long)n * n > c->S)
        return reject("n must be a power of two with n^2 <= slots", HE_ERR_ARG);
    const double cb = ct_bytes(c, c->L);
    switch (kind) {
    case HE_JOB_MATMUL: {
        if (j->n_in != 2 || !sched_ok()) return reject("a product takes A, B and a valid schedule", HE_ERR_ARG);
        int lv = std::min(j->in[0]->level, j->in[1]->level);
        if ((j->sched.dcd_z && (j->sched.dcd_z >= n || j->sched.dcd_z % j->sched.n1_z)) ||
            (j->sched.dcd_t && (j->sched.dcd_t >= n || j->sched.dcd_t % j->sched.n1_t)))
            return reject("a decomposition needs n' < n with the baby steps dividing n'", HE_ERR_ARG);
        if (lv < hmatmul_depth(n, j->sched.dcd_z, j->sched.dcd_t))
            return reject("not enough levels for the product", HE_ERR_LEVEL);
        *steps = matmul_steps(n, j->sched.n1_z, j->sched.n1_t, c->S, j->sched.dcd_z, j->sched.dcd_t);
        if (j->in[0]->period == n * n && j->in[1]->period == n * n) *skip_from = (long)n * n;
        *need_rlk = true;
        *charge = prod_bytes(c, lv, std::max(j->sched.n1_z, j->sched.n1_t)) + ct_bytes(c, lv - 3);
        return HE_OK;
    }
    case HE_JOB_COVARIANCE:
    case HE_JOB_XTX_BLOCK: {
        const int nrb = kind == HE_JOB_XTX_BLOCK ? 1 : j->n_row_blocks, k = j->k;
        if (nrb < 1 || k < 1 || j->s < 1 || j->n_in != nrb * k || !sched_ok())
            return reject("covariance blocks: n_in must be n_row_blocks * k with a valid schedule", HE_ERR_ARG);
        if ((j->sched.dcd_z && (j->sched.dcd_z >= n || j->sched.dcd_z % j->sched.n1_z)) ||
            (j->sched.dcd_t && (j->sched.dcd_t >= n || j->sched.dcd_t % j->sched.n1_t)))
            return reject("a decomposition needs n' < n with the baby steps dividing n'", HE_ERR_ARG);
        for (int i = 0; i < j->n_in; i++)
            if (j->in[i]->level != j->in[0]->level) return reject("blocks at different levels", HE_ERR_LEVEL);
        if (j->in[0]->level < hmatmul_depth(n, j->sched.dcd_z, j->sched.dcd_t) + 3)
            return reject("the covariance circuit needs the product's depth + 3 levels", HE_ERR_LEVEL);
        *steps = matmul_steps(n, j->sched.n1_z, j->sched.n1_t, c->S, j->sched.dcd_z, j->sched.dcd_t);
        std::vector<long> g = transpose_steps(n, j->sched.n1_z, c->S);
        steps->insert(steps->end(), g.begin(), g.end());
        if (kind == HE_JOB_COVARIANCE && !j->centered)
            for (long i = n; i < (long)n * n; i <<= 1) steps->push_back(i);
        *need_rlk = true;
        const int lv = j->in[0]->level, np = nrb * k * (k + 1) / 2;
        *charge = 2.0 * nrb * k * ct_bytes(c, lv) + std::min(np, S->cfg.max_batch) * prod_bytes(c, lv - 1, j->sched.n1_z) +
                  np * ct_bytes(c, lv - 4) + (double)k * k * ct_bytes(c, lv - 4);
        if (kind == HE_JOB_COVARIANCE && !j->centered) *charge += 4.0 * k * ct_bytes(c, lv);
        return HE_OK;
    }
    case HE_JOB_XTX_FINAL:
        if (j->n_in != 0) return reject("an X^T X final takes no inputs", HE_ERR_ARG);
        if (j->k < 1) return reject("an X^T X final needs k", HE_ERR_ARG);
        if (!pow2(n) || (long)n * n > c->S || !sched_ok())
            return reject("an X^T X final needs n and the G baby steps", HE_ERR_ARG);
        *charge = (double)j->k * j->k * ct_bytes(c, c->L) + prod_bytes(c, c->L, j->sched.n1_z);
        *steps = transpose_steps(n, j->sched.n1_z, c->S);
        *skip_from = (long)n * n;
        return HE_OK;
    case HE_JOB_PCA: {
        const int k = j->k;
        if (k < 1 || j->l_E < 1 || j->l_P < 1 || (j->axis != 0 && j->axis != 1) || !(j->B2 > 0) || !j->newton_counts ||
            j->n_in != k * k + j->l_E * k)
            return reject("PCA: n_in must be k*k covariance blocks plus l_E*k start vectors", HE_ERR_ARG);
        if (c->L < 4) return reject("the PowerMethod needs a chain of at least 4 levels", HE_ERR_LEVEL);
        for (long i = 1; i < (long)n * n; i <<= 1) {
            steps->push_back(i);
            steps->push_back((long)n * n - i);
        }
        *need_rlk = true;
        *charge = (3.0 * k * k + 8.0 * k + 16.0) * cb + 2.0 * prod_bytes(c, c->L, 1) +
                  (double)(j->l_E + j->l_E * k) * cb;
        return HE_OK;
    }
    default:
        return reject("unknown job kind", HE_ERR_ARG);
    }
}

extern "C" {

int he_server_create(const he_server_cfg *cfg, he_ctx *const *ctxs, int n_ctx, he_server **out) {
    if (!cfg || !ctxs || n_ctx < 1 || !out || cfg->max_batch < 1 || !(cfg->hbm_budget_bytes > 0))
        return reject("bad arguments", HE_ERR_ARG);
    std::set<Ctx *> seen;
    for (int i = 0; i < n_ctx; i++) {
        if (!ctxs[i] || !seen.insert(&ctxs[i]->c).second) return reject("null or repeated context", HE_ERR_ARG);
    }
    he_server *S = new (std::nothrow) he_server;
    if (!S) return reject("host allocation failed", HE_ERR_OOM);
    S->cfg = *cfg;
    for (int i = 0; i < n_ctx; i++) {
        auto w = std::make_unique<Worker>();
        w->c = &ctxs[i]->c;
        S->workers.push_back(std::move(w));
    }
    for (auto &w : S->workers) {
        Worker *wp = w.get();
        wp->th = std::thread([S, wp] { S->run(wp); });
    }
    *out = S;
    return HE_OK;
}

int he_server_submit(he_server *S, const he_job *j, uint64_t *job_id) {
    if (!S || !j || !job_id) return reject("bad arguments", HE_ERR_ARG);
    Ctx *c = nullptr;
    double charge = 0;
    std::vector<long> steps;
    bool need_rlk = false;
    long skip_from = 0;
    const int kind = (j->kind >= 1 && j->kind <= 5) ? j->kind : 0;
    int rc = check_job(S, j, &c, &charge, &steps, &need_rlk, &skip_from);
    if (rc == HE_OK) {
        if (long miss = first_missing_key(c, steps, skip_from)) {
            set_error("rotation key for step " + std::to_string(miss) + " missing");
            rc = HE_ERR_KEY_MISSING;
        } else if (need_rlk && !c->rlk) {
            rc = reject("relinearisation key missing", HE_ERR_KEY_MISSING);
        }
    }
    std::lock_guard<std::mutex> lk(S->m);
    for (int x : {0, kind}) S->submitted[x]++;
    if (rc != HE_OK) {
        if (rc == HE_ERR_ADMISSION)
            for (int x : {0, kind}) S->rejected[x]++;
        return rc;
    }
    if (S->stop) return reject("the server is stopping", HE_ERR_ARG);
    Job *J = new Job;
    J->spec = *j;
    J->in.assign(j->in, j->in + j->n_in);
    J->spec.in = nullptr;
    if (kind == HE_JOB_PCA) {
        J->counts.assign(j->newton_counts, j->newton_counts + j->l_P);
        J->spec.newton_counts = nullptr;
    }
    J->c = c;
    J->charge = charge;
    const double extra = S->acc_extra(J);
    const bool fits_now = S->waiting.empty() && S->charged + charge + extra <= S->cfg.hbm_budget_bytes;
    if (charge + extra > S->cfg.hbm_budget_bytes || (!fits_now && S->cfg.reject_when_full)) {
        delete J;
        for (int x : {0, kind}) S->rejected[x]++;
        return reject("rejected by the device-memory budget", HE_ERR_ADMISSION);
    }
    J->id = S->next_id++;
    J->t_submit = S->now();
    for (int x : {0, kind})
        if (S->first_submit[x] < 0) S->first_submit[x] = J->t_submit;
    S->jobs[J->id] = J;
    if (fits_now) {
        S->admit(J);
    } else {
        J->status = HE_JOB_WAITING;
        S->waiting.push_back(J);
        for (int x : {0, kind}) S->waited[x]++;
    }
    *job_id = J->id;
    return HE_OK;
}

int he_server_poll(he_server *S, uint64_t id, int *status, int *error, double *latency_ms) {
    if (!S) return reject("bad arguments", HE_ERR_ARG);
    std::lock_guard<std::mutex> lk(S->m);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return reject("unknown job id", HE_ERR_ARG);
    Job *J = it->second;
    if (status) *status = J->status;
    if (error) *error = J->err;
    if (latency_ms) *latency_ms = finished(J) ? 1000.0 * (J->t_done - J->t_submit) : 0.0;
    return HE_OK;
}

int he_server_wait(he_server *S, uint64_t id, double timeout_s, int *status) {
    if (!S || timeout_s < 0) return reject("bad arguments", HE_ERR_ARG);
    std::unique_lock<std::mutex> lk(S->m);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return reject("unknown job id", HE_ERR_ARG);
    Job *J = it->second;
    bool ok = S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                  [&] { return finished(J); });
    if (status) *status = J->status;
    if (!ok) return reject("timed out waiting for the job", HE_ERR_TIMEOUT);
    return HE_OK;
}

int he_server_result(he_server *S, uint64_t id, he_ct **outs, int max_outs, int *n_outs, int *aux, int max_aux,
                     int *n_aux) {
    if (!S || !n_outs || (max_outs > 0 && !outs)) return reject("bad arguments", HE_ERR_ARG);
    std::lock_guard<std::mutex> lk(S->m);
    auto it = S->jobs.find(id);
    if (it == S->jobs.end()) return reject("unknown job id", HE_ERR_ARG);
    Job *J = it->second;
    if (!finished(J)) return reject("the job has not finished", HE_ERR_ARG);
    if (J->status == HE_JOB_FAILED) {
        int code = J->err ? J->err : HE_ERR_ARG;
        set_error(J->msg);
        S->charged -= J->charge;
        S->jobs.erase(it);
        delete J;
        S->admit_waiting();
        return code;
    }
    if ((int)J->out.size() > max_outs) return reject("max_outs is smaller than the job's outputs", HE_ERR_ARG);
    if (aux && (int)J->aux.size() > max_aux) return reject("max_aux is smaller than the job's aux values", HE_ERR_ARG);
    for (size_t i = 0; i < J->out.size(); i++) outs[i] = J->out[i];
    *n_outs = (int)J->out.size();
    if (aux)
        for (size_t i = 0; i < J->aux.size(); i++) aux[i] = J->aux[i];
    if (n_aux) *n_aux = (int)J->aux.size();
    S->charged -= J->charge;
    S->jobs.erase(it);
    delete J;
    S->admit_waiting();
    return HE_OK;
}

int he_server_stats(he_server *S, int kind, he_serving_stats *o) {
    if (!S || !o || kind < 0 || kind > 5) return reject("bad arguments", HE_ERR_ARG);
    std::lock_guard<std::mutex> lk(S->m);
    he_serving_stats r{};
    r.submitted = S->submitted[kind];
    r.admitted = S->admitted[kind];
    r.rejected = S->rejected[kind];
    r.completed = S->completed[kind];
    r.failed = S->failed[kind];
    r.waited = S->waited[kind];
    std::vector<double> v = S->lat[kind];
    std::sort(v.begin(), v.end());
    auto rank = [&](double q) {
        size_t i = (size_t)std::ceil(q * v.size());
        return v[i == 0 ? 0 : i - 1];
    };
    if (!v.empty()) {
        r.p50_ms = rank(0.50);
        r.p99_ms = rank(0.99);
        double s = 0;
        for (double x : v) s += x;
        r.mean_ms = s / v.size();
        r.max_ms = v.back();
        double span = S->last_done[kind] - S->first_submit[kind];
        r.jobs_per_s = span > 0 ? v.size() / span : 0.0;
    }
    r.ticks = S->ticks;
    r.products = S->products;
    r.max_products_per_tick = S->max_tick_products;
    r.charged_bytes = S->charged;
    double kb = 0;
    for (auto &w : S->workers) kb += key_bytes(w->c);
    r.key_bytes = kb;
    *o = r;
    return HE_OK;
}

int he_server_destroy(he_server *S) {
    if (!S) return reject("bad arguments", HE_ERR_ARG);
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->stop = true;
        // jobs never admitted are dropped (they hold no device memory)
        for (Job *J : S->waiting) {
            S->jobs.erase(J->id);
            delete J;
        }
        S->waiting.clear();
    }
    S->cv_work.notify_all();
    for (auto &w : S->workers)
        if (w->th.joinable()) w->th.join();
    for (auto &kv : S->jobs) {
        for (he_ct *o : kv.second->out) free_ct(o);
        delete kv.second;
    }
    for (auto &w : S->workers)
        for (auto &kv : w->acc) {
            for (he_ct *u : kv.second.upper) free_ct(u);
            cov_free(kv.second.stage);
        }
    delete S;
    return HE_OK;
}

}  // extern "C"
