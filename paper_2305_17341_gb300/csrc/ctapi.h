// ctapi.h -- the opaque handles of include/he.h and their allocation.
#pragma once
#include "eval.h"

struct he_ctx {
    he::Ctx c;
};

// A ciphertext handle: NTT-domain data [2][level+1][N] from the context's pool.
struct he_ct {
    he::Ctx *ctx;
    u64 *d;
    int level;
    double scale;
    int period;
};

namespace he {
he_ct *new_ct(Ctx *c, int level, double scale, int period);
void free_ct(he_ct *ct);
size_t ct_words(const Ctx *c, int level);
}  // namespace he

namespace he {
// One encrypted product A*B of n x n blocks with baby-step counts n1z, n1t.
struct ProdSpec {
    const he_ct *A, *B;
    int n, n1z, n1t;
    bool relin_once = false;
    int dcd_z = 0, dcd_t = 0;
};

// Runs every product of `prods`, grouping those that share (context, level,
// n, n1z, n1t, replication state) into batched passes of at most max_batch
// items (max_batch <= 0: unbounded).  outs[i] receives product i (owned by
// the caller).  Enqueues on the contexts' streams without synchronising; on
// an exception every output already made is freed.
void run_products(const std::vector<ProdSpec> &prods, std::vector<he_ct *> &outs, int max_batch);

// Rotation steps (mod slots) of the product schedule and of the transpose G,
// as he_rot_steps_for_matmul / he_rot_steps_for_transpose list them.
std::vector<long> matmul_steps(int n, int n1z, int n1t, long slots, int dcd_z = 0, int dcd_t = 0);
std::vector<long> transpose_steps(int n, int n1, long slots);
// First step of `steps` with no rotation key in c (steps >= skip_from are
// ignored), or 0 if every key is present.
long first_missing_key(const Ctx *c, const std::vector<long> &steps, long skip_from);
}  // namespace he
