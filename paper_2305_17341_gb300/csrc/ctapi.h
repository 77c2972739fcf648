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
