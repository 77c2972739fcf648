// stages.h -- the covariance circuit split into stages and the PCA driver,
// for the serving loop (server.cu), which merges the block products of all
// queued jobs into one batched pass.
#pragma once
#include <vector>

#include "ctapi.h"

namespace he {

struct CovStage;

// Stage 1 of HCovMtrx (Sec. 5.2): transposes and replicas of the blocks;
// appends the block products to `prods`.  blocks[l*k + j] must stay alive
// until cov_finish.
CovStage *cov_begin(Ctx *c, he_ct *const *blocks, int nrb, int k, int n, int s, bool centered, int n1z, int n1t,
                    std::vector<ProdSpec> &prods, bool relin_once = false, int dcd_z = 0, int dcd_t = 0);
// Stage 2: takes ownership of the products made from stage 1's list (same
// order); upper[a*k + b] (a <= b) = sum over row blocks, others null.
void cov_upper(Ctx *c, CovStage *S, he_ct *const *outs, std::vector<he_ct *> &upper);
// Stage 3: fills the blocks below the diagonal, aligns levels and (not
// centred) subtracts the mean term; replaces blocks_io in place.
void cov_finish(Ctx *c, CovStage *S, std::vector<he_ct *> &blocks_io);
void cov_free(CovStage *S);

// l_E components of PCA (Sec. 6.2) with the interactive refresh counter.
void pca_run(Ctx *c, he_ct *const *cov, int k, int n, int l_E, he_ct *const *v0, int axis, int l_P,
             const int *counts, double B2, uint32_t &next_obj, int &count, std::vector<he_ct *> &lams,
             std::vector<he_ct *> &V, std::vector<int> &axes);

}  // namespace he
