// eval.h -- batched evaluation routines (see eval.cu).
#pragma once
#include <stdexcept>

#include "he_internal.h"

namespace he {

struct HeError : std::runtime_error {
    int code;
    HeError(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

uint32_t galois_of_step(const Ctx *c, long step);
void create_keys(Ctx *c);
u64 *gen_rotation_key(Ctx *c, uint32_t g);
u64 *gen_relin_key(Ctx *c);
void encrypt_poly(Ctx *c, const u64 *m_ntt, int level, uint32_t obj, bool refresh, u64 *out);
void encode_to(Ctx *c, const double *d_zr, const double *d_zi, double scale, u64 *out, int rows, const RowMap &rm);
const char *last_error();
double bfly_peak(int iters);
double mac_peak(int iters);

void modup(Ctx *c, const u64 *poly, long item_s, int B, int level, u64 *digits);
// add (may be null, item stride add_s; may equal out): out = add + ModDown(u)
void moddown(Ctx *c, const u64 *u, int items, int level, u64 *out, long out_s, const u64 *add = nullptr,
             long add_s = 0);
void rot_qp(Ctx *c, const u64 *ct, int B, int level, const u64 *digits, uint32_t g, u64 *out);
void rot_qp_multi(Ctx *c, const u64 *ct, int B, int level, const u64 *digits, const uint32_t *gs, int G,
                  u64 *const *outs);
void rotate_digits(Ctx *c, const u64 *ct, int B, int level, const u64 *digits, uint32_t g, u64 *out);
void rotate(Ctx *c, const u64 *ct, int B, int level, uint32_t g, u64 *out);
void rescale(Ctx *c, const u64 *in, int B, int level, u64 *out);
void drop(Ctx *c, const u64 *in, int B, int level, int to, u64 *out);
// b may sit at a higher level b_level (its first level + 1 limbs are used in place)
void mult_relin(Ctx *c, const u64 *a, const u64 *b, int B, int level, u64 *out, bool accumulate = false,
                int b_level = -1);
void add(Ctx *c, const u64 *a, const u64 *b, int B, int level, u64 *out);
const u64 *get_pt(Ctx *c, int kind, int n, long t, long rot, double value, int k, int level,
                  const DcdFactor *fac = nullptr);
void lintrans(Ctx *c, const u64 *in, int B, int level, int kind, int n, long a, int n1, int gi0, int gi1,
              double value, u64 *out, const DcdFactor *fac = nullptr, int n1_sub = 0);
// Decompositions (dcd.cu): which = 0 (Z_1), 1 (Z_2), 2 (T); levels a chain consumes.
const DcdChain &dcd_chain(Ctx *c, int which, int n, int n_prime);
// Factors (levels) of the decomposed Z (is_t false) or T; 1 without n'.
int dcd_levels(int n, int n_prime, bool is_t);
void launch_dcd_fill(Ctx *c, double *out, const int *diag, int n, long t, long rot, double value, cudaStream_t st);
// Levels a product consumes: the Z/T stage (1, or the longer decomposition
// chain), C^k, and the multiplication.
// sigma (is_t false) or tau of B items through the undecomposed transform or
// the decomposition chains, output dropped to level `to`.
void zt_stage_public(Ctx *c, const u64 *in, int B, int level, bool is_t, int n, int n1, int np, int to, u64 *out);
inline int hmatmul_depth(int n, int dcd_z, int dcd_t) {
    int mz = dcd_levels(n, dcd_z, false), mt = dcd_levels(n, dcd_t, true);
    return (mz > mt ? mz : mt) + 2;
}
void replicate(Ctx *c, u64 *ct, int B, int level, int n);
void hmatmul(Ctx *c, const u64 *A, const u64 *Bm, int Bn, int level, int n, int n1z, int n1t, u64 *out,
             bool relin_once = false, int dcd_z = 0, int dcd_t = 0);
// products A[ia[p]] B[ib[p]] of shared operands (each operand's transforms once)
void hmatmul_pairs(Ctx *c, const u64 *A, int nA, const u64 *Bm, int nB, const int *ia, const int *ib, int P,
                   int level, int n, int n1z, int n1t, u64 *out, bool relin_once = false, int dcd_z = 0,
                   int dcd_t = 0);

}  // namespace he
