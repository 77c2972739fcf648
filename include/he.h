/*
 * he.h -- C ABI of the GB300-native RNS-CKKS homomorphic matrix
 * multiplication library (one process, one GPU, sm_103a).
 *
 * Paper: "Improved Privacy-Preserving PCA Using Optimized Homomorphic Matrix
 * Multiplication" (arXiv 2305.17341).  The problem statement is the paper's
 * client/cloud model (Sec. 7.2.1): the client encrypts, the cloud computes on
 * ciphertexts, the client decrypts.  The primitives follow App. A (full-RNS
 * CKKS), the matrix product follows eq. 4 with the hoisting of Sec. 4.1.
 *
 * Conventions
 *   - Every function returns int: HE_OK (0) or a negative HE_ERR_* code.
 *     he_last_error() returns a thread-local message for the last failure.
 *   - he_ctx and he_ct are opaque, library-owned handles.  Ciphertexts and keys
 *     live in device memory (HBM) until freed with he_ct_free / he_ctx_destroy.
 *   - Host arrays passed in are caller-owned and only read or written during
 *     the call.  Calls that return host data synchronise the context's stream.
 *   - A context is used from one host thread at a time.
 *   - Ciphertext residues are exported in coefficient form, limb-major:
 *     [poly 0..1][limb 0..level][coefficient 0..N-1], each in [0, q_limb).
 *   - Matrices are packed row-major into slots [0, rows*cols) (Sec. 3.4);
 *     the remaining slots are zero.
 */
#ifndef HE_GB300_H
#define HE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HE_OK 0
#define HE_ERR_ARG (-1)         /* invalid argument (null handle, bad size) */
#define HE_ERR_PARAM (-2)       /* invalid or unsupported parameters */
#define HE_ERR_LEVEL (-3)       /* not enough levels left for the operation */
#define HE_ERR_SCALE (-4)       /* operands with different scales */
#define HE_ERR_KEY_MISSING (-5) /* a rotation or relinearisation key is absent */
#define HE_ERR_OOM (-6)         /* device allocation failed */
#define HE_ERR_ADMISSION (-7)   /* rejected by the device-memory budget */
#define HE_ERR_TIMEOUT (-8)     /* a bounded wait expired */
#define HE_ERR_CUDA (-9)        /* a CUDA runtime call failed */

typedef struct he_ctx he_ctx;
typedef struct he_ct he_ct;

/* Setparams (App. A): ring degree N = 2^logN; q_0..q_L and p_0..p_{alpha-1}
 * are primes = 1 mod 2N of the given bit sizes (q_0 and the p's: the largest
 * such primes below 2^bits, descending; q_1..q_L alternate around 2^bits:
 * first above, first below, second above, ...).  Digits of the hybrid key
 * switch hold alpha = n_p consecutive q's. */
typedef struct he_params {
    int logN;         /* 10..17 */
    int n_q;          /* L + 1, 1..48 */
    int q_bits[48];   /* each 30..60 */
    int n_p;          /* alpha, 1..4 */
    int p_bits[4];    /* each 30..60 */
    int log_delta;    /* default encoding scale 2^log_delta */
    double sigma;     /* standard deviation of the error distribution */
} he_params;

/* Schedule of the hoisted JKLS product (Table 1 "Optimized"): baby-step
 * counts of the double-hoisted BSGS transforms Z (sigma) and T (tau), both
 * powers of two dividing n, and the relinearisation placement:
 *   relin_once = 0  every product A^(k) B^(k) is relinearised (DMatrixMult's
 *                   Mult, Sec. 4.3) before the sum -- the paper's circuit;
 *   relin_once = 1  the n tensors (d0, d1, d2) are summed and relinearised
 *                   once (App. A Mult applied to the sum; not in the paper:
 *                   n - 1 fewer key switches, different noise, so different
 *                   bits). */
typedef struct he_mm_sched {
    int n1_z;
    int n1_t;
    int relin_once;
    /* Diagonal Convergence Decomposition (Sec. 4.2, DMatrixMult): 0 applies Z
     * and T undecomposed (one level each, in parallel); n' > 0 applies Z as
     * the factor chains of DCDforZ with maximum diagonal n' (dcd_z) and T as
     * the chain of DCDforT with maximum diagonal n' n (dcd_t), trading
     * floor((n-1)/n') + 1 levels (n/n' for n' | n) for fewer rotation keys
     * (Table 2).  n' < n and
     * the baby steps must divide n'.  A product consumes 2 + the longest
     * chain (3 without decomposition). */
    int dcd_z;
    int dcd_t;
} he_mm_sched;

/* One product of a batch: out = A . B for n x n matrices (eq. 4). */
typedef struct he_mm_job {
    const he_ct *A;
    const he_ct *B;
    int n;
    he_mm_sched sched;
} he_mm_job;

/* Message of the last failing call on this thread ("" if none). */
const char *he_last_error(void);

/* Parameter presets.  cfg_id 1: logN 14, q 60+3x40, p 60 (32x32 products);
 * 2: logN 16, q 60+20x40, p 2x60 (128x128 products, covariance);
 * 3: logN 16, q 60+13x40, p 2x60 (PowerMethod chain, Sec. 7.2.3);
 * 4: logN 15 with the chain of preset 2.  log_delta 40, sigma 3.2. */
int he_params_default(int cfg_id, he_params *out);

/* Creates a context on the current CUDA device: primes, NTT tables and the
 * secret/public key pair (SecKeyGen, PubKeyGen of App. A) drawn from the
 * Philox4x32-10 stream keyed by `seed`.  *out receives the handle. */
int he_ctx_create(const he_params *prm, uint64_t seed, he_ctx **out);
int he_ctx_destroy(he_ctx *ctx);

/* Makes the context launch on `stream` (a cudaStream_t; NULL = the context's
 * own stream).  The caller keeps ownership of a stream it passes. */
int he_ctx_set_stream(he_ctx *ctx, void *stream);

/* Launch-geometry autotuner (on by default): the first MultSum of each
 * (level, batch size, number of hoisted rotations) times its launch plans --
 * rotations per launch (1, 2, 4 or 8 sharing one read of the digits), items
 * per CTA, cached or streaming digit loads -- on those very launches and keeps
 * the fastest for the context; the first NTT of the context times the NTT
 * passes compiled for 2 and for 3 CTAs per SM on scratch rows.  Plans compute
 * identical words; only speed differs.  on = 0 uses the fixed defaults (8
 * rotations per launch, 8 items per CTA, cached loads; 2 NTT CTAs per SM). */
int he_ctx_set_autotune(he_ctx *ctx, int on);

/* Pins every MultSum launch of the context to one launch variant, with up to
 * 8 hoisted rotations per launch and no tuning (-1 returns to the tuner /
 * defaults).  Variants compute identical words; this is for tests and
 * measurement.  0..7: one thread per (item, coefficient, row), digit and key
 * words loaded by the threads (bits 0-1: 8/4/2/1 items per CTA, bit 2:
 * streaming digit loads); 8, 9, 10: persistent CTAs fed by bulk
 * asynchronous global->shared copies of digit and key segments issued by a
 * producer warp, tiles of 64 coefficients x 8 items (8 stages), 128 x 4 (6)
 * and 256 x 2 (4).
 * 16, 20: variants 0 and 4 with an L2 prefetch of the digit and key words
 * two digits ahead; 32, 36: variants 0 and 4 compiled for more resident CTAs
 * per SM (fewer registers), 48 the same with the prefetch of 16; 64, 65:
 * the rotations of a launch split over the CTA's warps, 1 or 2 per thread (a
 * thread's state no longer grows with the number of rotations; where that
 * number does not divide the 8 warps, as 32); 80, 84: two adjacent
 * coefficients per thread with 16-byte digit and key loads (cached /
 * streaming digit loads), more CTAs per SM, for at most two rotations per
 * launch (more: as 32 / 36); 96, 97: as 64, 65 with two coefficients per
 * thread and 16-byte loads.  The fused MultSum of a product's C^k babies
 * (both sources of a giant with their masks) follows: 96 and 97 pin its
 * rotations-split-over-warps form (97 with launches of 8 rotations where 8
 * remain), every other variant its thread-per-word form.  Errors: HE_ERR_ARG for other values. */
int he_ctx_set_multsum_variant(he_ctx *ctx, int variant);

/* Pins the context's NTT passes (N = 2^14 .. 2^16) to one variant, without
 * tuning (-1 returns to the tuner, which times them at the next transform).
 * Variants compute identical words; this is for tests and measurement.
 * 2, 3, 5: one 8-stage tile per CTA, 2, 3 or 4 CTAs per SM (forward and
 * inverse); 4: forward passes on persistent CTAs whose tiles arrive through
 * bulk asynchronous copies (a producer warp, two buffers), inverse as 3;
 * 6 (N = 2^16; otherwise as 3): the forward transform of a limb in one pass
 * by a cluster of 8 CTAs exchanging through distributed shared memory (one
 * read and one write of every word), inverse as 3.
 * Errors: HE_ERR_ARG for other values. */
int he_ctx_set_ntt_variant(he_ctx *ctx, int variant);

/* Rows per launch pair of the two-pass NTTs (both directions): with rows > 0
 * a transform of many rows runs as chunks of that many rows, pass 0 then
 * pass 1 per chunk, so that pass 1 finds pass 0's output in L2 when a
 * chunk's rows fit there (0: every row in one pair of launches).  The tuner
 * sets it per direction (all, 96 MiB or 48 MiB chunks) when it tunes the
 * NTT; this call overrides it until the next tuning.  Words are identical.
 * Errors: HE_ERR_ARG for a negative count. */
int he_ctx_set_ntt_chunk(he_ctx *ctx, int rows);

/* Newton composition for the PowerMethod's inverse square root (Sec. 7: two
 * InvSRT iterations composited into one that spends one level less).  With
 * on != 0, he_power_method / he_pca / PCA jobs on this context run each pair
 * of Newton iterations as one composite of five levels instead of six
 * (u = x y^2; y1/2 = (y/4)(3 - u); x y1^2 = (u/4)(3 - u)^2;
 * y2 = (y1/2)(3 - x y1^2)); an odd count ends with one ordinary step.  The
 * results are those of the same schedule in the oracle (bit-exact), not of
 * the uncomposed circuit.  Off by default. */
int he_ctx_set_newton_composition(he_ctx *ctx, int on);

/* Packed eigenvector refresh (App. C: the components of the approximate
 * eigenvector, spread over k ciphertexts, are gathered into one ciphertext,
 * refreshed once and spread back).  With on != 0, the PowerMethod on this
 * context checks the vector before each covariance transformation: when a
 * segment has fewer than 2 levels left and every segment has at least 1,
 * segment j keeps only its row (axis 0) or column (axis 1) j, the k lines are
 * added and refreshed as one ciphertext, and each segment is cut out and
 * replicated again (one level and log2 n rotations each); the segments come
 * back at level L - 1.  Results are those of the same schedule in the oracle
 * (bit-exact).  Off by default. */
int he_ctx_set_packed_refresh(he_ctx *ctx, int on);

/* The autotuner's record: one line per timed launch plan (kernel, shape,
 * plan, best of two device times in ms).  Copies at most cap - 1 bytes and a
 * terminating NUL into out; *len (may be NULL) receives the full length. */
int he_autotune_log(const he_ctx *ctx, char *out, int cap, int *len);

/* Copies the primes: q_out[0..L] and p_out[0..alpha-1] (host arrays). */
int he_ctx_primes(const he_ctx *ctx, uint64_t *q_out, uint64_t *p_out);

/* Basic sizes of the context: N, slots, L, alpha, dnum (any pointer may be NULL). */
int he_ctx_info(const he_ctx *ctx, int *N, int *slots, int *L, int *alpha, int *dnum);

/* Secret key s (SecKeyGen, App. A) as signed coefficients s_i in {-1, 0, 1}
 * (host array of N entries).  The secret key belongs to the client; this call
 * is for the client side of the protocol (decryption, refresh) and tests. */
int he_sk_export(const he_ctx *ctx, int64_t *s_out);

/* SwitchKeyGen (App. A) for the rotation keys rtk_k = swk(s, kappa_{5^k}(s))
 * of every step in rot_steps[0..n_steps) (taken mod the slot count; 0 is
 * ignored) and, if want_relin, the relinearisation key swk(s, s^2).  Keys are
 * generated on the device and stay resident ("loaded into memory prior to the
 * computation", Sec. 3.3).  Existing keys are kept. */
int he_keygen(he_ctx *ctx, const int32_t *rot_steps, int n_steps, int want_relin);

/* Lists the rotation steps of the hoisted product schedule for n x n
 * matrices in `slots` slots: replication steps, Z babies/giants, T
 * babies/giants, the C^k step -n (Table 1 MinRotKeys).  out must hold 4n+64
 * entries; *count receives the number written. */
int he_rot_steps_for_matmul(int n, int n1_z, int n1_t, int slots, int32_t *out, int *count);

/* Steps of the transposition G (BSGS with stride n-1, baby count n1). */
/* The rotation steps of the product under a full schedule (baby steps and
 * decompositions): he_rot_steps_for_matmul's set with Z's and T's steps
 * replaced by those of their decompositions when dcd_z / dcd_t are set. */
int he_rot_steps_for_sched(int n, const he_mm_sched *sched, int slots, int32_t *out, int *count);

int he_rot_steps_for_transpose(int n, int n1, int slots, int32_t *out, int *count);

/* Simple key substitution (Sec. 4.2, Table 2's SmpKeySub rows) for the
 * double-hoisted BSGS of Z (kind 0, sigma, eq. 5) or T (kind 1, tau, eq. 6):
 * the babies use only the rotation keys of the head a s, 0 < s < n1_sub, of
 * their arithmetic progression (a = 1 for Z, n for T).  They are formed in
 * groups of n1_sub - 1; each later group starts from the last baby of the
 * previous one, ModDown'd and Decomposed (one more Decompose and ModDown per
 * group), so the transform needs n1_sub + 2 n/n1 - 2 (Z) or n1_sub + n/n1 - 2
 * (T) matrix rotation keys instead of n1 + 2 n/n1 - 2 or n1 + n/n1 - 2, at
 * the same MultSum count.  n1 is a power of two dividing n, 2 <= n1_sub <=
 * n1 (n1_sub = n1 is the plain transform).  The input is replicated to
 * period n^2 first when it is not; the output is one level lower.
 * he_rot_steps_for_ksub lists the slot rotation steps (the transform's and
 * the replication's): on entry *count is the capacity of out, on return the
 * number of steps; out may be NULL to ask for the number only.
 * Errors: HE_ERR_ARG, HE_ERR_LEVEL, HE_ERR_KEY_MISSING, HE_ERR_OOM, HE_ERR_CUDA. */
int he_linear_transform_ksub(he_ctx *ctx, const he_ct *ct, int kind, int n, int n1, int n1_sub, he_ct **out);
int he_rot_steps_for_ksub(int n, int kind, int n1, int n1_sub, int slots, int32_t *out, int *count);

/* Encode (App. A) a real slot vector z[0..nslots) (rest zero) at scale
 * 2^log_delta and encrypt it (Enc, App. A) at `level` with the public key;
 * the encryption randomness is the Philox stream at object `enc_counter`. */
int he_encrypt_slots(he_ctx *ctx, const double *z, int nslots, int level, uint64_t enc_counter, he_ct **out);

/* Row-major matrix A (rows x cols) packed into slots [0, rows*cols), then
 * he_encrypt_slots. */
int he_encrypt_matrix(he_ctx *ctx, const double *A, int rows, int cols, int level, uint64_t enc_counter,
                      he_ct **out);

/* Dec + Decode (App. A): writes nslots real slot values (host). */
int he_decrypt_slots(he_ctx *ctx, const he_ct *ct, double *z, int nslots);
int he_decrypt_matrix(he_ctx *ctx, const he_ct *ct, double *out, int rows, int cols);

/* Level, scale and slot period (n^2 after replication, else the slot count). */
int he_ct_info(const he_ct *ct, int *level, double *scale, int *period);

/* Residues in coefficient form (see Conventions): 2*(level+1)*N words. */
int he_ct_export(const he_ct *ct, uint64_t *residues);

/* Builds a ciphertext from host residues in coefficient form (upload + NTT). */
int he_ct_import(he_ctx *ctx, const uint64_t *residues, int level, double scale, int period, he_ct **out);

int he_ct_free(he_ct *ct);

/* Slot rotation rho(ct; step) (App. A Rotation; hoisted key switch with the
 * Decompose-then-Permute order of Sec. 3.3). */
int he_rotate(he_ctx *ctx, const he_ct *ct, int step, he_ct **out);

/* Slot rotation for callers that cannot allocate device memory at the point
 * of the call (memory owned by another runtime's arena, latency-critical
 * threads, pipelines that must not fail on an allocation).  The paper has no
 * counterpart; it is the rotation of he_rotate with caller-owned buffers.
 *   in_dev, out_dev: device arrays of 2*(level+1)*N words, ciphertext residues
 *     in coefficient form as he_ct_export writes them; they may not overlap.
 *   Every temporary lives in one 32 MiB array that the library reserves in
 *     device memory when it is loaded (each device that loads the library
 *     holds it until the process exits); no call allocates.  The first call
 *     on a device looks up the array's device address.
 *   Stream: the work runs on the context's stream, which is not ordered
 *     after the caller's streams.  The caller must have finished every write
 *     to in_dev and out_dev (e.g. synchronised the stream that made them)
 *     before the call; the call waits for its own work before returning.
 *   Returns HE_ERR_ARG when the ring degree and level need more than 32 MiB
 *     of temporaries (at N = 2^16: above level 4 with two special primes,
 *     above level 3 with one), HE_ERR_KEY_MISSING without the rotation key.
 *   All calls share the array: calls whose work overlaps on the GPU race,
 *     and a call must not overlap any other call on the same context. */
int he_rotate_noalloc(he_ctx *ctx, const uint64_t *in_dev, int level, int step, uint64_t *out_dev);

/* Add (App. A Addition module): same level and scale. */
/* Hoisted rotations (Sec. 3.3.1): every ciphertext is Decomposed once and
 * that Decompose output serves all n_steps rotations; ciphertexts of one
 * level run as one batch, so each rotation key is read once per batch.
 * outs[i*n_steps + s] = Rot(cts[i], steps[s]) (caller frees).  Bit-identical
 * to he_rotate.  Errors: HE_ERR_ARG, HE_ERR_KEY_MISSING (no outputs made). */
int he_rotate_hoisted(he_ctx *ctx, const he_ct *const *cts, int n_cts, const int32_t *steps, int n_steps,
                      he_ct **outs);

int he_add(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct **out);

/* Mult (App. A): tensor product then relinearisation; scale multiplies. */
int he_mult(he_ctx *ctx, const he_ct *a, const he_ct *b, he_ct **out);

/* Rescale (App. A): round(c / q_l), level l -> l-1, scale / q_l. */
int he_rescale(he_ctx *ctx, const he_ct *a, he_ct **out);

/* Replicates an n x n matrix ciphertext to slot period n^2:
 * ct + Rot(ct, -n^2 2^j) for j = 0 .. log2(slots/n^2)-1. */
int he_replicate(he_ctx *ctx, const he_ct *ct, int n, he_ct **out);

/* Encrypted product of two n x n matrices (eq. 4, DMatrixMult without
 * decomposition): double-hoisted BSGS Z and T (Sec. 3.3, Table 1), hoisted
 * C^k / R^k, per-product relinearisation, one final rescale.  Consumes 3
 * levels; the output is replicated with period n^2. */
int he_hmatmul(he_ctx *ctx, const he_ct *A, const he_ct *B, int n, const he_mm_sched *sched, he_ct **out);

/* Batched products: jobs are grouped by (context, level, n, schedule); each
 * group runs as one pass in which every kernel covers all jobs of the group
 * and every key is read once per group.  outs[i] receives job i's product,
 * bit-identical to he_hmatmul on the same inputs. */
int he_hmatmul_batch(const he_mm_job *jobs, int n_jobs, he_ct **outs);

/* Transposition G (Sec. 3.4) of an n x n matrix ciphertext; consumes 1
 * level.  Every diagonal is multiplied by `prescale` (1.0 for a plain
 * transpose). */
int he_transpose(he_ctx *ctx, const he_ct *ct, int n, int n1, double prescale, he_ct **out);

/* One double-hoisted BSGS linear transform of eq. 3' on a matrix ciphertext
 * (Sec. 3.3.1, Table 1 "Optimized" rows): kind 0 = sigma (the Z transform
 * of eq. 5, diagonals k, -n < k < n), 1 = tau (T of eq. 6, diagonals n k,
 * 0 <= k < n), 2 = the transpose G (diagonals (n - 1) k); n1 baby steps.
 * With n_prime > 0 (kinds 0 and 1) the transform runs as its Diagonal
 * Convergence Decomposition (Sec. 4.2) with maximum diagonal n' (Z) or n' n
 * (T): floor((n-1)/n') + 1 factor transforms, one level each.
 * Replicates a zero-padded input to period n^2 first; consumes one level per
 * factor (the plaintext diagonals are encoded at scale q_l and rescaled away,
 * so the scale is kept).  Errors: HE_ERR_ARG, HE_ERR_LEVEL, HE_ERR_KEY_MISSING. */
#define HE_LT_SIGMA 0
#define HE_LT_TAU 1
#define HE_LT_TRANSPOSE 2
int he_linear_transform(he_ctx *ctx, const he_ct *ct, int kind, int n, int n1, int n_prime, he_ct **out);

/* State of the interactive modulus refresh (Sec. 7.2.3, App. C): the Philox
 * object of the next refresh is next_obj + 1; count counts refreshes. */
typedef struct he_refresh_state {
    uint32_t next_obj;
    int count;
} he_refresh_state;

/* Interactive modulus refresh (the client's step, Sec. 7.2.3): decrypt to the
 * integer message at q_0, centred lift, re-encrypt the same integers at the
 * top level with the next refresh object.  Needs the secret key. */
int he_refresh(he_ctx *ctx, const he_ct *ct, he_refresh_state *rs, he_ct **out);

/* Aggregate (Sec. 5.2): axis 0 sums the rows of an n x n block (rotations
 * n, 2n, ..., every row becomes the column sums); axis 1 sums within rows
 * (rotations 1, 2, ..., first-column mask (1 level), rotations -1, -2, ...,
 * every column becomes the row sums). */
int he_aggregate(he_ctx *ctx, const he_ct *ct, int axis, int n, he_ct **out);

/* HCovMtrx (Sec. 5.2): blocks[l*k + j] = encrypted X_j[l], the l-th n x n
 * row block of the j-th feature block of an s x (k n) dataset (zero-padded,
 * same level >= 6).  cov[a*k + b] receives block (a, b) of
 * X^T X / s - mu^T mu (or X^T X / s if centered): blocks a <= b by matrix
 * products summed over row blocks, a > b by transposition, 1/s folded into
 * the transposition of X, mu from Aggregate.  Consumes 5 levels. */
int he_covariance(he_ctx *ctx, he_ct *const *blocks, int n_row_blocks, int k, int n, int s, int centered,
                  const he_mm_sched *sched, he_ct **cov);

/* HCovMtrx over row blocks spread across devices (Sec. 5.2: the block
 * products of different row blocks are independent, so each device takes a
 * share of the rows).  he_covariance_partial runs on one device's row blocks
 * (blocks as in he_covariance, n_row_blocks of them; s is the TOTAL row
 * count of the dataset): upper[u] receives, for the pairs (a, b) with a <= b
 * in row-major order (u = 0 .. k(k+1)/2 - 1), the sum over these row blocks
 * of X_a[l]^T X_b[l] / s, and, unless centered, colsum[j] the sum over these
 * row blocks of X_j[l] (level of the blocks).  The parts of all devices are
 * added residue by residue modulo each prime (an all-reduce of the
 * exported residues; they are linear in the ciphertexts), imported, and
 * he_covariance_finish turns the sums into the k*k covariance blocks:
 * exactly the words he_covariance gives on all row blocks at once.
 * block_level is the level of the input blocks.  Errors as he_covariance. */
int he_covariance_partial(he_ctx *ctx, he_ct *const *blocks, int n_row_blocks, int k, int n, int s, int centered,
                          const he_mm_sched *sched, he_ct **upper, he_ct **colsum);
int he_covariance_finish(he_ctx *ctx, he_ct *const *upper, he_ct *const *colsum, int k, int n, int s, int centered,
                         const he_mm_sched *sched, int block_level, he_ct **cov);

/* Newton-iteration counts of Lazy Normalization (Sec. 6.1.2): the PowerMethod
 * simulation with contraction coefficient S, error bound e, precision bound
 * Bp, interval (0, B2] and the order-1 Taylor start at B2/2 + 1; counts[t]
 * for t < t_iters (host computation). */
int he_lazy_normalization_schedule(int t_iters, double S, double e, double Bp, double B2, int max_iters,
                                   int *counts);

/* HPowerMethod (Sec. 6.1): l_P normalised covariance transformations of the
 * replicated vector v0[0..k) (axis 0: rows equal, 1: columns equal), Newton
 * counts per iteration, then one more transformation for the eigenvalue.
 * Refreshes a ciphertext just before an operation that needs more levels than
 * it has.  Outputs: lambda (all slots), V[0..k) in *axis_out, VT[0..k) its
 * flip. */
int he_power_method(he_ctx *ctx, he_ct *const *cov, int k, int n, he_ct *const *v0, int axis, int l_P,
                    const int *newton_counts, double B2, he_refresh_state *rs, he_ct **lambda, he_ct **V,
                    he_ct **VT, int *axis_out);

/* HEigenShift (Sec. 6.2): cov[a*k + b] -= lambda v_a v_b^T in place. */
int he_eigen_shift(he_ctx *ctx, he_ct **cov, int k, int n, const he_ct *lambda, he_ct *const *V, int axis,
                   he_ct *const *VT, he_refresh_state *rs);

/* Privacy-Preserving PCA (Sec. 6.2): for m < l_E, HPowerMethod from the
 * start vector v0[m*k .. m*k+k) on the current covariance, then HEigenShift
 * (not after the last component).  cov is left unchanged.  Outputs
 * lambdas[m], V[m*k + j] and the axis of each eigenvector in axes[m]. */
int he_pca(he_ctx *ctx, he_ct *const *cov, int k, int n, int l_E, he_ct *const *v0, int axis, int l_P,
           const int *newton_counts, double B2, he_refresh_state *rs, he_ct **lambdas, he_ct **V, int *axes);

/* Negacyclic NTT over rows in device memory: the transform that puts
 * polynomials in the NTT domain where the full-RNS CKKS of App. A multiplies
 * them (Sec. 3.2); Decompose and ModDown spend most of their time in it
 * (Sec. 3.3.1).  rows_dev holds n_rows rows of N words; row r is reduced
 * modulo prime r mod (level+1+alpha) of Q_level P (q_0..q_level, then
 * p_0..p_{alpha-1}).  Forward: coefficients in [0, q) -> evaluations in
 * bit-reversed order, in [0, q).  Inverse (inverse != 0): the converse.
 * Runs on the context's stream and returns when it is done.
 * Errors: HE_ERR_ARG (null or negative sizes), HE_ERR_LEVEL (level outside
 * 0..L), HE_ERR_CUDA. */
int he_ntt(he_ctx *ctx, uint64_t *rows_dev, long long n_rows, int level, int inverse);

/* Decompose alone (Sec. 3.3, "Dp"; App. A KeySwitch): the digits of
 * polynomials over Q_level, each extended to Q_level P by the fast basis
 * conversion.  poly_dev: n_items polynomials of level+1 rows of N words in
 * the NTT domain (item stride (level+1) N).  digits_dev: n_items x dnum'
 * digits of level+1+alpha rows, NTT domain, laid out
 * [item][digit][row][N], rows q_0..q_level then p_0..p_{alpha-1}; dnum' =
 * ceil((level+1)/alpha).  Both device buffers are caller-owned, 16-byte
 * aligned and disjoint.  Runs on the context's stream and returns when it is
 * done.  Errors: HE_ERR_ARG (null, misaligned or negative sizes, more than
 * 2^20 items), HE_ERR_LEVEL, HE_ERR_OOM, HE_ERR_CUDA. */
int he_decompose(he_ctx *ctx, const uint64_t *poly_dev, long long n_items, int level, uint64_t *digits_dev);

/* ModDown alone (Sec. 3.3, "MD"; App. A KeySwitch): round(X / P) over
 * Q_level for elements X of Q_level P.  in_dev: n_items elements of
 * level+1+alpha rows (q_0..q_level, then p_0..p_{alpha-1}) of N words in
 * the NTT domain; out_dev: n_items polynomials of level+1 rows, NTT domain.
 * The overflow of the fast conversion is counted exactly, so the result is
 * round(X / P) for every coefficient.  Both device buffers are
 * caller-owned, 16-byte aligned and disjoint.  Runs on the context's stream
 * and returns when it is done.  Errors: as he_decompose. */
int he_moddown(he_ctx *ctx, const uint64_t *in_dev, long long n_items, int level, uint64_t *out_dev);

/* Counters of the key-switch phases since the last reset: MultSum, Decompose,
 * ModDown (Table 1 caption), and kernel launches.  Any pointer may be NULL. */
int he_counters(he_ctx *ctx, long long *ms, long long *dp, long long *md, long long *launches, int reset);

/* Kernel tracing.  While enabled, the library records a CUDA event pair on the
 * context's stream around every launch of the traced kernel classes
 *   0 MultSum (key-switch inner product), 1 forward NTT, 2 inverse NTT,
 *   3 ModUp basis conversion (Decompose), 4 ModDown basis conversion
 * and adds the launch's algorithmic bytes (words the operation must read and
 * write once).  he_trace_read synchronises the stream and returns, for one
 * class, the number of launches, their summed device time (ms) and bytes. */
int he_trace_enable(he_ctx *ctx, int on);

/* Integer roofline of the NTT: measured rate (butterflies per second) of the
 * lazy Shoup butterfly with register operands on the current device, `iters`
 * rounds of 16 butterflies per thread over 8 CTAs of 256 threads per SM. */
int he_bench_butterfly(int iters, double *bfly_per_s);
int he_trace_read(he_ctx *ctx, int cls, long long *count, double *total_ms, double *bytes, int reset);

/* Arithmetic of a traced class since its last reset by he_trace_read:
 * for class 0 (MultSum) the number of digit-key products accumulated (each
 * (digit word, key word) pair of every output word); 0 for the other
 * classes.  Read it before the he_trace_read call that resets the class.
 * Errors: HE_ERR_ARG. */
int he_trace_ops(he_ctx *ctx, int cls, double *ops);

/* Integer roofline of MultSum: measured rate (products per second) of the
 * 96-bit product accumulation of its 40-bit limbs (eight 32-bit
 * multiply-adds with carries per product) with register operands on the
 * current device, `iters` rounds of 16 products per thread over 8 CTAs of
 * 256 threads per SM.  Errors: HE_ERR_ARG, HE_ERR_CUDA. */
int he_bench_mac(int iters, double *products_per_s);

/* Captured batched products.  he_mm_plan_create runs the jobs once (grouped
 * as he_hmatmul_batch groups them: context, level, block size, schedule) and
 * records every launch of that batched step -- gathers, replication, the
 * hoisted product passes -- as one CUDA graph in which every group is a
 * branch of its own (forked from and joined to the plan's stream), so the
 * groups run concurrently at replay; he_mm_plan_run replays it and returns
 * fresh output ciphertexts, bit-identical to he_hmatmul_batch on the inputs'
 * contents at the time of the run.  Jobs may come from several contexts of
 * one device (different ring degrees, levels, block sizes).  The plan keeps
 * the device addresses of the jobs' input ciphertexts: those handles must
 * stay alive (contents may change between runs) until he_mm_plan_destroy.
 * Each branch's temporaries live in memory of its own that the plan owns
 * (the working set of the whole batch, held until destroy).  A run waits for
 * work queued on the jobs' contexts before it starts; runs of one plan, and
 * anything else on those contexts, must not overlap a run.  The paper runs
 * its products as parallel CPU threads (Sec. 4.1.2); the concurrent branches
 * are this library's form of that parallel step.
 * Errors as he_hmatmul_batch, plus HE_ERR_KEY_MISSING at creation. */
typedef struct he_mm_plan he_mm_plan;
int he_mm_plan_create(const he_mm_job *jobs, int n_jobs, he_mm_plan **out);
int he_mm_plan_run(he_mm_plan *plan, he_ct **outs);
/* Kernel launches one run replays, and the plan's device bytes.  Either
 * pointer may be NULL. */
int he_mm_plan_info(const he_mm_plan *plan, long long *launches, double *scratch_bytes);
int he_mm_plan_destroy(he_mm_plan *plan);

/* ------------------------------------------------------------------ serving
 * A service over contexts whose keys stay resident (Sec. 2: the keys are on
 * the server before the computation; the paper's throughput is bounded by
 * device memory, Sec. 7).  One worker thread per context drains that
 * context's queue in ticks: every job queued when a tick starts joins it,
 * the block products of all its matrix-product and covariance jobs run as
 * batched passes (at most max_batch products per pass), then each job's own
 * remaining steps run.  Jobs that arrive during a tick join the next one.
 *
 * While a server runs, its contexts belong to it: the caller may still call
 * he_ct_export, he_decrypt_*, he_ct_info and he_ct_free on ciphertexts of
 * those contexts (from any thread), and nothing else on them.  Input
 * ciphertexts stay caller-owned and must stay alive and unchanged until the
 * job completes; results pass to the caller through he_server_result.
 *
 * Admission: every job is charged an estimate of the device bytes it holds
 * from admission until its results are taken (its batched temporaries, the
 * intermediates of its circuit and its outputs; resident keys are not
 * charged).  A job whose charge alone exceeds hbm_budget_bytes is rejected
 * with HE_ERR_ADMISSION.  A job that fits the budget but not what is left of
 * it waits (HE_JOB_WAITING) and is admitted, in submission order, as earlier
 * jobs give their charges back (completion without outputs, or
 * he_server_result) -- unless reject_when_full is set, which rejects it. */
typedef struct he_server he_server;

typedef struct he_server_cfg {
    double hbm_budget_bytes; /* bound on the summed charges of admitted jobs */
    int max_batch;           /* products per batched pass (>= 1) */
    int reject_when_full;    /* 0: a job that does not fit now waits; 1: it is rejected */
} he_server_cfg;

#define HE_JOB_MATMUL 1     /* in: A, B; out: A*B (one ciphertext) */
#define HE_JOB_COVARIANCE 2 /* in: n_row_blocks*k blocks; out: k*k covariance blocks (he_covariance) */
#define HE_JOB_XTX_BLOCK 3  /* in: the k blocks of one row block; adds X_l^T X_l / s into accumulator acc_id */
#define HE_JOB_XTX_FINAL 4  /* out: the k*k blocks of the accumulated X^T X / s; the accumulator is consumed */
#define HE_JOB_PCA 5        /* in: k*k covariance blocks, then l_E*k start vectors; out: l_E eigenvalue
                             * ciphertexts, then l_E*k eigenvector blocks (he_pca) */

typedef struct he_job {
    int kind;                  /* HE_JOB_* */
    he_ctx *ctx;               /* the context of a job without inputs (X^T X final); else NULL or the inputs' */
    he_ct *const *in;          /* inputs, all of one context served by this server */
    int n_in;
    int n;                     /* block dimension (power of two, n*n <= slots) */
    he_mm_sched sched;         /* baby steps of Z/T (and of G: n1_z) */
    int n_row_blocks, k, s;    /* covariance / X^T X: row blocks, feature blocks, total rows s */
    int centered;              /* covariance: the data is already centred */
    uint64_t acc_id;           /* X^T X accumulator; one accumulation stream per id and context */
    int l_E, l_P, axis;        /* PCA: components, PowerMethod iterations, start-vector axis */
    const int *newton_counts;  /* PCA: l_P Newton counts (copied at submission) */
    double B2;                 /* PCA: Lazy Normalization bound */
    uint32_t refresh_obj;      /* PCA: first refresh object counter */
} he_job;

#define HE_JOB_QUEUED 0
#define HE_JOB_RUNNING 1
#define HE_JOB_DONE 2
#define HE_JOB_FAILED 3
#define HE_JOB_WAITING 4  /* accepted, waiting for device memory to be admitted */

typedef struct he_serving_stats {
    long long submitted, admitted, rejected, completed, failed;
    long long waited;                       /* jobs that waited for admission */
    double p50_ms, p99_ms, mean_ms, max_ms; /* submit -> done latency of completed jobs (nearest rank) */
    double jobs_per_s;                      /* completed jobs / (last completion - first submission) */
    long long ticks, products, max_products_per_tick;
    double charged_bytes;                   /* summed charges of admitted jobs not yet collected */
    double key_bytes;                       /* resident rotation and relinearisation keys */
} he_serving_stats;

/* Starts one worker per context.  Errors: HE_ERR_ARG (null, empty, repeated
 * context, max_batch < 1, budget <= 0). */
int he_server_create(const he_server_cfg *cfg, he_ctx *const *ctxs, int n_ctx, he_server **out);

/* Validates and queues a job; *job_id identifies it.  Errors, with no job
 * queued: HE_ERR_ARG (bad kind, operands, sizes or a context not served),
 * HE_ERR_LEVEL (too few levels), HE_ERR_KEY_MISSING (a rotation key the job
 * needs is absent), HE_ERR_ADMISSION (over the budget). */
int he_server_submit(he_server *srv, const he_job *job, uint64_t *job_id);

/* Status (HE_JOB_*) of a job; *error = its HE_ERR_* code if it failed;
 * *latency_ms = submit -> done once done.  Any output pointer may be NULL. */
int he_server_poll(he_server *srv, uint64_t job_id, int *status, int *error, double *latency_ms);

/* Waits up to timeout_s seconds (host wait) for a job to finish; returns
 * HE_ERR_TIMEOUT if it has not. */
int he_server_wait(he_server *srv, uint64_t job_id, double timeout_s, int *status);

/* Moves a finished job's outputs to the caller (max_outs must hold them all)
 * and forgets the job, releasing its charge.  aux (may be NULL) receives, for
 * PCA, the l_E eigenvector axes followed by the number of refreshes.  A
 * failed job returns its error code (and is forgotten). */
int he_server_result(he_server *srv, uint64_t job_id, he_ct **outs, int max_outs, int *n_outs, int *aux,
                     int max_aux, int *n_aux);

/* Counters and latency percentiles over jobs of one kind (0: all kinds). */
int he_server_stats(he_server *srv, int kind, he_serving_stats *out);

/* Finishes every queued job, stops the workers, frees uncollected outputs
 * and accumulators. */
int he_server_destroy(he_server *srv);

#ifdef __cplusplus
}
#endif
#endif
