/*
 * oracle.c -- plain, slow CPU primitives of the RNS-CKKS oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / --impl reference legs may use it.  It shares no code with the
 * CUDA path (paper_2305_17341_gb300/csrc).
 *
 * Every routine is the textbook definition written out with unsigned __int128
 * products and '%' reductions.  The only "fast" step is the number-theoretic
 * transform used as a library primitive for negacyclic polynomial products;
 * it is pinned against schoolbook convolution in the tests.
 *
 * Paper: "Improved Privacy-Preserving PCA Using Optimized Homomorphic Matrix
 * Multiplication" (arXiv 2305.17341).  Citations give the section / appendix.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC oracle.c -o liboracle.so -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;
typedef uint64_t u64;
typedef int64_t i64;
typedef uint32_t u32;

/* ---------------------------------------------------------------- modular */

static inline u64 mulmod(u64 a, u64 b, u64 q) { return (u64)(((u128)a * b) % q); }
static inline u64 addmod(u64 a, u64 b, u64 q) { u64 s = a + b; return s >= q ? s - q : s; }
static inline u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

static u64 powmod(u64 a, u64 e, u64 q) {
    u64 r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

/* inverse of a modulo a prime q (Fermat) */
static u64 invmod(u64 a, u64 q) { return powmod(a, q - 2, q); }

u64 or_powmod(u64 a, u64 e, u64 q) { return powmod(a, e, q); }
u64 or_invmod(u64 a, u64 q) { return invmod(a, q); }

/* Deterministic Miller-Rabin for n < 2^64 with the first twelve prime bases. */
int or_is_prime(u64 n) {
    static const u64 bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return 0;
    for (int i = 0; i < 12; i++) {
        if (n == bases[i]) return 1;
        if (n % bases[i] == 0) return 0;
    }
    u64 d = n - 1;
    int r = 0;
    while ((d & 1) == 0) { d >>= 1; r++; }
    for (int i = 0; i < 12; i++) {
        u64 x = powmod(bases[i], d, n);
        if (x == 1 || x == n - 1) continue;
        int composite = 1;
        for (int k = 1; k < r; k++) {
            x = mulmod(x, x, n);
            if (x == n - 1) { composite = 0; break; }
        }
        if (composite) return 0;
    }
    return 1;
}

static int already_used(const u64 *used, int nused, u64 c) {
    for (int i = 0; i < nused; i++)
        if (used[i] == c) return 1;
    return 0;
}

/*
 * Prime chain (App. A, Setparams: q_i, p_i = 1 mod 2N).  The paper fixes only
 * the congruence and the bit sizes; the reading used by both sides:
 *   q_0 and then p_0..p_{alpha-1}: the largest primes = 1 mod 2N below
 *     2^bits, taken in descending order;
 *   q_1..q_L: primes = 1 mod 2N around 2^bits, alternating: first the
 *     smallest one above 2^bits, then the largest one below, then the second
 *     above, the second below, ...  (keeps prod q_i / 2^(40 L) near 1).
 *     A prime already taken by the descending search is an error.
 * Returns 0 on success, -1 if a search runs out of candidates.
 */
int or_gen_primes(int logN, int nq, const int *qbits, int np, const int *pbits,
                  u64 *out_q, u64 *out_p) {
    u64 M = (u64)2 << logN;
    u64 used[256];
    int nused = 0;
    if (nq + np > 256) return -1;

    /* descending search for q_0 then the special primes */
    for (int t = 0; t < 1 + np; t++) {
        int b = (t == 0) ? qbits[0] : pbits[t - 1];
        u64 top = (u64)1 << b;
        u64 c = ((top - 1) / M) * M + 1; /* largest candidate = 1 mod M below 2^b */
        if (c >= top) c -= M;
        while (c > M && (!or_is_prime(c) || already_used(used, nused, c))) c -= M;
        if (c <= M) return -1;
        used[nused++] = c;
        if (t == 0) out_q[0] = c; else out_p[t - 1] = c;
    }
    /* alternating search around 2^b for q_1..q_L (cursor per distinct size) */
    for (int i = 1; i < nq; i++) {
        int b = qbits[i];
        u64 centre = (u64)1 << b;
        /* count how many earlier q's had the same size to know the parity */
        int k = 0;
        for (int j = 1; j < i; j++)
            if (qbits[j] == b) k++;
        int up = (k % 2 == 0);
        /* find the (k/2)-th prime in the chosen direction that is unused */
        int want = k / 2, seen = 0;
        u64 c;
        if (up) {
            c = ((centre + M - 1) / M) * M + 1; /* smallest = 1 mod M above 2^b */
            if (c < centre) c += M;
            for (;;) {
                if (or_is_prime(c)) {
                    if (seen == want) break;
                    seen++;
                }
                c += M;
            }
        } else {
            c = ((centre - 1) / M) * M + 1;
            if (c >= centre) c -= M;
            for (;;) {
                if (c <= M) return -1;
                if (or_is_prime(c)) {
                    if (seen == want) break;
                    seen++;
                }
                c -= M;
            }
        }
        if (already_used(used, nused, c)) return -1; /* sizes must not collide */
        used[nused++] = c;
        out_q[i] = c;
    }
    return 0;
}

/* ------------------------------------------------------------ Philox4x32-10
 * Counter-based generator of Salmon, Moraes, Dror, Shaw (SC'11), written out
 * from its published definition: 10 rounds; each round multiplies words 0 and
 * 2 by the constants 0xD2511F53 and 0xCD9E8D57 (full 64-bit product split in
 * hi/lo) and mixes with the round key; the key is bumped by the Weyl
 * constants 0x9E3779B9, 0xBB67AE85 between rounds.
 */
void or_philox4x32_10(const u32 ctr_in[4], const u32 key_in[2], u32 out[4]) {
    u32 c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    u32 k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        u64 p0 = (u64)0xD2511F53u * c0;
        u64 p1 = (u64)0xCD9E8D57u * c2;
        u32 hi0 = (u32)(p0 >> 32), lo0 = (u32)p0;
        u32 hi1 = (u32)(p1 >> 32), lo1 = (u32)p1;
        u32 n0 = hi1 ^ c1 ^ k0;
        u32 n1 = lo1;
        u32 n2 = hi0 ^ c3 ^ k1;
        u32 n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_block(u64 seed, u32 i, u32 j, u32 obj, u32 tag, u32 w[4]) {
    u32 ctr[4] = {i, j, obj, tag};
    u32 key[2] = {(u32)seed, (u32)(seed >> 32)};
    or_philox4x32_10(ctr, key, w);
}

/* Uniform residue mod q for coefficient i of limb j: the 128-bit block
 * (w3 w2 w1 w0) read as hi64 = w2 | w3<<32, lo64 = w0 | w1<<32, reduced mod q. */
void or_sample_uniform(u64 seed, u32 obj, u32 tag, u32 limb, u64 q, int N, u64 *out) {
    for (int i = 0; i < N; i++) {
        u32 w[4];
        philox_block(seed, (u32)i, limb, obj, tag, w);
        u64 lo = (u64)w[0] | ((u64)w[1] << 32);
        u64 hi = (u64)w[2] | ((u64)w[3] << 32);
        u128 v = ((u128)hi << 64) | lo;
        out[i] = (u64)(v % q);
    }
}

/* Ternary secret / ephemeral (App. A, chi_s): w0 mod 3 -> {0, +1, -1}. */
void or_sample_ternary(u64 seed, u32 obj, u32 tag, int N, i64 *out) {
    for (int i = 0; i < N; i++) {
        u32 w[4];
        philox_block(seed, (u32)i, 0, obj, tag, w);
        u32 r = w[0] % 3u;
        out[i] = (r == 0) ? 0 : (r == 1 ? 1 : -1);
    }
}

/* Cumulative table of the discrete Gaussian truncated to |x| <= 19 (App. A,
 * chi_e with standard deviation sigma).  T[k] = floor(2^63 * P(|x| <= k)),
 * T[19] = 2^63.  Evaluated in one fixed order: rho[v] = exp(-v^2 / (2 sigma^2))
 * for v = 0..19, total = rho[0] + 2 rho[1] + ... + 2 rho[19] added in
 * increasing v, and the cumulative sums in increasing k (the CUDA side runs
 * the same sequence of IEEE operations). */
void or_gauss_table(double sigma, u64 *T) {
    double denom = (2.0 * sigma) * sigma;
    double rho[20];
    for (int v = 0; v < 20; v++) rho[v] = exp(-((double)(v * v)) / denom);
    double total = rho[0];
    for (int v = 1; v < 20; v++) total += 2.0 * rho[v];
    double cum = rho[0];
    for (int k = 0; k < 19; k++) {
        if (k > 0) cum += 2.0 * rho[k];
        T[k] = (u64)floor((cum / total) * 9223372036854775808.0);
    }
    T[19] = (u64)1 << 63;
}

/* Discrete Gaussian by CDT inversion: r = 63-bit uniform (w1:w0 >> 1);
 * |x| = smallest k with r < T[k]; sign from bit 0 of w2. */
void or_sample_gauss(u64 seed, u32 obj, u32 tag, double sigma, int N, i64 *out) {
    u64 T[20];
    or_gauss_table(sigma, T);
    for (int i = 0; i < N; i++) {
        u32 w[4];
        philox_block(seed, (u32)i, 0, obj, tag, w);
        u64 r = (((u64)w[1] << 32) | (u64)w[0]) >> 1;
        int k = 0;
        while (r >= T[k]) k++;
        i64 x = k;
        if (x != 0 && (w[2] & 1u)) x = -x;
        out[i] = x;
    }
}

/* --------------------------------------------------------- polynomial ring
 * R_q = Z_q[X]/(X^N + 1) (Sec. 3.2).  Products are negacyclic convolutions.
 */

/* Schoolbook negacyclic product, the definition itself (O(N^2)). */
void or_polymul_schoolbook(u64 q, int N, const u64 *a, const u64 *b, u64 *out) {
    u64 *acc = (u64 *)calloc((size_t)N, sizeof(u64));
    for (int i = 0; i < N; i++) {
        if (a[i] == 0) continue;
        for (int j = 0; j < N; j++) {
            u64 p = mulmod(a[i], b[j], q);
            int k = i + j;
            if (k < N) acc[k] = addmod(acc[k], p, q);
            else acc[k - N] = submod(acc[k - N], p, q);
        }
    }
    memcpy(out, acc, sizeof(u64) * (size_t)N);
    free(acc);
}

/* A primitive 2N-th root of unity mod q: smallest g^((q-1)/2N) over g = 2,3,...
 * whose N-th power is q-1. */
static u64 find_psi(u64 q, int N) {
    u64 M = 2 * (u64)N;
    for (u64 g = 2;; g++) {
        u64 psi = powmod(g, (q - 1) / M, q);
        if (powmod(psi, (u64)N, q) == q - 1) return psi;
    }
}

/* Cyclic length-N transform A_k = sum_i a_i w^(ik), textbook iterative
 * radix-2: bit-reversal permutation then log2(N) butterfly passes. */
static void ntt_cyclic(u64 *a, int N, u64 w, u64 q) {
    for (int i = 1, j = 0; i < N; i++) {
        int bit = N >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) { u64 t = a[i]; a[i] = a[j]; a[j] = t; }
    }
    for (int len = 2; len <= N; len <<= 1) {
        u64 wl = powmod(w, (u64)(N / len), q);
        int half = len >> 1;
        u64 *pw = (u64 *)malloc(sizeof(u64) * (size_t)half);
        pw[0] = 1;
        for (int k = 1; k < half; k++) pw[k] = mulmod(pw[k - 1], wl, q);
        for (int s = 0; s < N; s += len) {
            for (int k = 0; k < half; k++) {
                u64 u = a[s + k];
                u64 v = mulmod(a[s + k + half], pw[k], q);
                a[s + k] = addmod(u, v, q);
                a[s + k + half] = submod(u, v, q);
            }
        }
        free(pw);
    }
}

/* Negacyclic forward transform: a_i <- a_i psi^i, then cyclic NTT with psi^2. */
static void nega_fwd(u64 *a, int N, u64 psi, u64 q) {
    u64 p = 1;
    for (int i = 0; i < N; i++) { a[i] = mulmod(a[i], p, q); p = mulmod(p, psi, q); }
    ntt_cyclic(a, N, mulmod(psi, psi, q), q);
}

/* Inverse: cyclic NTT with psi^-2, times N^-1 psi^-i. */
static void nega_inv(u64 *a, int N, u64 psi, u64 q) {
    u64 ipsi = invmod(psi, q);
    ntt_cyclic(a, N, mulmod(ipsi, ipsi, q), q);
    u64 ninv = invmod((u64)N, q);
    u64 p = ninv;
    for (int i = 0; i < N; i++) { a[i] = mulmod(a[i], p, q); p = mulmod(p, ipsi, q); }
}

/* out = a * b in R_q (coefficient form in and out). */
void or_polymul(u64 q, int N, const u64 *a, const u64 *b, u64 *out) {
    u64 psi = find_psi(q, N);
    u64 *ta = (u64 *)malloc(sizeof(u64) * (size_t)N);
    u64 *tb = (u64 *)malloc(sizeof(u64) * (size_t)N);
    memcpy(ta, a, sizeof(u64) * (size_t)N);
    memcpy(tb, b, sizeof(u64) * (size_t)N);
    nega_fwd(ta, N, psi, q);
    nega_fwd(tb, N, psi, q);
    for (int i = 0; i < N; i++) ta[i] = mulmod(ta[i], tb[i], q);
    nega_inv(ta, N, psi, q);
    memcpy(out, ta, sizeof(u64) * (size_t)N);
    free(ta);
    free(tb);
}

/*
 * Sum of products over several limbs:
 *   out[l] = sum_t a[t][l] * b[t][l]  in R_{q_l},  l < nlimbs, t < nterms.
 * a, b: [nterms][nlimbs][N]; out: [nlimbs][N]; all coefficient form.
 * Limbs are independent (RNS isomorphism, App. A) and run in parallel.
 */
void or_polymul_sum(int N, int nlimbs, const u64 *qs, int nterms, const u64 *a, const u64 *b,
                    u64 *out) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int l = 0; l < nlimbs; l++) {
        u64 q = qs[l];
        u64 psi = find_psi(q, N);
        u64 *acc = (u64 *)calloc((size_t)N, sizeof(u64));
        u64 *ta = (u64 *)malloc(sizeof(u64) * (size_t)N);
        u64 *tb = (u64 *)malloc(sizeof(u64) * (size_t)N);
        for (int t = 0; t < nterms; t++) {
            const u64 *pa = a + ((size_t)t * nlimbs + l) * N;
            const u64 *pb = b + ((size_t)t * nlimbs + l) * N;
            memcpy(ta, pa, sizeof(u64) * (size_t)N);
            memcpy(tb, pb, sizeof(u64) * (size_t)N);
            nega_fwd(ta, N, psi, q);
            nega_fwd(tb, N, psi, q);
            for (int i = 0; i < N; i++) acc[i] = addmod(acc[i], mulmod(ta[i], tb[i], q), q);
        }
        nega_inv(acc, N, psi, q);
        memcpy(out + (size_t)l * N, acc, sizeof(u64) * (size_t)N);
        free(acc);
        free(ta);
        free(tb);
    }
}

/* out[l][i] = a[l][i] * c[l] mod q_l (a scalar per limb). */
void or_mulconst_limbs(int N, int nlimbs, const u64 *qs, const u64 *a, const u64 *c, u64 *out) {
#pragma omp parallel for
    for (int l = 0; l < nlimbs; l++)
        for (int i = 0; i < N; i++)
            out[(size_t)l * N + i] = mulmod(a[(size_t)l * N + i], c[l] % qs[l], qs[l]);
}

/* ------------------------------------------------------ basis conversion
 * Fast (approximate) CRT basis extension used by Decompose and ModDown
 * (Sec. 3.3 hoisting; App. A KeySwitch):
 *   y_i   = [x_i * (Qs/q_i)^-1]_{q_i} in [0, q_i)
 *   out_r = sum_i y_i * (Qs/q_i mod r)  mod r
 * src: [ns][N] over primes sq; out: [nd][N] over primes dq.
 */
void or_bconv(int N, int ns, const u64 *sq, const u64 *src, int nd, const u64 *dq, u64 *out) {
    u64 *qhat_inv = (u64 *)malloc(sizeof(u64) * (size_t)ns);
    u64 *qhat_mod = (u64 *)malloc(sizeof(u64) * (size_t)ns * (size_t)nd);
    for (int i = 0; i < ns; i++) {
        u64 prod = 1;
        for (int k = 0; k < ns; k++)
            if (k != i) prod = mulmod(prod, sq[k] % sq[i], sq[i]);
        qhat_inv[i] = invmod(prod, sq[i]);
        for (int r = 0; r < nd; r++) {
            u64 pr = 1;
            for (int k = 0; k < ns; k++)
                if (k != i) pr = mulmod(pr, sq[k] % dq[r], dq[r]);
            qhat_mod[(size_t)i * nd + r] = pr;
        }
    }
#pragma omp parallel for
    for (int x = 0; x < N; x++) {
        u64 y[64];
        for (int i = 0; i < ns; i++) y[i] = mulmod(src[(size_t)i * N + x], qhat_inv[i], sq[i]);
        for (int r = 0; r < nd; r++) {
            u64 acc = 0;
            for (int i = 0; i < ns; i++)
                acc = addmod(acc, mulmod(y[i] % dq[r], qhat_mod[(size_t)i * nd + r], dq[r]), dq[r]);
            out[(size_t)r * N + x] = acc;
        }
    }
    free(qhat_inv);
    free(qhat_mod);
}

/*
 * Unsigned integers of BN_LIMBS little-endian 32-bit limbs: enough for a
 * product of up to 8 primes below 2^62 times 8 (the ModDown overflow sums).
 */
#define BN_LIMBS 17
static void bn_from_u64(u32 *a, u64 v) {
    memset(a, 0, BN_LIMBS * sizeof(u32));
    a[0] = (u32)v;
    a[1] = (u32)(v >> 32);
}
static void bn_mul_u64(u32 *a, u64 m) {    /* a <- a m */
    u128 carry = 0;
    for (int i = 0; i < BN_LIMBS; i++) {
        u128 t = (u128)a[i] * m + carry;
        a[i] = (u32)t;
        carry = t >> 32;
    }
}
static void bn_add(u32 *a, const u32 *b) {   /* a <- a + b */
    u64 carry = 0;
    for (int i = 0; i < BN_LIMBS; i++) {
        u64 t = (u64)a[i] + b[i] + carry;
        a[i] = (u32)t;
        carry = t >> 32;
    }
}
static int bn_less(const u32 *a, const u32 *b) {
    for (int i = BN_LIMBS - 1; i >= 0; i--)
        if (a[i] != b[i]) return a[i] < b[i];
    return 0;
}

/*
 * ModDown with rounding (App. A KeySwitch: round(P^-1 <a, swk>) mod Q_l).
 * Input: an element X of Q_l P given by residues uQ [nq][N] and uP [np][N].
 * With h = (P-1)/2 and Y = X + h, the result is floor(Y / P) = round(X / P):
 *   v_j   = (uP_j + h) mod p_j
 *   y_j   = [v_j (P/p_j)^-1]_{p_j}
 *   e     = floor(sum_j y_j (P/p_j) / P)    (exact, big integers)
 *   Y mod P = sum_j y_j (P/p_j) - e P       (reduced mod each q_i)
 *   out_i = ((uQ_i + h) - (Y mod P)) P^-1 mod q_i.
 * e counts how often the sum of the y_j (P/p_j), each below P, passes P.
 */
void or_moddown_round(int N, int nq, const u64 *qs, const u64 *uQ, int np, const u64 *ps, const u64 *uP, u64 *out) {
    u64 hp[8], phat_inv[8], hq[64], Pq[64], Pinv[64], phat_q[8][64];
    for (int j = 0; j < np; j++) {
        u64 p = ps[j];
        u64 Pm = 1, ph = 1;
        for (int k = 0; k < np; k++) {
            Pm = mulmod(Pm, ps[k] % p, p);
            if (k != j) ph = mulmod(ph, ps[k] % p, p);
        }
        hp[j] = mulmod(submod(Pm, 1 % p, p), invmod(2, p), p); /* (P-1)/2 mod p */
        phat_inv[j] = invmod(ph, p);
        for (int i = 0; i < nq; i++) {
            u64 q = qs[i], v = 1;
            for (int k = 0; k < np; k++)
                if (k != j) v = mulmod(v, ps[k] % q, q);
            phat_q[j][i] = v;
        }
    }
    for (int i = 0; i < nq; i++) {
        u64 q = qs[i], Pm = 1;
        for (int k = 0; k < np; k++) Pm = mulmod(Pm, ps[k] % q, q);
        Pq[i] = Pm;
        Pinv[i] = invmod(Pm, q);
        hq[i] = mulmod(submod(Pm, 1, q), invmod(2, q), q);
    }
    /* P and P/p_j as big integers */
    u32 Pbig[BN_LIMBS], phat[8][BN_LIMBS];
    bn_from_u64(Pbig, 1);
    for (int k = 0; k < np; k++) bn_mul_u64(Pbig, ps[k]);
    for (int j = 0; j < np; j++) {
        bn_from_u64(phat[j], 1);
        for (int k = 0; k < np; k++)
            if (k != j) bn_mul_u64(phat[j], ps[k]);
    }
#pragma omp parallel for
    for (int x = 0; x < N; x++) {
        u64 y[8];
        for (int j = 0; j < np; j++) {
            u64 v = addmod(uP[(size_t)j * N + x], hp[j], ps[j]);
            y[j] = mulmod(v, phat_inv[j], ps[j]);
        }
        u32 S[BN_LIMBS], term[BN_LIMBS], bound[BN_LIMBS];
        bn_from_u64(S, 0);
        for (int j = 0; j < np; j++) {
            memcpy(term, phat[j], sizeof term);
            bn_mul_u64(term, y[j]);
            bn_add(S, term);
        }
        u64 e = 0;   /* the largest e with e P <= S */
        memcpy(bound, Pbig, sizeof bound);
        while (!bn_less(S, bound)) {
            e++;
            bn_add(bound, Pbig);
        }
        for (int i = 0; i < nq; i++) {
            u64 q = qs[i];
            u64 conv = 0;
            for (int j = 0; j < np; j++) conv = addmod(conv, mulmod(y[j] % q, phat_q[j][i], q), q);
            conv = submod(conv, mulmod(e % q, Pq[i], q), q);
            u64 t = submod(addmod(uQ[(size_t)i * N + x], hq[i], q), conv, q);
            out[(size_t)i * N + x] = mulmod(t, Pinv[i], q);
        }
    }
}

/* -------------------------------------------------------- encode / decode
 * Canonical embedding (App. A Encode/Decode): slot j holds m(zeta^(5^j)),
 * zeta = exp(i pi / N), S = N/2 slots.  The inverse map, written as
 *   u_i = (1/S) sum_j z_j zeta^(-i 5^j),  m_i = Re u_i,  m_(i+S) = Im u_i,
 * is evaluated in this fixed order:
 *   1. x[t] = z[j] with t = (5^j mod 2N - 1)/4   (5^j = 1 + 4t runs over all
 *      residues = 1 mod 4 exactly once),
 *   2. bit-reversal permutation of x over log2(S) bits,
 *   3. radix-2 decimation-in-time passes len = 2, 4, ..., S with twiddle
 *      W_len^k = conj(zeta^(4 k S/len)) (a length-S DFT with exponent -1),
 *   4. y_i = x_i * conj(zeta^i), then m = round(y * scale / S).
 * Complex products are (ar*br - ai*bi, ar*bi + ai*br); no fused multiply-add.
 * zeta^e = (cos a_e, sin a_e) with a_e = (M_PI * (double)e) / (double)N.
 */
static void zeta_table(int N, double *zr, double *zi) {
    for (int e = 0; e < 2 * N; e++) {
        double a = (M_PI * (double)e) / (double)N;
        zr[e] = cos(a);
        zi[e] = sin(a);
    }
}

static void bitrev_perm(double *xr, double *xi, int S) {
    for (int i = 1, j = 0; i < S; i++) {
        int bit = S >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double t = xr[i]; xr[i] = xr[j]; xr[j] = t;
            t = xi[i]; xi[i] = xi[j]; xi[j] = t;
        }
    }
}

/* length-S radix-2 DIT pass structure; sign = -1 (encode) or +1 (decode). */
static void dft_passes(double *xr, double *xi, int S, const double *zr, const double *zi, int sign) {
    for (int len = 2; len <= S; len <<= 1) {
        int half = len >> 1;
        int step = 4 * (S / len); /* zeta exponent of the pass root */
        for (int s = 0; s < S; s += len) {
            for (int k = 0; k < half; k++) {
                int e = k * step;
                double wr = zr[e];
                double wi = sign < 0 ? -zi[e] : zi[e];
                double br = xr[s + k + half], bi = xi[s + k + half];
                double tr = br * wr - bi * wi;
                double ti = br * wi + bi * wr;
                double ar = xr[s + k], ai = xi[s + k];
                xr[s + k] = ar + tr;
                xi[s + k] = ai + ti;
                xr[s + k + half] = ar - tr;
                xi[s + k + half] = ai - ti;
            }
        }
    }
}

void or_encode(int N, const double *z_re, const double *z_im, double scale, i64 *m) {
    int S = N / 2;
    u64 M = 2 * (u64)N;
    double *zr = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    double *zi = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    double *xr = (double *)malloc(sizeof(double) * (size_t)S);
    double *xi = (double *)malloc(sizeof(double) * (size_t)S);
    zeta_table(N, zr, zi);
    u64 g = 1;
    for (int j = 0; j < S; j++) {
        u64 t = (g - 1) / 4;
        xr[t] = z_re[j];
        xi[t] = z_im[j];
        g = (g * 5) % M;
    }
    bitrev_perm(xr, xi, S);
    dft_passes(xr, xi, S, zr, zi, -1);
    double f = scale / (double)S;
    for (int i = 0; i < S; i++) {
        double wr = zr[i], wi = -zi[i];
        double yr = xr[i] * wr - xi[i] * wi;
        double yi = xr[i] * wi + xi[i] * wr;
        m[i] = (i64)round(yr * f);
        m[i + S] = (i64)round(yi * f);
    }
    free(zr); free(zi); free(xr); free(xi);
}

/* Decode (App. A): z_j = sum_i u_i zeta^(i 5^j) with u_i = (m_i + I m_(i+S)) / scale.
 * coef: real coefficients m_i (already centred and converted to double). */
void or_decode(int N, const double *coef, double scale, double *z_re, double *z_im) {
    int S = N / 2;
    u64 M = 2 * (u64)N;
    double *zr = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    double *zi = (double *)malloc(sizeof(double) * 2 * (size_t)N);
    double *xr = (double *)malloc(sizeof(double) * (size_t)S);
    double *xi = (double *)malloc(sizeof(double) * (size_t)S);
    zeta_table(N, zr, zi);
    for (int i = 0; i < S; i++) {
        double ur = coef[i] / scale, ui = coef[i + S] / scale;
        xr[i] = ur * zr[i] - ui * zi[i];
        xi[i] = ur * zi[i] + ui * zr[i];
    }
    bitrev_perm(xr, xi, S);
    dft_passes(xr, xi, S, zr, zi, +1);
    u64 g = 1;
    for (int j = 0; j < S; j++) {
        u64 t = (g - 1) / 4;
        z_re[j] = xr[t];
        z_im[j] = xi[t];
        g = (g * 5) % M;
    }
    free(zr); free(zi); free(xr); free(xi);
}

/* Direct O(N*S) evaluation of the encoding sum, the definition itself,
 * used only to pin or_encode on small N (before rounding). */
void or_encode_direct(int N, const double *z_re, const double *z_im, double scale, double *m_real) {
    int S = N / 2;
    u64 M = 2 * (u64)N;
    for (int i = 0; i < N; i++) {
        long double acc = 0.0L;
        u64 g = 1;
        for (int j = 0; j < S; j++) {
            /* Re( z_j * zeta^(-i g) ) */
            u64 e = (M - ((u64)i * g) % M) % M;
            long double a = (long double)M_PI * (long double)e / (long double)N;
            acc += (long double)z_re[j] * cosl(a) - (long double)z_im[j] * sinl(a);
            g = (g * 5) % M;
        }
        m_real[i] = (double)(acc * (long double)scale / (long double)S);
    }
}
