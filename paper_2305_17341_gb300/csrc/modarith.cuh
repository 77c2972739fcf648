// modarith.cuh -- 64-bit modular arithmetic for residues of primes q < 2^60.
//
// Every RNS limb of the paper's full-RNS CKKS (App. A) is a polynomial with
// coefficients mod a prime q_i = 1 mod 2N.  All arithmetic stays exact.
//   * Shoup multiplication by a precomputed constant w (w' = floor(w 2^64 / q)):
//     one 64x64 high product and two low products, result in [0, 2q).
//   * Montgomery reduction (R = 2^64) of a 128-bit value x < q R, used for
//     products of two variable operands and for lazily accumulated sums of
//     products (sum of up to 15 products of residues < q stays below q R).
#pragma once
#include <cstdint>

typedef unsigned long long u64;
typedef long long i64;
typedef unsigned int u32;

struct ModQ {
    u64 q;       // the prime
    u64 qinv;    // -q^-1 mod 2^64 (Montgomery)
    u64 r2;      // 2^128 mod q
    u64 twoq;
    u64 wone;    // floor(2^64 / q): the Shoup companion of 1
};

__device__ __forceinline__ u64 mulhi64(u64 a, u64 b) { return __umul64hi(a, b); }

// a * w mod q, lazily in [0, 2q), for any a < 2^64.
__device__ __forceinline__ u64 shoup_lazy(u64 a, u64 w, u64 wp, u64 q) {
    u64 h = mulhi64(a, wp);
    return a * w - h * q;
}

// High word of the 128-bit product a b from three of its four 32 x 32
// partial products: dropping al bl and the low halves of ah bl and al bh
// loses less than 3 units of 2^64, so the result is the exact high word
// minus 0, 1 or 2.
__device__ __forceinline__ u64 mulhi64_trunc(u64 a, u64 b) {
    const u32 al = (u32)a, ah = (u32)(a >> 32), bl = (u32)b, bh = (u32)(b >> 32);
    return (u64)ah * bh + __umulhi(ah, bl) + __umulhi(al, bh);
}

// a * w mod q in [0, 4q) for any a < 2^64 and q < 2^62: Shoup's product with
// the truncated quotient (exact quotient minus at most 2).
__device__ __forceinline__ u64 shoup_lazy4(u64 a, u64 w, u64 wp, u64 q) {
    return a * w - mulhi64_trunc(a, wp) * q;
}

__device__ __forceinline__ u64 shoup(u64 a, u64 w, u64 wp, u64 q) {
    u64 r = shoup_lazy(a, w, wp, q);
    return r >= q ? r - q : r;
}

__device__ __forceinline__ u64 reduce2q(u64 a, u64 q) { return a >= q ? a - q : a; }

// a mod q for any 64-bit a: Shoup's product by 1 lands in [0, 2q), then one
// conditional subtraction.
__device__ __forceinline__ u64 reduce_any(u64 a, u64 q, u64 wone) {
    u64 r = a - mulhi64(a, wone) * q;
    return r >= q ? r - q : r;
}

__device__ __forceinline__ u64 reduce4q(u64 a, u64 q) {
    a = a >= 2 * q ? a - 2 * q : a;
    return a >= q ? a - q : a;
}

__device__ __forceinline__ u64 addmod(u64 a, u64 b, u64 q) {
    u64 s = a + b;
    return s >= q ? s - q : s;
}

__device__ __forceinline__ u64 submod(u64 a, u64 b, u64 q) { return a >= b ? a - b : a + q - b; }

// 128-bit accumulator
struct U128 {
    u64 lo, hi;
};

__device__ __forceinline__ void mac128(U128 &acc, u64 a, u64 b) {
    u64 lo = a * b;
    u64 hi = mulhi64(a, b);
    u64 nlo = acc.lo + lo;
    acc.hi += hi + (nlo < lo ? 1ull : 0ull);
    acc.lo = nlo;
}

// acc += a b for residues a, b < q < 2^60, keeping acc below q 2^64 (the
// Montgomery reduction's input bound) however many terms are summed: each
// product is below q 2^60, so after it the high word is below q + q/16 + 1,
// and subtracting q 2^64 (a multiple of q) once restores the bound.
__device__ __forceinline__ void mac128_q(U128 &acc, u64 a, u64 b, u64 q) {
    mac128(acc, a, b);
    if (acc.hi >= q) acc.hi -= q;
}

// 96-bit accumulation (w2 w1 w0) of products of residues below 2^42: each
// product is below 2^84, so a sum of up to 2^12 of them stays below 2^96.
// (w2 w1 w0) += a b from the four 32 x 32 partial products with the carry
// chain of the 32-bit multiply-add (a1 b1 < 2^20 has no high word).
__device__ __forceinline__ void mac96(u32 &w0, u32 &w1, u32 &w2, u64 a, u64 b) {
    const u32 a0 = (u32)a, a1 = (u32)(a >> 32), b0 = (u32)b, b1 = (u32)(b >> 32);
    asm("mad.lo.cc.u32 %0, %3, %5, %0;\n\t"
        "madc.hi.cc.u32 %1, %3, %5, %1;\n\t"
        "addc.u32 %2, %2, 0;\n\t"
        "mad.lo.cc.u32 %1, %3, %6, %1;\n\t"
        "madc.hi.u32 %2, %3, %6, %2;\n\t"
        "mad.lo.cc.u32 %1, %4, %5, %1;\n\t"
        "madc.hi.u32 %2, %4, %5, %2;\n\t"
        "mad.lo.u32 %2, %4, %6, %2;"
        : "+r"(w0), "+r"(w1), "+r"(w2)
        : "r"(a0), "r"(a1), "r"(b0), "r"(b1));
}

// Montgomery REDC with the prime and -q^-1 mod 2^64 given directly.
__device__ __forceinline__ u64 redc_q(u64 lo, u64 hi, u64 q, u64 qinv) {
    const u64 t = lo * qinv;
    const u64 r = hi + mulhi64(t, q) + (lo != 0 ? 1ull : 0ull);
    return r >= q ? r - q : r;
}

// Montgomery REDC: x * 2^-64 mod q for x < q 2^64, result in [0, q).
__device__ __forceinline__ u64 redc(u64 lo, u64 hi, const ModQ &m) {
    u64 t = lo * m.qinv;
    u64 mh = mulhi64(t, m.q);
    u64 r = hi + mh + (lo != 0 ? 1ull : 0ull);
    return r >= m.q ? r - m.q : r;
}

// a * b mod q for two residues (double REDC with R^2).
__device__ __forceinline__ u64 mulmod(u64 a, u64 b, const ModQ &m) {
    u64 t = redc(a * b, mulhi64(a, b), m);           // a b R^-1
    return redc(t * m.r2, mulhi64(t, m.r2), m);      // a b
}

// a * bM mod q where bM = b R mod q is in Montgomery form.
__device__ __forceinline__ u64 mulmont(u64 a, u64 bM, const ModQ &m) {
    return redc(a * bM, mulhi64(a, bM), m);
}

// (hi 2^64 + lo) mod q for any 128-bit value.
__device__ __forceinline__ u64 mod128(u64 hi, u64 lo, const ModQ &m) {
    u64 h = hi % m.q, l = lo % m.q;
    u64 t = redc(l, h, m);                           // (h R + l) R^-1
    return redc(t * m.r2, mulhi64(t, m.r2), m);      // t R
}

// signed integer -> residue
__device__ __forceinline__ u64 from_signed(i64 x, u64 q) {
    if (x >= 0) return ((u64)x) % q;
    u64 r = ((u64)(-x)) % q;
    return r ? q - r : 0;
}
