// Modular arithmetic on 64-bit words for primes q < 2^62 (device side).
//
// Blackwell has no single-instruction 64x64 integer multiply: the compiler
// builds each 64-bit product from 32-bit IMADs.  The routines below are the
// ones the hot path needs and nothing more:
//
//  * shoup_mul(x, w, w')      x*w mod q in [0, 2q) for any 64-bit x, with
//                             w' = floor(w * 2^64 / q) precomputed (twiddles,
//                             scalars, CRT constants).  Shoup, "NTL" 2001;
//                             Harvey, "Faster arithmetic for number-theoretic
//                             transforms", JSC 2014.
//  * mont_mul(a, b)           a*b*2^-64 mod q in [0, q) for a, b < q
//                             (Montgomery, Math. Comp. 1985), used when one
//                             operand is stored pre-scaled by 2^64 (keys,
//                             encoded plaintexts).
//  * reduce64(x)              x mod q for any 64-bit x via floor(2^64/q).
//
// All values stored in memory are canonical representatives in [0, q).
#pragma once
#include <stdint.h>

namespace lola {

struct Mod {
  uint64_t q;       // the prime
  uint64_t qinv;    // -q^{-1} mod 2^64 (Montgomery)
  uint64_t r2;      // 2^128 mod q (to enter Montgomery form)
  uint64_t floor64; // floor(2^64 / q)
};

__device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) { return __umul64hi(a, b); }

// x * w mod q, result in [0, 2q); valid for every 64-bit x when q < 2^63.
__device__ __forceinline__ uint64_t shoup_mul_lazy(uint64_t x, uint64_t w, uint64_t wp, uint64_t q) {
  uint64_t qh = mulhi64(x, wp);
  return x * w - qh * q;
}

__device__ __forceinline__ uint64_t csub(uint64_t x, uint64_t q) { return x >= q ? x - q : x; }

__device__ __forceinline__ uint64_t shoup_mul(uint64_t x, uint64_t w, uint64_t wp, uint64_t q) {
  return csub(shoup_mul_lazy(x, w, wp, q), q);
}

__device__ __forceinline__ uint64_t add_mod(uint64_t a, uint64_t b, uint64_t q) { return csub(a + b, q); }

__device__ __forceinline__ uint64_t sub_mod(uint64_t a, uint64_t b, uint64_t q) {
  return a >= b ? a - b : a + q - b;
}

__device__ __forceinline__ uint64_t neg_mod(uint64_t a, uint64_t q) { return a ? q - a : 0; }

// Montgomery product a*b*2^-64 mod q for a*b < q*2^64; result in [0, q).
__device__ __forceinline__ uint64_t mont_mul(uint64_t a, uint64_t b, uint64_t q, uint64_t qinv) {
  uint64_t lo = a * b;
  uint64_t hi = mulhi64(a, b);
  uint64_t m = lo * qinv;
  uint64_t t = hi + mulhi64(m, q) + (lo != 0);
  return csub(t, q);
}

// x mod q for any 64-bit x, given f = floor(2^64 / q).
__device__ __forceinline__ uint64_t reduce64(uint64_t x, uint64_t q, uint64_t f) {
  uint64_t r = x - mulhi64(x, f) * q;
  return csub(r, q);
}

// Signed 64-bit value (|v| < 2^62) to its residue mod q.
__device__ __forceinline__ uint64_t from_signed(int64_t v, uint64_t q, uint64_t f) {
  if (v >= 0) return reduce64((uint64_t)v, q, f);
  uint64_t r = reduce64((uint64_t)(-v), q, f);
  return r ? q - r : 0;
}

}  // namespace lola
