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

// Shoup's lazy product from 32-bit halves (the default; LOLA_SHOUP_C keeps
// the compiler's 64-bit arithmetic for comparison).  With x = x1 2^32 + x0
// and w' = p1 2^32 + p0:
//   floor(x w' / 2^64) = x1 p1 + a_hi + b_hi  exactly, where
//   a = x0 p1 + hi32(x0 p0)  and  b = x1 p0 + a_lo  (both fit 64 bits),
// because the remaining terms b_lo 2^32 + lo32(x0 p0) stay below 2^64.
// The result x w - qh q lies in [0, 2q), so it equals its value mod 2^64:
//   lo64(x w + qh (2^64 - q)), whose high word needs only the low 32 bits of
// the four cross products.  One mul.hi, five mad.wide, four mad.lo and a
// 64-bit add: 11 multiply-class instructions against the 10 wide products
// plus carry chains of the generic 64-bit code.
// nq = 2^64 - q (computed by the caller, so loops hoist it).
__device__ __forceinline__ uint64_t shoup_mul_lazy_ptx(uint64_t x, uint64_t w, uint64_t wp, uint64_t nq) {
  uint64_t r;
  asm("{\n\t"
      ".reg .u32 x0, x1, p0, p1, w0, w1, n0, n1, t, al, ah, bl, bh, h0, h1, rl, rh;\n\t"
      ".reg .u64 a, b, c, lo;\n\t"
      "mov.b64 {x0, x1}, %1;\n\t"
      "mov.b64 {w0, w1}, %2;\n\t"
      "mov.b64 {p0, p1}, %3;\n\t"
      "mov.b64 {n0, n1}, %4;\n\t"
      "mul.hi.u32 t, x0, p0;\n\t"
      "cvt.u64.u32 c, t;\n\t"
      "mad.wide.u32 a, x0, p1, c;\n\t"
      "mov.b64 {al, ah}, a;\n\t"
      "cvt.u64.u32 c, al;\n\t"
      "mad.wide.u32 b, x1, p0, c;\n\t"
      "mov.b64 {bl, bh}, b;\n\t"
      "cvt.u64.u32 c, bh;\n\t"
      "mad.wide.u32 c, x1, p1, c;\n\t"
      "mov.b64 {h0, h1}, c;\n\t"
      "add.cc.u32 h0, h0, ah;\n\t"
      "addc.u32 h1, h1, 0;\n\t"
      "mul.wide.u32 lo, x0, w0;\n\t"
      "mad.wide.u32 lo, h0, n0, lo;\n\t"
      "mov.b64 {rl, rh}, lo;\n\t"
      "mad.lo.u32 rh, x0, w1, rh;\n\t"
      "mad.lo.u32 rh, x1, w0, rh;\n\t"
      "mad.lo.u32 rh, h0, n1, rh;\n\t"
      "mad.lo.u32 rh, h1, n0, rh;\n\t"
      "mov.b64 %0, {rl, rh};\n\t"
      "}"
      : "=l"(r)
      : "l"(x), "l"(w), "l"(wp), "l"(nq));
  return r;
}

// x * w mod q, result in [0, 2q); valid for every 64-bit x when q < 2^63.
__device__ __forceinline__ uint64_t shoup_mul_lazy(uint64_t x, uint64_t w, uint64_t wp, uint64_t q) {
#ifdef LOLA_SHOUP_C
  uint64_t qh = mulhi64(x, wp);
  return x * w - qh * q;
#else
  return shoup_mul_lazy_ptx(x, w, wp, 0ull - q);
#endif
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

// REDC of a 128-bit sum T < q 2^64: T 2^-64 mod q in [0, q).
__device__ __forceinline__ uint64_t redc128(unsigned __int128 T, uint64_t q, uint64_t qinv) {
  const uint64_t lo = (uint64_t)T, hi = (uint64_t)(T >> 64);
  const uint64_t m = lo * qinv;
  return csub(hi + mulhi64(m, q) + (lo != 0), q);
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
