// Negacyclic NTT over Z_q[x]/(x^n+1), one limb-polynomial per CTA.
//
// Sec. 3.1 of the paper relies on Z_q[x]/(x^n+1) being isomorphic to Z_q^n
// when q = 1 mod 2n; the transform below is that isomorphism, used to turn
// every ring product into a pointwise one.
//
// Forward: Cooley-Tukey butterflies with the 2n-th root psi merged into the
// twiddles (tw[2^s + i] = psi^brev(2^s + i)), natural-order input, output
// position k holds a(psi^(2 brev(k) + 1)).  Inverse: the Gentleman-Sande
// mirror image with psi^-1, scaled at the end by a caller-given constant
// (n^-1, possibly times an extra factor).  Lazy reduction (Harvey) between
// stages: forward values stay below 4q + 2^32 (the "a" operand of each
// butterfly is brought below 2q + 2^32 by comparing only its high 32 bits
// with those of 2q), inverse values below 2q; q < 2^61 keeps every
// intermediate below 2^64.  What the loader supplies and what the storer
// receives is canonical [0, q).
//
// Layout: the CTA holds the whole limb (n words) in shared memory.  Each
// thread owns E = 2^LOGE words per pass and runs up to LOGE radix-2 stages
// in registers; passes exchange through shared memory with an XOR swizzle
// that keeps every 64-bit access of a half-warp on distinct banks.  The first
// forward pass reads global memory directly (coalesced: the thread index is
// the low index bits there) and the last inverse pass writes it directly.
#pragma once
#include <stdint.h>

#include "modarith.cuh"

namespace lola {

template <int LOGE>
__device__ __forceinline__ int swz(int idx) {
  return idx ^ ((idx >> LOGE) & 15);
}

// global index of local element k for thread tid in the bit window [hb .. lb]
__device__ __forceinline__ int win_index(int tid, int k, int hb, int lb) {
  return ((tid >> lb) << (hb + 1)) | (k << lb) | (tid & ((1 << lb) - 1));
}

template <int LOGN, int LOGE>
struct NttGeom {
  static_assert(LOGE >= 1 && LOGE <= LOGN, "bad NTT geometry");
  static constexpr int N = 1 << LOGN;
  static constexpr int E = 1 << LOGE;
  static constexpr int T = N >> LOGE;
  static constexpr int NPASS = (LOGN + LOGE - 1) / LOGE;
  // forward pass p covers distance bits [fhb(p) .. flb(p)], top bits first
  static constexpr int fhb(int p) { return (LOGN - 1 - p * LOGE) > (LOGE - 1) ? (LOGN - 1 - p * LOGE) : (LOGE - 1); }
  static constexpr int flb(int p) { return fhb(p) - LOGE + 1; }
  // lowest distance bit already processed before pass p (forward)
  static constexpr int fdone(int p) { return p == 0 ? LOGN : flb(p - 1); }
  // inverse pass p covers bits [ilb(p) + LOGE - 1 .. ilb(p)], low bits first
  static constexpr int ilb(int p) { return (p * LOGE + LOGE - 1 <= LOGN - 1) ? p * LOGE : LOGN - LOGE; }
  static constexpr int idone(int p) { return p == 0 ? 0 : ilb(p - 1) + LOGE; }
};

// Twiddle tables hold (w, floor(w 2^64 / q)) pairs so one 16-byte load
// fetches both; `tw` points at the pair array of one prime.
__device__ __forceinline__ ulonglong2 tw_pair(const uint64_t* __restrict__ tw, int ti) {
  return __ldg(reinterpret_cast<const ulonglong2*>(tw) + ti);
}

template <int LOGN, int LOGE, int P>
__device__ __forceinline__ void fwd_stages(uint64_t (&x)[1 << LOGE], const uint64_t* __restrict__ tw, uint64_t q,
                                           int tid) {
  using G = NttGeom<LOGN, LOGE>;
  constexpr int hb = G::fhb(P), lb = G::flb(P), top = G::fdone(P) - 1;
  const uint64_t q2 = 2 * q;
  const uint32_t q2hi = (uint32_t)(q2 >> 32);
#pragma unroll
  for (int bp = top; bp >= lb; --bp) {
    const int s = LOGN - 1 - bp;
    const int lbit = bp - lb;
    // twiddle index (1 << s) + (j >> (bp + 1)) splits into a per-stage,
    // per-thread base and the compile-time k >> (lbit + 1)
    const ulonglong2* twb = reinterpret_cast<const ulonglong2*>(tw) + (1 << s) + ((tid >> lb) << (hb - bp));
#pragma unroll
    for (int k = 0; k < G::E; ++k) {
      if (k & (1 << lbit)) continue;
      const ulonglong2 wq = __ldg(twb + (k >> (lbit + 1)));
      const uint64_t w = wq.x, wp = wq.y;
      uint64_t a = x[k];
      if ((uint32_t)(a >> 32) > q2hi) a -= q2;
      const uint64_t t = shoup_mul_lazy(x[k | (1 << lbit)], w, wp, q);
      x[k] = a + t;
      x[k | (1 << lbit)] = a - t + q2;
    }
  }
}

template <int LOGN, int LOGE, int P, class Loader, class Storer>
__device__ __forceinline__ void fwd_pass(uint64_t* sm, uint64_t (&x)[1 << LOGE], const uint64_t* __restrict__ tw,
                                         uint64_t q, uint64_t qf, const Loader& ld, const Storer& st, int tid) {
  using G = NttGeom<LOGN, LOGE>;
  constexpr int hb = G::fhb(P), lb = G::flb(P);
  if constexpr (P == 0) {
#pragma unroll
    for (int k = 0; k < G::E; ++k) x[k] = ld(win_index(tid, k, hb, lb));
  } else {
    __syncthreads();
#pragma unroll
    for (int k = 0; k < G::E; ++k) x[k] = sm[swz<LOGE>(win_index(tid, k, hb, lb))];
  }
  fwd_stages<LOGN, LOGE, P>(x, tw, q, tid);
  __syncthreads();
  if constexpr (P + 1 < G::NPASS) {
#pragma unroll
    for (int k = 0; k < G::E; ++k) sm[swz<LOGE>(win_index(tid, k, hb, lb))] = x[k];
    fwd_pass<LOGN, LOGE, P + 1>(sm, x, tw, q, qf, ld, st, tid);
  } else {
#pragma unroll
    for (int k = 0; k < G::E; ++k) sm[swz<LOGE>(win_index(tid, k, hb, lb))] = reduce64(x[k], q, qf);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < G::E; ++k) {
      const int i = tid + k * G::T;
      st(i, sm[swz<LOGE>(i)]);
    }
  }
}

// Forward transform.  ld(i) returns input coefficient i (canonical);
// st(i, v) receives output position i (canonical), called once per i.
// tw: the prime's (w, w') twiddle pairs; qf = floor(2^64 / q).
// Every thread of the CTA must call this (it synchronises).
template <int LOGN, int LOGE, class Loader, class Storer>
__device__ __forceinline__ void ntt_forward(uint64_t* sm, const uint64_t* __restrict__ tw, uint64_t q, uint64_t qf,
                                            const Loader& ld, const Storer& st) {
  uint64_t x[1 << LOGE];
  fwd_pass<LOGN, LOGE, 0>(sm, x, tw, q, qf, ld, st, (int)threadIdx.x);
}

template <int LOGN, int LOGE, int P>
__device__ __forceinline__ void inv_stages(uint64_t (&x)[1 << LOGE], const uint64_t* __restrict__ tw, uint64_t q,
                                           int tid) {
  using G = NttGeom<LOGN, LOGE>;
  constexpr int lb = G::ilb(P), hb = lb + LOGE - 1, first = G::idone(P);
  const uint64_t q2 = 2 * q;
#pragma unroll
  for (int bp = first; bp <= hb; ++bp) {
    const int s = LOGN - 1 - bp;
    const int lbit = bp - lb;
    const ulonglong2* twb = reinterpret_cast<const ulonglong2*>(tw) + (1 << s) + ((tid >> lb) << (hb - bp));
#pragma unroll
    for (int k = 0; k < G::E; ++k) {
      if (k & (1 << lbit)) continue;
      const ulonglong2 wq = __ldg(twb + (k >> (lbit + 1)));
      const uint64_t w = wq.x, wp = wq.y;
      const uint64_t a = x[k], b = x[k | (1 << lbit)];
      uint64_t u = a + b;
      u = u >= q2 ? u - q2 : u;
      x[k] = u;
      x[k | (1 << lbit)] = shoup_mul_lazy(a - b + q2, w, wp, q);
    }
  }
}

template <int LOGN, int LOGE, int P, class Storer>
__device__ __forceinline__ void inv_pass(uint64_t* sm, uint64_t (&x)[1 << LOGE], const uint64_t* __restrict__ tw,
                                         uint64_t q, uint64_t c, uint64_t cs, const Storer& st, int tid) {
  using G = NttGeom<LOGN, LOGE>;
  constexpr int lb = G::ilb(P), hb = lb + LOGE - 1;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < G::E; ++k) x[k] = sm[swz<LOGE>(win_index(tid, k, hb, lb))];
  inv_stages<LOGN, LOGE, P>(x, tw, q, tid);
  if constexpr (P + 1 < G::NPASS) {
    __syncthreads();
#pragma unroll
    for (int k = 0; k < G::E; ++k) sm[swz<LOGE>(win_index(tid, k, hb, lb))] = x[k];
    inv_pass<LOGN, LOGE, P + 1>(sm, x, tw, q, c, cs, st, tid);
  } else {
#pragma unroll
    for (int k = 0; k < G::E; ++k) st(win_index(tid, k, hb, lb), shoup_mul(x[k], c, cs, q));
  }
}

// Inverse transform, output scaled by c (n^-1, possibly times an extra
// factor), cs = floor(c 2^64 / q).  ld(i) is read once per i.
template <int LOGN, int LOGE, class Loader, class Storer>
__device__ __forceinline__ void ntt_inverse(uint64_t* sm, const uint64_t* __restrict__ tw, uint64_t q, uint64_t c,
                                            uint64_t cs, const Loader& ld, const Storer& st) {
  using G = NttGeom<LOGN, LOGE>;
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < G::E; ++k) {
    const int i = tid + k * G::T;
    sm[swz<LOGE>(i)] = ld(i);
  }
  uint64_t x[1 << LOGE];
  inv_pass<LOGN, LOGE, 0>(sm, x, tw, q, c, cs, st, tid);
}

// Inverse transform of data the caller has already placed in shared memory
// (element i at sm[swz<LOGE>(i)], canonical).  The first pass synchronises
// before reading.
template <int LOGN, int LOGE, class Storer>
__device__ __forceinline__ void ntt_inverse_smem(uint64_t* sm, const uint64_t* __restrict__ tw, uint64_t q,
                                                 uint64_t c, uint64_t cs, const Storer& st) {
  uint64_t x[1 << LOGE];
  inv_pass<LOGN, LOGE, 0>(sm, x, tw, q, c, cs, st, (int)threadIdx.x);
}

}  // namespace lola
