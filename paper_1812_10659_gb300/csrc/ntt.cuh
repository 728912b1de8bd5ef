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
// stages.  Forward: on even stages the "a" operand of each butterfly is
// brought below 4q + 2^32 by comparing only its high 32 bits with those of
// 4q; odd stages skip that step, so values stay below 6q + 2^32 after an
// even stage and below 8q + 2^32 after an odd one (twiddle products are in
// [0, 2q)).  Inverse values stay below 2q.  q < 2^61 - 2^30 keeps every
// intermediate below 2^64.  The forward loader may supply any value below
// 8q + 2^32; what the storer receives is canonical [0, q).
//
// Layout: the CTA holds the whole limb (n words) in shared memory.  Each
// thread owns E = 2^LOGE words per pass and runs up to LOGE radix-2 stages
// in registers; passes exchange through shared memory with an XOR swizzle
// that keeps every 64-bit access of a half-warp on distinct banks.  The first
// forward pass reads global memory directly (coalesced: the thread index is
// the low index bits there) and the last inverse pass writes it directly.
#pragma once
#include <stdint.h>

#include <type_traits>

#include <cooperative_groups.h>

#include "modarith.cuh"

namespace lola {

template <int LOGE>
__device__ __forceinline__ int swz(int idx) {
  return idx ^ ((idx >> LOGE) & 15);
}

// A forward storer is either a callable st(i, v) or an object with
// fetch(i) -> f and operator()(i, v, f): the final phase then issues the
// fetches of a group of outputs before their stores (the fetch is a global
// load the store may alias, so the compiler would not hoist it itself).
template <class S, class = void>
struct has_fetch : std::false_type {};
template <class S>
struct has_fetch<S, std::void_t<decltype(std::declval<const S&>().fetch(0))>> : std::true_type {};

template <int LOGE, int E, int T, class Storer>
__device__ __forceinline__ void store_outputs(const uint64_t* sm, const Storer& st, int tid, int base) {
  if constexpr (has_fetch<Storer>::value) {
    constexpr int GRP = 8 < E ? 8 : E;
#pragma unroll
    for (int k0 = 0; k0 < E; k0 += GRP) {
      uint64_t f[GRP];
#pragma unroll
      for (int j = 0; j < GRP; ++j) f[j] = st.fetch(base + tid + (k0 + j) * T);
#pragma unroll
      for (int j = 0; j < GRP; ++j) {
        const int i = tid + (k0 + j) * T;
        st(base + i, sm[swz<LOGE>(i)], f[j]);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < E; ++k) {
      const int i = tid + k * T;
      st(base + i, sm[swz<LOGE>(i)]);
    }
  }
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
  const uint64_t q2 = 2 * q, q4 = 4 * q;
  const uint32_t q4hi = (uint32_t)(q4 >> 32);
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
      if ((s & 1) == 0 && (uint32_t)(a >> 32) > q4hi) a -= q4;
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
    store_outputs<LOGE, G::E, G::T>(sm, st, tid, 0);
  }
}

// Forward transform.  ld(i) returns input coefficient i (below 8q + 2^32);
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


// ---------------------------------------------------------------------------
// Cluster variant: one transform split over a cluster of C = 2^LOGC CTAs.
// CTA h of the cluster owns the contiguous chunk [h n/C, (h+1) n/C) in its
// own shared memory.  Forward: the first pass (the stages whose distance
// crosses chunks, LOGC <= LOGE) runs on the full index space with the
// cluster's threads acting as the single-CTA thread block, and each thread
// writes its results into the owning CTA's shared memory (distributed shared
// memory); after a cluster barrier the remaining passes are local.  Inverse:
// mirror image, the last pass reads the owners' shared memory.  Twiddle
// indices are those of the single-CTA transform.
namespace ncl {

template <int LOGN, int LOGE, int LOGC>
struct Geom {
  static_assert(LOGC >= 1 && LOGC <= LOGE, "cluster larger than one pass window");
  using G = NttGeom<LOGN, LOGE>;
  static constexpr int N = 1 << LOGN, E = 1 << LOGE, C = 1 << LOGC;
  static constexpr int LOGNL = LOGN - LOGC;          // chunk bits
  static constexpr int NC = 1 << LOGNL;
  static constexpr int T = N >> (LOGE + LOGC);       // threads per CTA
};

// forward stages of pass P on x; j_global = (h << LOGNL) | j_local, with the
// window index computed from `tid` over `idx_bits` bits (LOGN for the first
// pass with the virtual thread, LOGNL for local passes with h the chunk)
template <int LOGN, int LOGE, int P>
__device__ __forceinline__ void fwd_stages_c(uint64_t (&x)[1 << LOGE], const uint64_t* __restrict__ tw, uint64_t q,
                                             int tid, int h, int lognl) {
  using G = NttGeom<LOGN, LOGE>;
  constexpr int hb = G::fhb(P), lb = G::flb(P), top = G::fdone(P) - 1;
  const uint64_t q2 = 2 * q, q4 = 4 * q;
  const uint32_t q4hi = (uint32_t)(q4 >> 32);
#pragma unroll
  for (int bp = top; bp >= lb; --bp) {
    const int s = LOGN - 1 - bp;
    const int lbit = bp - lb;
    const ulonglong2* twb = reinterpret_cast<const ulonglong2*>(tw) + (1 << s) + (h << (lognl - bp - 1)) +
                            ((tid >> lb) << (hb - bp));
#pragma unroll
    for (int k = 0; k < G::E; ++k) {
      if (k & (1 << lbit)) continue;
      const ulonglong2 wq = __ldg(twb + (k >> (lbit + 1)));
      uint64_t a = x[k];
      if ((s & 1) == 0 && (uint32_t)(a >> 32) > q4hi) a -= q4;
      const uint64_t t = shoup_mul_lazy(x[k | (1 << lbit)], wq.x, wq.y, q);
      x[k] = a + t;
      x[k | (1 << lbit)] = a - t + q2;
    }
  }
}

template <int LOGN, int LOGE, int P>
__device__ __forceinline__ void inv_stages_c(uint64_t (&x)[1 << LOGE], const uint64_t* __restrict__ tw, uint64_t q,
                                             int tid, int h, int lognl) {
  using G = NttGeom<LOGN, LOGE>;
  constexpr int lb = G::ilb(P), hb = lb + LOGE - 1, first = G::idone(P);
  const uint64_t q2 = 2 * q;
#pragma unroll
  for (int bp = first; bp <= hb; ++bp) {
    const int s = LOGN - 1 - bp;
    const int lbit = bp - lb;
    const ulonglong2* twb = reinterpret_cast<const ulonglong2*>(tw) + (1 << s) + (h << (lognl - bp - 1)) +
                            ((tid >> lb) << (hb - bp));
#pragma unroll
    for (int k = 0; k < G::E; ++k) {
      if (k & (1 << lbit)) continue;
      const ulonglong2 wq = __ldg(twb + (k >> (lbit + 1)));
      const uint64_t a = x[k], b = x[k | (1 << lbit)];
      uint64_t u = a + b;
      u = u >= q2 ? u - q2 : u;
      x[k] = u;
      x[k | (1 << lbit)] = shoup_mul_lazy(a - b + q2, wq.x, wq.y, q);
    }
  }
}

template <int LOGN, int LOGE, int LOGC, int P, class Storer>
__device__ __forceinline__ void fwd_local_pass(uint64_t* sm, uint64_t (&x)[1 << LOGE], const uint64_t* __restrict__ tw,
                                               uint64_t q, uint64_t qf, const Storer& st, int tid, int h) {
  using GC = Geom<LOGN, LOGE, LOGC>;
  using G = typename GC::G;
  constexpr int hb = G::fhb(P), lb = G::flb(P);
  __syncthreads();
#pragma unroll
  for (int k = 0; k < G::E; ++k) x[k] = sm[swz<LOGE>(win_index(tid, k, hb, lb))];
  fwd_stages_c<LOGN, LOGE, P>(x, tw, q, tid, h, GC::LOGNL);
  __syncthreads();
  if constexpr (P + 1 < G::NPASS) {
#pragma unroll
    for (int k = 0; k < G::E; ++k) sm[swz<LOGE>(win_index(tid, k, hb, lb))] = x[k];
    fwd_local_pass<LOGN, LOGE, LOGC, P + 1>(sm, x, tw, q, qf, st, tid, h);
  } else {
#pragma unroll
    for (int k = 0; k < G::E; ++k) sm[swz<LOGE>(win_index(tid, k, hb, lb))] = reduce64(x[k], q, qf);
    __syncthreads();
    store_outputs<LOGE, G::E, GC::T>(sm, st, tid, h << GC::LOGNL);
  }
}

// Forward transform over the cluster.  ld(i), i in [0, n): any coefficient;
// st(i, v) is called for the i of this CTA's chunk.  All threads of all CTAs
// of the cluster must call it, before any other use of the shared memory by
// a peer (the first pass writes into the peers' shared memory).
template <int LOGN, int LOGE, int LOGC, class Loader, class Storer>
__device__ __forceinline__ void ntt_forward_cluster(uint64_t* sm, const uint64_t* __restrict__ tw, uint64_t q,
                                                    uint64_t qf, const Loader& ld, const Storer& st) {
  using GC = Geom<LOGN, LOGE, LOGC>;
  using G = typename GC::G;
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int h = (int)cl.block_rank();
  const int tid = threadIdx.x;
  const int tv = h * GC::T + tid;                    // thread of the single-CTA geometry
  constexpr int hb = G::fhb(0), lb = G::flb(0);
  // every CTA of the cluster must have started before its shared memory is
  // written; the arrive/wait pair overlaps that barrier with the first pass
  cl.barrier_arrive();
  uint64_t x[1 << LOGE];
#pragma unroll
  for (int k = 0; k < G::E; ++k) x[k] = ld(win_index(tv, k, hb, lb));
  fwd_stages_c<LOGN, LOGE, 0>(x, tw, q, tv, 0, LOGN);
  cl.barrier_wait();
  // the destination chunk of element (k << lb) | tv is k >> (LOGE - LOGC)
#pragma unroll
  for (int k = 0; k < G::E; ++k) {
    const int idx = win_index(tv, k, hb, lb);
    uint64_t* dst = cl.map_shared_rank(sm, idx >> GC::LOGNL);
    dst[swz<LOGE>(idx & (GC::NC - 1))] = x[k];
  }
  cl.sync();
  fwd_local_pass<LOGN, LOGE, LOGC, 1>(sm, x, tw, q, qf, st, tid, h);
}

template <int LOGN, int LOGE, int LOGC, int P, class Storer>
__device__ __forceinline__ void inv_local_pass(uint64_t* sm, uint64_t (&x)[1 << LOGE], const uint64_t* __restrict__ tw,
                                               uint64_t q, uint64_t c, uint64_t cs, const Storer& st, int tid, int h) {
  using GC = Geom<LOGN, LOGE, LOGC>;
  using G = typename GC::G;
  namespace cg = cooperative_groups;
  if constexpr (P + 1 < G::NPASS) {
    constexpr int lb = G::ilb(P), hb = lb + LOGE - 1;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < G::E; ++k) x[k] = sm[swz<LOGE>(win_index(tid, k, hb, lb))];
    inv_stages_c<LOGN, LOGE, P>(x, tw, q, tid, h, GC::LOGNL);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < G::E; ++k) sm[swz<LOGE>(win_index(tid, k, hb, lb))] = x[k];
    inv_local_pass<LOGN, LOGE, LOGC, P + 1>(sm, x, tw, q, c, cs, st, tid, h);
  } else {
    // last pass: crosses chunks; read the owners' shared memory
    constexpr int lb = G::ilb(P), hb = lb + LOGE - 1;
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    const int tv = h * GC::T + tid;
#pragma unroll
    for (int k = 0; k < G::E; ++k) {
      const int idx = win_index(tv, k, hb, lb);
      const uint64_t* src = cl.map_shared_rank(sm, idx >> GC::LOGNL);
      x[k] = src[swz<LOGE>(idx & (GC::NC - 1))];
    }
    inv_stages_c<LOGN, LOGE, P>(x, tw, q, tv, 0, LOGN);
#pragma unroll
    for (int k = 0; k < G::E; ++k) st(win_index(tv, k, hb, lb), shoup_mul(x[k], c, cs, q));
    cl.sync();                                        // peers may still read this CTA's shared memory
  }
}

// Inverse transform over the cluster, from data the caller has placed in this
// CTA's shared memory (element h n/C + i at sm[swz(i)]); st(i, v) for any i.
template <int LOGN, int LOGE, int LOGC, class Storer>
__device__ __forceinline__ void ntt_inverse_cluster_smem(uint64_t* sm, const uint64_t* __restrict__ tw, uint64_t q,
                                                         uint64_t c, uint64_t cs, const Storer& st) {
  namespace cg = cooperative_groups;
  const int h = (int)cg::this_cluster().block_rank();
  uint64_t x[1 << LOGE];
  inv_local_pass<LOGN, LOGE, LOGC, 0>(sm, x, tw, q, c, cs, st, (int)threadIdx.x, h);
}

// Inverse transform over the cluster; ld(i) is called for the i of this CTA's chunk.
template <int LOGN, int LOGE, int LOGC, class Loader, class Storer>
__device__ __forceinline__ void ntt_inverse_cluster(uint64_t* sm, const uint64_t* __restrict__ tw, uint64_t q,
                                                    uint64_t c, uint64_t cs, const Loader& ld, const Storer& st) {
  using GC = Geom<LOGN, LOGE, LOGC>;
  namespace cg = cooperative_groups;
  const int h = (int)cg::this_cluster().block_rank();
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < (1 << LOGE); ++k) {
    const int i = tid + k * GC::T;
    sm[swz<LOGE>(i)] = ld((h << GC::LOGNL) + i);
  }
  ntt_inverse_cluster_smem<LOGN, LOGE, LOGC>(sm, tw, q, c, cs, st);
}

}  // namespace ncl
}  // namespace lola
