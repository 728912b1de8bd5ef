// Shared pieces of the NTT-family kernel files (ntt_kernels.cu: plain
// transforms; ntt_keyswitch.cu: one-CTA key-switch transforms and the
// key-switch dispatch; ntt_cluster.cu: 2-CTA cluster versions at n = 16384):
// launch geometry, dispatch over ring degrees, the mod-down storer.
#pragma once
#include "internal.h"
#include "kernels.h"
#include "ntt.cuh"

namespace lola {

// Words per thread per pass.  At n = 16384 a CTA holds the whole limb in
// 128 KiB of shared memory, so one CTA runs per SM: 2^4 words (1024 threads,
// at most 64 registers) hides more latency, 2^5 words (512 threads, up to 128
// registers) avoids register spills in the forward transforms that read their
// input straight from global memory.  Measured per kernel: the mod-up,
// mod-down and plain forward / inverse transforms are faster with 512
// threads, decompose with 1024.
#ifndef LOLA_NTT14_LOGE
#define LOLA_NTT14_LOGE 4
#endif
#ifndef LOLA_NTT14_LOGE_MODUP
#define LOLA_NTT14_LOGE_MODUP 5
#endif

template <int LOGN, int LOGE14 = LOLA_NTT14_LOGE>
struct Cfg {
  static constexpr int LOGE = LOGN >= 14 ? LOGE14 : 4;
  static constexpr int N = 1 << LOGN;
  static constexpr int T = N >> LOGE;
};
template <int LOGN>
using CfgM = Cfg<LOGN, LOLA_NTT14_LOGE_MODUP>;

// (w, w') pair tables, 2n words per prime
#define TW_F(C, p) (C)->tw_fwd + (size_t)(p) * (2u << LOGN)
#define TW_I(C, p) (C)->tw_inv + (size_t)(p) * (2u << LOGN)

// Mod-up loader: digit g of a ciphertext at coefficient k, reduced towards
// prime j (a forward-transform input, below 8 q_j + 2^32).  dig: the
// ciphertext's digit limbs [L][n] in coefficient form, limb i = [c]_{q_i}.
// GROUPED = false (one prime per digit): the digit is limb g itself, passed
// raw when every prime is within a factor 8.  GROUPED = true: a two-prime
// digit over q_a, q_b (b = a + 1) is the integer a + q_a v, v = (b - a)
// q_a^-1 mod q_b, in [0, q_a q_b); the last digit of an odd L is single.
// The two forms are separate instantiations, so the one-prime kernels carry
// none of the two-prime code.
template <bool GROUPED>
struct ModupDigit {
  const uint64_t* da;   // limb a
  const uint64_t* db;   // limb b, or null for a single-prime digit
  uint64_t qa_j, qa_j_s, inv, inv_s;
  const PrimeDev* Pj;
  const PrimeDev* Pb;
  bool raw, lazy_a;
  __device__ __forceinline__ uint64_t operator()(int k) const {
    const uint64_t a = da[k];
    if (!GROUPED || !db) return raw ? a : reduce64(a, Pj->q, Pj->f64);
    const uint64_t qb = Pb->q;
    const uint64_t ab = a >= qb ? a - qb : a;                      // q_a < 2 q_b
    const uint64_t v = shoup_mul(sub_mod(db[k], ab, qb), inv, inv_s, qb);
    const uint64_t aj = lazy_a ? a : reduce64(a, Pj->q, Pj->f64);
    return aj + shoup_mul_lazy(v, qa_j, qa_j_s, Pj->q);
  }
};

template <bool GROUPED>
__device__ __forceinline__ ModupDigit<GROUPED> modup_digit(const CtxDev* __restrict__ C, const uint64_t* dig, int g,
                                                           int j, size_t n) {
  ModupDigit<GROUPED> m;
  m.Pj = &C->pr[j];
  m.raw = C->modup_raw != 0;
  if (!GROUPED) {
    m.da = dig + (size_t)g * n;
    m.db = nullptr;
    return m;
  }
  const int a = g * (int)C->alpha;
  m.da = dig + (size_t)a * n;
  m.db = (C->alpha > 1 && a + 1 < (int)C->L) ? dig + (size_t)(a + 1) * n : nullptr;
  m.Pb = &C->pr[a + 1 < (int)C->L ? a + 1 : a];
  m.lazy_a = C->modup_lazy_a != 0;
  if (m.db) {
    m.qa_j = C->grp_qa[g][j];
    m.qa_j_s = C->grp_qa_s[g][j];
    m.inv = C->grp_inv[g];
    m.inv_s = C->grp_inv_s[g];
  }
  return m;
}

// Mod-down loader: x~ P^-1 mod q_j (below 6 q_j) from the special-prime
// limbs of one inner product in coefficient form, x~ the centered residue
// of x mod P.  K2 = false (one special prime): x in [0, P), x P^-1 minus 1
// (= P P^-1) when x > (P-1)/2.  K2 = true: x = x1 + P1 v with v = (x2 - x1)
// P1^-1 mod P2, x > (P-1)/2 decided on the mixed-radix digits (v, x1), and
// x P^-1 = x1 P^-1 + v P1 P^-1.
template <bool K2>
struct ModDownLoad {
  const uint64_t* x1;
  const uint64_t* x2;   // second special-prime limb (K2)
  const CtxDev* C;
  const PrimeDev* Pj;
  const PrimeDev* P2;
  uint64_t Phalf, q2m1, Pinv, Pinv_s, P1Pinv, P1Pinv_s;
  __device__ __forceinline__ uint64_t operator()(int k) const {
    const uint64_t a = x1[k];
    if (!K2) return shoup_mul_lazy(a, Pinv, Pinv_s, Pj->q) + (a > Phalf ? q2m1 : 0);
    const uint64_t p2 = P2->q;
    const uint64_t a2 = reduce64(a, p2, P2->f64);
    const uint64_t v = shoup_mul(sub_mod(x2[k], a2, p2), C->P1invP2, C->P1invP2_s, p2);
    const bool neg = v > C->phv || (v == C->phv && a > C->ph1);
    return shoup_mul_lazy(a, Pinv, Pinv_s, Pj->q) + shoup_mul_lazy(v, P1Pinv, P1Pinv_s, Pj->q) + (neg ? q2m1 : 0);
  }
};

// xP: the special-prime limbs of the inner products in coefficient form,
// [ct][2][K][n]; out limb (ct, comp, j)
template <bool K2>
__device__ __forceinline__ ModDownLoad<K2> moddown_load(const CtxDev* __restrict__ C, const uint64_t* xP, size_t ct,
                                                       int comp, int j, size_t n) {
  ModDownLoad<K2> m;
  const int K = K2 ? 2 : 1;
  m.x1 = xP + (ct * 2 + comp) * (size_t)K * n;
  m.x2 = K2 ? m.x1 + n : nullptr;
  m.C = C;
  m.Pj = &C->pr[j];
  m.P2 = &C->pr[C->iP + (K2 ? 1 : 0)];
  m.Phalf = (C->pr[C->iP].q - 1) / 2;
  m.q2m1 = 2 * m.Pj->q - 1;
  m.Pinv = C->PinvQ[j];
  m.Pinv_s = C->PinvQ_s[j];
  if (K2) {
    m.P1Pinv = C->P1PinvQ[j];
    m.P1Pinv_s = C->P1PinvQ_s[j];
  }
  return m;
}

// mod-down epilogue: the inner-product limb is fetched ahead of the stores
struct ModDownStore {
  const uint64_t* acc;
  uint64_t* dst;
  uint64_t q;
  __device__ __forceinline__ uint64_t fetch(int k) const { return acc[k]; }
  __device__ __forceinline__ void operator()(int k, uint64_t v, uint64_t f) const { dst[k] = sub_mod(f, v, q); }
};

// ------------------------------------------------------------------ dispatch
#define LOLA_DISPATCH(logn, KERNEL, grid, stream, ...) LOLA_DISPATCH_CFG(Cfg, logn, KERNEL, grid, stream, __VA_ARGS__)
#define LOLA_DISPATCH_CFG(CFG, logn, KERNEL, grid, stream, ...)                                     \
  do {                                                                                             \
    switch (logn) {                                                                                \
      case 4: LOLA_LAUNCH(CFG, 4, KERNEL, grid, stream, __VA_ARGS__); break;                       \
      case 5: LOLA_LAUNCH(CFG, 5, KERNEL, grid, stream, __VA_ARGS__); break;                            \
      case 6: LOLA_LAUNCH(CFG, 6, KERNEL, grid, stream, __VA_ARGS__); break;                            \
      case 7: LOLA_LAUNCH(CFG, 7, KERNEL, grid, stream, __VA_ARGS__); break;                            \
      case 8: LOLA_LAUNCH(CFG, 8, KERNEL, grid, stream, __VA_ARGS__); break;                            \
      case 9: LOLA_LAUNCH(CFG, 9, KERNEL, grid, stream, __VA_ARGS__); break;                            \
      case 10: LOLA_LAUNCH(CFG, 10, KERNEL, grid, stream, __VA_ARGS__); break;                          \
      case 11: LOLA_LAUNCH(CFG, 11, KERNEL, grid, stream, __VA_ARGS__); break;                          \
      case 12: LOLA_LAUNCH(CFG, 12, KERNEL, grid, stream, __VA_ARGS__); break;                          \
      case 13: LOLA_LAUNCH(CFG, 13, KERNEL, grid, stream, __VA_ARGS__); break;                          \
      case 14: LOLA_LAUNCH(CFG, 14, KERNEL, grid, stream, __VA_ARGS__); break;                          \
      default: return fail(LOLA_E_PARAM, "unsupported ring degree");                                \
    }                                                                                              \
  } while (0)

#define LOLA_LAUNCH(CFG, LG, KERNEL, grid, stream, ...)                                            \
  do {                                                                                             \
    const size_t smem = sizeof(uint64_t) << (LG);                                                  \
    static bool attr_done = false;                                                                 \
    if (!attr_done) {                                                                              \
      cudaFuncSetAttribute(KERNEL<LG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);    \
      attr_done = true;                                                                            \
    }                                                                                              \
    KERNEL<LG><<<(unsigned)(grid), CFG<LG>::T, smem, stream>>>(__VA_ARGS__);                       \
  } while (0)

static inline int post_launch(Ctx* c, cudaStream_t) {
  c->root->launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LOLA_E_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return LOLA_OK;
}

// ------------------------------------------- n = 16384: cluster versions
// Each limb transform is split over a cluster of 2 or 4 CTAs (1/C of the
// limb each in shared memory), so a launch with few limbs still keeps more
// SMs busy and each dependent step of a rotation takes less time.
// Geometries: 2 CTAs with 2^5 words per thread (256 threads per CTA, up to
// 128 registers) for launches of many limbs, where per-thread ILP and three
// passes win; 2 CTAs with 2^4 words (512 threads, 64 registers, four passes)
// for small launches, where more threads per transform shorten its latency;
// 4 CTAs with 2^4 words (256 threads and 32 KiB per CTA) for the smallest
// launches (single-request evaluation), where a transform's latency is the
// step's.
constexpr int CL_LOGN = 14, CL_LOGC = 1;
template <int LOGE, int LOGC = CL_LOGC>
constexpr int cl_threads() { return (1 << CL_LOGN) >> (LOGE + LOGC); }
// plain transforms (ntt_fwd_map / ntt_inv_map) at n = 16384: launches of
// fewer limbs than these run as 4-CTA / 2-CTA clusters (16 words a thread)
#ifndef LOLA_NTT_CL4_UNITS
#define LOLA_NTT_CL4_UNITS 128
#endif
#ifndef LOLA_NTT_CL2_UNITS
#define LOLA_NTT_CL2_UNITS 512
#endif
// launches with fewer limb transforms than this use the 2^4 geometry
#ifndef LOLA_CL_SMALL_UNITS
#define LOLA_CL_SMALL_UNITS 400
#endif

#define LOLA_LAUNCH_CLUSTER(KERNEL, LOGC, units, threads, stream, ...)                              \
  do {                                                                                             \
    const size_t smem = sizeof(uint64_t) << (CL_LOGN - (LOGC));                                     \
    static bool attr_done = false;                                                                 \
    if (!attr_done) {                                                                              \
      cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
      attr_done = true;                                                                            \
    }                                                                                              \
    KERNEL<<<(unsigned)((units) << (LOGC)), threads, smem, stream>>>(__VA_ARGS__);                  \
  } while (0)

namespace k {
// cluster launches (ntt_cluster.cu); `variant` is a TuneVariant other than TV_CTA
int ks_decompose_cluster(Ctx* c, const KsDev& a, cudaStream_t s, int variant);
int ks_modup_cluster(Ctx* c, const KsDev& a, bool skip_diag, cudaStream_t s, int variant);
int ks_intt_p_cluster(Ctx* c, const KsDev& a, cudaStream_t s, int variant);
int ks_moddown_cluster(Ctx* c, const KsDev& a, cudaStream_t s, int variant);
// plain transforms of small launches at n = 16384
int ntt_fwd_cluster(Ctx* c, const uint64_t* in, uint64_t* out, size_t n_polys, uint32_t limbs, const PrimeMap& pm,
                    cudaStream_t s, int variant);
int ntt_inv_cluster(Ctx* c, const uint64_t* in, uint64_t* out, size_t n_polys, uint32_t limbs, const PrimeMap& pm,
                    bool mont_fix, cudaStream_t s, int variant);
}  // namespace k
}  // namespace lola
