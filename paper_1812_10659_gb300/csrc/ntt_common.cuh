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
}  // namespace k
}  // namespace lola
