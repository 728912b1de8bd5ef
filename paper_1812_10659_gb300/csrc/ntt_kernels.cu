// NTT-family kernels: every kernel here runs one negacyclic transform per
// CTA (ntt.cuh) with a kernel-specific loader (what feeds the transform) and
// storer (what happens to each output word).  Fusing the neighbouring
// element-wise work into the transform's first load / last store is what
// keeps each limb to one HBM read and one HBM write.
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

// ------------------------------------------------------------ plain transforms
template <int LOGN>
__global__ void __launch_bounds__(CfgM<LOGN>::T) kn_fwd(const CtxDev* __restrict__ C, const uint64_t* in,
                                                        uint64_t* out, uint32_t limbs, PrimeMap pm) {
  extern __shared__ uint64_t sm[];
  constexpr int N = CfgM<LOGN>::N;
  const size_t poly = blockIdx.x;
  const int p = pm.p[poly % limbs];
  const uint64_t* src = in + poly * N;
  uint64_t* dst = out + poly * N;
  ntt_forward<LOGN, CfgM<LOGN>::LOGE>(sm, TW_F(C, p), C->pr[p].q, C->pr[p].f64, [&](int i) { return src[i]; },
                                      [&](int i, uint64_t v) { dst[i] = v; });
}

template <int LOGN>
__global__ void __launch_bounds__(CfgM<LOGN>::T) kn_inv(const CtxDev* __restrict__ C, const uint64_t* in,
                                                        uint64_t* out, uint32_t limbs, PrimeMap pm, int mont_fix) {
  extern __shared__ uint64_t sm[];
  constexpr int N = CfgM<LOGN>::N;
  const size_t poly = blockIdx.x;
  const int p = pm.p[poly % limbs];
  const PrimeDev& P = C->pr[p];
  const uint64_t* src = in + poly * N;
  uint64_t* dst = out + poly * N;
  const uint64_t c = mont_fix ? P.ninvr : P.ninv, cs = mont_fix ? P.ninvr_s : P.ninv_s;
  ntt_inverse<LOGN, CfgM<LOGN>::LOGE>(sm, TW_I(C, p), P.q, c, cs, [&](int i) { return src[i]; },
                                      [&](int i, uint64_t v) { dst[i] = v; });
}

// small signed integers (int64 [poly][n]) -> NTT mod each prime of the map
template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::T) kn_fwd_signed(const CtxDev* __restrict__ C, const int64_t* in,
                                                               uint64_t* out, uint32_t limbs, PrimeMap pm) {
  extern __shared__ uint64_t sm[];
  constexpr int N = Cfg<LOGN>::N;
  const size_t blk = blockIdx.x;
  const size_t poly = blk / limbs;
  const int p = pm.p[blk % limbs];
  const PrimeDev& P = C->pr[p];
  const int64_t* src = in + poly * N;
  uint64_t* dst = out + blk * N;
  ntt_forward<LOGN, Cfg<LOGN>::LOGE>(sm, TW_F(C, p), P.q, P.f64,
                                      [&](int i) { return from_signed(src[i], P.q, P.f64); },
                                      [&](int i, uint64_t v) { dst[i] = v; });
}

// plaintext polynomial mod t -> centered lift -> mod q_l -> NTT (-> Montgomery)
template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::T) kn_encode_lift(const CtxDev* __restrict__ C, const uint64_t* in,
                                                                const uint32_t* tidx, uint64_t* out, uint32_t limbs,
                                                                int mont) {
  extern __shared__ uint64_t sm[];
  constexpr int N = Cfg<LOGN>::N;
  const size_t blk = blockIdx.x;
  const size_t poly = blk / limbs;
  const int l = blk % limbs;
  const PrimeDev& P = C->pr[l];
  const uint64_t t = C->pr[C->iT + tidx[poly]].q;
  const uint64_t* src = in + poly * N;
  uint64_t* dst = out + blk * N;
  ntt_forward<LOGN, Cfg<LOGN>::LOGE>(
      sm, TW_F(C, l), P.q, P.f64,
      [&](int i) {
        const uint64_t x = src[i];
        return x <= (t - 1) / 2 ? reduce64(x, P.q, P.f64) : neg_mod(reduce64(t - x, P.q, P.f64), P.q);
      },
      [&](int i, uint64_t v) { dst[i] = mont ? mont_mul(v, P.r2, P.q, P.qinv) : v; });
}

// slots (mod t) -> plaintext coefficients: inverse transform mod t fed through the slot map
template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::T) kn_slots_to_coeff(const CtxDev* __restrict__ C, const uint64_t* slots,
                                                                   const uint32_t* tidx, const uint32_t* slot_at_pos,
                                                                   uint64_t* coeff) {
  extern __shared__ uint64_t sm[];
  constexpr int N = Cfg<LOGN>::N;
  const size_t poly = blockIdx.x;
  const int p = C->iT + tidx[poly];
  const PrimeDev& P = C->pr[p];
  const uint64_t* src = slots + poly * N;
  uint64_t* dst = coeff + poly * N;
  ntt_inverse<LOGN, Cfg<LOGN>::LOGE>(sm, TW_I(C, p), P.q, P.ninv, P.ninv_s,
                                      [&](int i) { return src[slot_at_pos[i]]; },
                                      [&](int i, uint64_t v) { dst[i] = v; });
}

template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::T) kn_coeff_to_slots(const CtxDev* __restrict__ C, const uint64_t* coeff,
                                                                   const uint32_t* tidx, const uint32_t* slot_at_pos,
                                                                   uint64_t* slots) {
  extern __shared__ uint64_t sm[];
  constexpr int N = Cfg<LOGN>::N;
  const size_t poly = blockIdx.x;
  const int p = C->iT + tidx[poly];
  const uint64_t* src = coeff + poly * N;
  uint64_t* dst = slots + poly * N;
  ntt_forward<LOGN, Cfg<LOGN>::LOGE>(sm, TW_F(C, p), C->pr[p].q, C->pr[p].f64, [&](int i) { return src[i]; },
                                      [&](int i, uint64_t v) { dst[slot_at_pos[i]] = v; });
}

// encryption: NTT_j(Delta_t * m + e1) per limb (m coefficients mod t, e1 signed)
template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::T) kn_enc_msg(const CtxDev* __restrict__ C, const uint64_t* m,
                                                            const int64_t* e1, const uint32_t* tidx, uint64_t* out,
                                                            uint32_t L) {
  extern __shared__ uint64_t sm[];
  constexpr int N = Cfg<LOGN>::N;
  const size_t blk = blockIdx.x;
  const size_t poly = blk / L;
  const int j = blk % L;
  const PrimeDev& P = C->pr[j];
  const uint32_t ti = tidx[poly];
  const uint64_t d = C->deltaQ[ti][j], ds = C->deltaQ_s[ti][j];
  const uint64_t* ms = m + poly * N;
  const int64_t* es = e1 + poly * N;
  uint64_t* dst = out + blk * N;
  ntt_forward<LOGN, Cfg<LOGN>::LOGE>(
      sm, TW_F(C, j), P.q, P.f64,
      [&](int i) { return add_mod(shoup_mul(ms[i], d, ds, P.q), from_signed(es[i], P.q, P.f64), P.q); },
      [&](int i, uint64_t v) { dst[i] = v; });
}

// ------------------------------------------------------------- key switching
// A: the Galois automorphism in NTT form is a permutation of positions.
//    Load c1 limb i coalesced and scatter it through the inverse permutation
//    into shared memory; write the permuted limb (the diagonal block D[i][i])
//    back coalesced; inverse-transform it into digit i.  When c0p is given,
//    tau_g(c0) is written the same way first (otherwise the inner product
//    gathers it).
template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::T) kn_ks_decompose(const CtxDev* __restrict__ C, KsDev a) {
  extern __shared__ uint64_t sm[];
  constexpr int N = Cfg<LOGN>::N, T = Cfg<LOGN>::T, LOGE = Cfg<LOGN>::LOGE;
  const int L = C->L, LK = C->L + C->K;
  const size_t ct = blockIdx.x / L;
  const int i = blockIdx.x % L;
  const uint32_t g = a.d_gal ? a.d_gal[ct / a.gal_div] : a.gal;
  const uint32_t ginv = inv_odd32(g) & ((2u << LOGN) - 1);
  const int tid = threadIdx.x;
  const uint64_t* src0 = a.c1 + (ct * 2 * L + i) * (size_t)N;
  const uint64_t* src1 = a.c1 + (ct * 2 * L + L + i) * (size_t)N;
  uint64_t* diag = a.D + ((ct * L + i) * LK + i) * (size_t)N;
  uint64_t* dig = a.dig + (ct * L + i) * (size_t)N;
  const PrimeDev& P = C->pr[i];
  uint64_t v[N / T];
  if (a.c0p) {
    // tau_g(c0): all loads of the thread first (the compiler may not move a
    // global load above a shared store through a generic pointer)
    uint64_t* c0p = a.c0p + (ct * L + i) * (size_t)N;
#pragma unroll
    for (int k = 0; k < N / T; ++k) v[k] = src0[tid + k * T];
#pragma unroll
    for (int k = 0; k < N / T; ++k) sm[swz<LOGE>(gal_dst(tid + k * T, ginv, LOGN))] = v[k];
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < N / T; ++k) {
      const int idx = tid + k * T;
      c0p[idx] = sm[swz<LOGE>(idx)];
    }
    __syncthreads();
  }
  // tau_g(c1): diagonal block, then digit
#pragma unroll
  for (int k = 0; k < N / T; ++k) v[k] = src1[tid + k * T];
#pragma unroll
  for (int k = 0; k < N / T; ++k) sm[swz<LOGE>(gal_dst(tid + k * T, ginv, LOGN))] = v[k];
  __syncthreads();
#pragma unroll 4
  for (int k = 0; k < N / T; ++k) {
    const int idx = tid + k * T;
    diag[idx] = sm[swz<LOGE>(idx)];
  }
  ntt_inverse_smem<LOGN, LOGE>(sm, TW_I(C, i), P.q, P.ninv, P.ninv_s, [&](int k2, uint64_t v) { dig[k2] = v; });
}

// B: digit i reduced mod prime j, forward transform -> D[i][j]
template <int LOGN>
__global__ void __launch_bounds__(CfgM<LOGN>::T) kn_ks_modup(const CtxDev* __restrict__ C, KsDev a, int skip_diag) {
  extern __shared__ uint64_t sm[];
  constexpr int N = CfgM<LOGN>::N;
  const int L = C->L, LK = C->L + C->K;
  const int per = skip_diag ? L * (LK - 1) : L * LK;
  const size_t ct = blockIdx.x / per;
  const int r = blockIdx.x % per;
  const int i = r / (skip_diag ? LK - 1 : LK);
  int j = r % (skip_diag ? LK - 1 : LK);
  if (skip_diag && j >= i) ++j;
  const uint64_t* dig = a.dig + (ct * L + i) * (size_t)N;
  uint64_t* dst = a.D + ((ct * L + i) * LK + j) * (size_t)N;
  const PrimeDev& P = C->pr[j];
  const bool raw = C->modup_raw != 0;
  ntt_forward<LOGN, CfgM<LOGN>::LOGE>(sm, TW_F(C, j), P.q, P.f64, [&](int k) { return raw ? dig[k] : reduce64(dig[k], P.q, P.f64); },
                                      [&](int k, uint64_t v) { dst[k] = v; });
}

// D: inverse transform of the special-prime inner products (both components)
template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::T) kn_ks_intt_p(const CtxDev* __restrict__ C, KsDev a) {
  extern __shared__ uint64_t sm[];
  constexpr int N = Cfg<LOGN>::N;
  const int LK = C->L + C->K, ip = C->iP;
  const size_t ct = blockIdx.x >> 1;
  const int comp = blockIdx.x & 1;
  const PrimeDev& P = C->pr[ip];
  const uint64_t* src = a.acc + ct * a.acc_stride + (size_t)(comp * LK + ip) * N;
  uint64_t* dst = a.xP + (ct * 2 + comp) * (size_t)N;
  ntt_inverse<LOGN, Cfg<LOGN>::LOGE>(sm, TW_I(C, ip), P.q, P.ninv, P.ninv_s, [&](int k) { return src[k]; },
                                      [&](int k, uint64_t v) { dst[k] = v; });
}

// mod-down epilogue: the inner-product limb is fetched ahead of the stores
struct ModDownStore {
  const uint64_t* acc;
  uint64_t* dst;
  uint64_t q;
  __device__ __forceinline__ uint64_t fetch(int k) const { return acc[k]; }
  __device__ __forceinline__ void operator()(int k, uint64_t v, uint64_t f) const { dst[k] = sub_mod(f, v, q); }
};

// E: output limb out[comp][j] = ACC'[comp][j] - NTT(x~ P^-1 mod q_j), with
//    x~ = centered(x mod P); the inner-product kernel left ACC' = ACC P^-1 +
//    addend + accumulator (the keys carry P^-1).  The loader multiplies the
//    raw residue x in [0, P) by P^-1 mod q_j (Shoup, any 64-bit input) and
//    subtracts 1 = P P^-1 where x~ = x - P; its value stays below 4q, which
//    the forward butterflies accept.
template <int LOGN>
__global__ void __launch_bounds__(CfgM<LOGN>::T) kn_ks_moddown(const CtxDev* __restrict__ C, KsDev a) {
  extern __shared__ uint64_t sm[];
  constexpr int N = CfgM<LOGN>::N;
  const int L = C->L, LK = C->L + C->K;
  const size_t ct = blockIdx.x / (2 * L);
  const int r = blockIdx.x % (2 * L);
  const int comp = r / L, j = r % L;
  const uint32_t g = a.d_gal ? a.d_gal[ct / a.gal_div] : a.gal;
  const uint64_t* accp = a.acc + ct * a.acc_stride + (size_t)(comp * LK + j) * N;
  const PrimeDev& P = C->pr[j];
  const uint64_t Phalf = (C->pr[C->iP].q - 1) / 2, q2m1 = 2 * P.q - 1;
  const uint64_t Pinv = C->PinvQ[j], Pinv_s = C->PinvQ_s[j];
  const uint64_t* x = a.xP + (ct * 2 + comp) * (size_t)N;
  uint64_t* dst = a.out + ((ct * 2 + comp) * L + j) * (size_t)N;
  ntt_forward<LOGN, CfgM<LOGN>::LOGE>(
      sm, TW_F(C, j), P.q, P.f64,
      [&](int k) {
        const uint64_t v = x[k];
        return shoup_mul_lazy(v, Pinv, Pinv_s, P.q) + (v > Phalf ? q2m1 : 0);
      },
      ModDownStore{accp, dst, P.q});
}

// ------------------------------------------- n = 16384: 2-CTA cluster versions
// Each limb transform is split over a cluster of two CTAs (half the limb each,
// 64 KiB of shared memory), so a launch with few limbs still keeps twice as
// many SMs busy and each dependent step of a rotation takes half as long.
// Two geometries: 2^5 words per thread (256 threads per CTA, up to 128
// registers) for launches of many limbs, where per-thread ILP and three
// passes win; 2^4 words (512 threads, 64 registers, four passes) for small
// launches, where more threads per transform shorten its latency.
constexpr int CL_LOGN = 14, CL_LOGC = 1;
template <int LOGE>
constexpr int cl_threads() { return (1 << CL_LOGN) >> (LOGE + CL_LOGC); }
// launches with fewer limb transforms than this use the 2^4 geometry
#ifndef LOLA_CL_SMALL_UNITS
#define LOLA_CL_SMALL_UNITS 400
#endif

template <int CL_LOGE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(cl_threads<CL_LOGE>(), 2)
    kc_ks_modup(const CtxDev* __restrict__ C, KsDev a, int skip_diag) {
  extern __shared__ uint64_t sm[];
  constexpr int N = 1 << CL_LOGN;
  const int L = C->L, LK = C->L + C->K;
  const int per = skip_diag ? L * (LK - 1) : L * LK;
  const size_t unit = blockIdx.x >> 1;
  const size_t ct = unit / per;
  const int r = unit % per;
  const int i = r / (skip_diag ? LK - 1 : LK);
  int j = r % (skip_diag ? LK - 1 : LK);
  if (skip_diag && j >= i) ++j;
  const uint64_t* dig = a.dig + (ct * L + i) * (size_t)N;
  uint64_t* dst = a.D + ((ct * L + i) * LK + j) * (size_t)N;
  const PrimeDev& P = C->pr[j];
  const bool raw = C->modup_raw != 0;
  ncl::ntt_forward_cluster<CL_LOGN, CL_LOGE, CL_LOGC>(sm, C->tw_fwd + (size_t)j * (2u << CL_LOGN), P.q, P.f64,
                                                [&](int k) { return raw ? dig[k] : reduce64(dig[k], P.q, P.f64); },
                                                [&](int k, uint64_t v) { dst[k] = v; });
}

template <int CL_LOGE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(cl_threads<CL_LOGE>(), 2) kc_ks_intt_p(const CtxDev* __restrict__ C, KsDev a) {
  extern __shared__ uint64_t sm[];
  constexpr int N = 1 << CL_LOGN;
  const int LK = C->L + C->K, ip = C->iP;
  const size_t unit = blockIdx.x >> 1;
  const size_t ct = unit >> 1;
  const int comp = unit & 1;
  const PrimeDev& P = C->pr[ip];
  const uint64_t* src = a.acc + ct * a.acc_stride + (size_t)(comp * LK + ip) * N;
  uint64_t* dst = a.xP + (ct * 2 + comp) * (size_t)N;
  ncl::ntt_inverse_cluster<CL_LOGN, CL_LOGE, CL_LOGC>(sm, C->tw_inv + (size_t)ip * (2u << CL_LOGN), P.q, P.ninv, P.ninv_s,
                                                [&](int k) { return src[k]; },
                                                [&](int k, uint64_t v) { dst[k] = v; });
}

template <int CL_LOGE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(cl_threads<CL_LOGE>(), 2) kc_ks_moddown(const CtxDev* __restrict__ C, KsDev a) {
  extern __shared__ uint64_t sm[];
  constexpr int N = 1 << CL_LOGN;
  const int L = C->L, LK = C->L + C->K;
  const size_t unit = blockIdx.x >> 1;
  const size_t ct = unit / (2 * L);
  const int r = unit % (2 * L);
  const int comp = r / L, j = r % L;
  const uint64_t* accp = a.acc + ct * a.acc_stride + (size_t)(comp * LK + j) * N;
  const PrimeDev& P = C->pr[j];
  const uint64_t Phalf = (C->pr[C->iP].q - 1) / 2, q2m1 = 2 * P.q - 1;
  const uint64_t Pinv = C->PinvQ[j], Pinv_s = C->PinvQ_s[j];
  const uint64_t* x = a.xP + (ct * 2 + comp) * (size_t)N;
  uint64_t* dst = a.out + ((ct * 2 + comp) * L + j) * (size_t)N;
  ncl::ntt_forward_cluster<CL_LOGN, CL_LOGE, CL_LOGC>(
      sm, C->tw_fwd + (size_t)j * (2u << CL_LOGN), P.q, P.f64,
      [&](int k) {
        const uint64_t v = x[k];
        return shoup_mul_lazy(v, Pinv, Pinv_s, P.q) + (v > Phalf ? q2m1 : 0);
      },
      ModDownStore{accp, dst, P.q});
}

template <int CL_LOGE>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(cl_threads<CL_LOGE>(), 2) kc_ks_decompose(const CtxDev* __restrict__ C, KsDev a) {
  extern __shared__ uint64_t sm[];
  namespace cg = cooperative_groups;
  constexpr int N = 1 << CL_LOGN, LOGE = CL_LOGE, LOGNL = CL_LOGN - CL_LOGC, NC = 1 << LOGNL;
  constexpr int T = N >> (LOGE + CL_LOGC);
  cg::cluster_group cl = cg::this_cluster();
  const int h = (int)cl.block_rank();
  const int L = C->L, LK = C->L + C->K;
  const size_t unit = blockIdx.x >> 1;
  const size_t ct = unit / L;
  const int i = unit % L;
  const uint32_t g = a.d_gal ? a.d_gal[ct / a.gal_div] : a.gal;
  const uint32_t ginv = inv_odd32(g) & ((2u << CL_LOGN) - 1);
  const int tid = threadIdx.x;
  const uint64_t* src0 = a.c1 + (ct * 2 * L + i) * (size_t)N;
  const uint64_t* src1 = a.c1 + (ct * 2 * L + L + i) * (size_t)N;
  uint64_t* diag = a.D + ((ct * L + i) * LK + i) * (size_t)N;
  uint64_t* dig = a.dig + (ct * L + i) * (size_t)N;
  const PrimeDev& P = C->pr[i];
  // the peers must have started before their shared memory is written: a
  // cluster barrier, overlapped with the first loads
  cl.barrier_arrive();
  if (a.c0p) {
    // tau_g(c0): this CTA reads its chunk of c0 and scatters through the
    // inverse permutation (c0p is the same for the whole cluster)
    uint64_t* c0p = a.c0p + (ct * L + i) * (size_t)N;
    uint64_t v[NC / T];
#pragma unroll
    for (int k = 0; k < NC / T; ++k) v[k] = src0[(h << LOGNL) + tid + k * T];
    cl.barrier_wait();
#pragma unroll
    for (int k = 0; k < NC / T; ++k) {
      const uint32_t d = gal_dst((h << LOGNL) + tid + k * T, ginv, CL_LOGN);
      cl.map_shared_rank(sm, (int)(d >> LOGNL))[swz<LOGE>(d & (NC - 1))] = v[k];
    }
    cl.sync();
#pragma unroll 4
    for (int k = 0; k < NC / T; ++k) {
      const int li = tid + k * T;
      c0p[(h << LOGNL) + li] = sm[swz<LOGE>(li)];
    }
    cl.sync();
  } else {
    cl.barrier_wait();
  }
  // tau_g(c1): diagonal block, then the digit
#pragma unroll 4
  for (int k = 0; k < NC / T; ++k) {
    const int idx = (h << LOGNL) + tid + k * T;
    const uint32_t d = gal_dst(idx, ginv, CL_LOGN);
    cl.map_shared_rank(sm, (int)(d >> LOGNL))[swz<LOGE>(d & (NC - 1))] = src1[idx];
  }
  cl.sync();
#pragma unroll 4
  for (int k = 0; k < NC / T; ++k) {
    const int li = tid + k * T;
    diag[(h << LOGNL) + li] = sm[swz<LOGE>(li)];
  }
  ncl::ntt_inverse_cluster_smem<CL_LOGN, LOGE, CL_LOGC>(sm, C->tw_inv + (size_t)i * (2u << CL_LOGN), P.q, P.ninv,
                                                        P.ninv_s, [&](int k2, uint64_t v) { dig[k2] = v; });
}

#define LOLA_LAUNCH_CLUSTER(KERNEL, units, threads, stream, ...)                                    \
  do {                                                                                             \
    const size_t smem = sizeof(uint64_t) << (CL_LOGN - CL_LOGC);                                    \
    static bool attr_done = false;                                                                 \
    if (!attr_done) {                                                                              \
      cudaFuncSetAttribute(KERNEL, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);        \
      attr_done = true;                                                                            \
    }                                                                                              \
    KERNEL<<<(unsigned)((units) << CL_LOGC), threads, smem, stream>>>(__VA_ARGS__);                 \
  } while (0)

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

static int post_launch(Ctx* c, cudaStream_t) {
  c->launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LOLA_E_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return LOLA_OK;
}

namespace k {

static PrimeMap contiguous_map(uint32_t limbs, uint32_t prime0) {
  PrimeMap m{};
  for (uint32_t l = 0; l < limbs && l < sizeof(m.p); ++l) m.p[l] = (uint8_t)(prime0 + l);
  return m;
}

int ntt_fwd_map(Ctx* c, const uint64_t* in, uint64_t* out, size_t n_polys, uint32_t limbs, const PrimeMap& pm,
                cudaStream_t s) {
  if (!n_polys) return LOLA_OK;
  ProfScope ps(c, KI_NTT_FWD, s, n_polys);
  LOLA_DISPATCH_CFG(CfgM, c->logn, kn_fwd, n_polys, s, c->dev, in, out, limbs, pm);
  return post_launch(c, s);
}

int ntt_inv_map(Ctx* c, const uint64_t* in, uint64_t* out, size_t n_polys, uint32_t limbs, const PrimeMap& pm,
                bool mont_fix, cudaStream_t s) {
  if (!n_polys) return LOLA_OK;
  ProfScope ps(c, KI_NTT_INV, s, n_polys);
  LOLA_DISPATCH_CFG(CfgM, c->logn, kn_inv, n_polys, s, c->dev, in, out, limbs, pm, (int)mont_fix);
  return post_launch(c, s);
}

int ntt_fwd(Ctx* c, uint64_t* data, size_t n_polys, uint32_t limbs, uint32_t prime0, cudaStream_t s) {
  return ntt_fwd_map(c, data, data, n_polys * limbs, limbs, contiguous_map(limbs, prime0), s);
}

int ntt_inv(Ctx* c, uint64_t* data, size_t n_polys, uint32_t limbs, uint32_t prime0, bool mont_fix,
            cudaStream_t s) {
  return ntt_inv_map(c, data, data, n_polys * limbs, limbs, contiguous_map(limbs, prime0), mont_fix, s);
}

int ntt_fwd_from_signed(Ctx* c, const int64_t* in, uint64_t* out, size_t n_polys, uint32_t limbs, uint32_t prime0,
                        cudaStream_t s) {
  if (!n_polys) return LOLA_OK;
  PrimeMap pm = contiguous_map(limbs, prime0);
  ProfScope ps(c, KI_NTT_SIGNED, s, n_polys * limbs);
  LOLA_DISPATCH(c->logn, kn_fwd_signed, n_polys * limbs, s, c->dev, in, out, limbs, pm);
  return post_launch(c, s);
}

int encode_lift(Ctx* c, const uint64_t* in, const uint32_t* d_tidx, uint64_t* out, size_t n_polys, uint32_t limbs,
                bool mont, cudaStream_t s) {
  if (!n_polys) return LOLA_OK;
  ProfScope ps(c, KI_ENCODE_LIFT, s, n_polys * limbs);
  LOLA_DISPATCH(c->logn, kn_encode_lift, n_polys * limbs, s, c->dev, in, d_tidx, out, limbs, (int)mont);
  return post_launch(c, s);
}

int slots_to_coeff(Ctx* c, const uint64_t* slots, const uint32_t* d_tidx, uint64_t* coeff, size_t n_polys,
                   cudaStream_t s) {
  if (!n_polys) return LOLA_OK;
  ProfScope ps(c, KI_SLOTS_TO_COEFF, s, n_polys);
  LOLA_DISPATCH(c->logn, kn_slots_to_coeff, n_polys, s, c->dev, slots, d_tidx, (const uint32_t*)c->d_slotpos.p, coeff);
  return post_launch(c, s);
}

int coeff_to_slots(Ctx* c, const uint64_t* coeff, const uint32_t* d_tidx, uint64_t* slots, size_t n_polys,
                   cudaStream_t s) {
  if (!n_polys) return LOLA_OK;
  ProfScope ps(c, KI_COEFF_TO_SLOTS, s, n_polys);
  LOLA_DISPATCH(c->logn, kn_coeff_to_slots, n_polys, s, c->dev, coeff, d_tidx, (const uint32_t*)c->d_slotpos.p, slots);
  return post_launch(c, s);
}

int enc_msg(Ctx* c, const uint64_t* m, const int64_t* e1, const uint32_t* d_tidx, uint64_t* out, size_t n_polys,
            cudaStream_t s) {
  if (!n_polys) return LOLA_OK;
  ProfScope ps(c, KI_ENC_MSG, s, n_polys * c->L);
  LOLA_DISPATCH(c->logn, kn_enc_msg, n_polys * c->L, s, c->dev, m, e1, d_tidx, out, c->L);
  return post_launch(c, s);
}

// which key-switch transforms run as 2-CTA clusters at n = 16384 (bit 0
// decompose, 1 mod-up, 2 INTT mod P, 3 mod-down)
#ifndef LOLA_CLUSTER_MASK
#define LOLA_CLUSTER_MASK 0xE
#endif
static constexpr unsigned kClusterMask = LOLA_CLUSTER_MASK;

int ks_decompose(Ctx* c, const KsDev& a, cudaStream_t s) {
  ProfScope ps(c, KI_KS_DECOMPOSE, s, a.count * c->L);
  if ((kClusterMask & 1u) && c->logn == CL_LOGN) {
    if (a.count * c->L < LOLA_CL_SMALL_UNITS)
      LOLA_LAUNCH_CLUSTER(kc_ks_decompose<4>, a.count * c->L, cl_threads<4>(), s, c->dev, a);
    else
      LOLA_LAUNCH_CLUSTER(kc_ks_decompose<5>, a.count * c->L, cl_threads<5>(), s, c->dev, a);
    return post_launch(c, s);
  }
  LOLA_DISPATCH(c->logn, kn_ks_decompose, a.count * c->L, s, c->dev, a);
  return post_launch(c, s);
}

int ks_modup(Ctx* c, const KsDev& a, bool skip_diag, cudaStream_t s) {
  const uint32_t LK = c->L + c->K;
  const size_t per = skip_diag ? (size_t)c->L * (LK - 1) : (size_t)c->L * LK;
  if (!per) return LOLA_OK;
  ProfScope ps(c, KI_KS_MODUP, s, a.count * per);
  if ((kClusterMask & 2u) && c->logn == CL_LOGN) {
    if (a.count * per < LOLA_CL_SMALL_UNITS)
      LOLA_LAUNCH_CLUSTER(kc_ks_modup<4>, a.count * per, cl_threads<4>(), s, c->dev, a, (int)skip_diag);
    else
      LOLA_LAUNCH_CLUSTER(kc_ks_modup<5>, a.count * per, cl_threads<5>(), s, c->dev, a, (int)skip_diag);
    return post_launch(c, s);
  }
  LOLA_DISPATCH_CFG(CfgM, c->logn, kn_ks_modup, a.count * per, s, c->dev, a, (int)skip_diag);
  return post_launch(c, s);
}

int ks_intt_p(Ctx* c, const KsDev& a, cudaStream_t s) {
  ProfScope ps(c, KI_KS_IP_P, s, a.count * 2);
  if ((kClusterMask & 4u) && c->logn == CL_LOGN) {
    if (a.count * 2 < LOLA_CL_SMALL_UNITS)
      LOLA_LAUNCH_CLUSTER(kc_ks_intt_p<4>, a.count * 2, cl_threads<4>(), s, c->dev, a);
    else
      LOLA_LAUNCH_CLUSTER(kc_ks_intt_p<5>, a.count * 2, cl_threads<5>(), s, c->dev, a);
    return post_launch(c, s);
  }
  LOLA_DISPATCH(c->logn, kn_ks_intt_p, a.count * 2, s, c->dev, a);
  return post_launch(c, s);
}

int ks_moddown(Ctx* c, const KsDev& a, cudaStream_t s) {
  ProfScope ps(c, KI_KS_MODDOWN, s, a.count * 2 * c->L);
  if ((kClusterMask & 8u) && c->logn == CL_LOGN) {
    if (a.count * 2 * c->L < LOLA_CL_SMALL_UNITS)
      LOLA_LAUNCH_CLUSTER(kc_ks_moddown<4>, a.count * 2 * c->L, cl_threads<4>(), s, c->dev, a);
    else
      LOLA_LAUNCH_CLUSTER(kc_ks_moddown<5>, a.count * 2 * c->L, cl_threads<5>(), s, c->dev, a);
    return post_launch(c, s);
  }
  LOLA_DISPATCH_CFG(CfgM, c->logn, kn_ks_moddown, a.count * 2 * c->L, s, c->dev, a);
  return post_launch(c, s);
}

}  // namespace k
}  // namespace lola
