// Key-switching transforms, one CTA per limb (any ring degree), and the
// key-switch dispatch, which sends the n = 16384 launches to the 2-CTA
// cluster versions of ntt_cluster.cu.
#include "ntt_common.cuh"

namespace lola {

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

namespace k {
// which key-switch transforms run as 2-CTA clusters at n = 16384 (bit 0
// decompose, 1 mod-up, 2 INTT mod P, 3 mod-down)
#ifndef LOLA_CLUSTER_MASK
#define LOLA_CLUSTER_MASK 0xE
#endif
static constexpr unsigned kClusterMask = LOLA_CLUSTER_MASK;

int ks_decompose(Ctx* c, const KsDev& a, cudaStream_t s) {
  ProfScope ps(c, KI_KS_DECOMPOSE, s, a.count * c->L);
  if ((kClusterMask & 1u) && c->logn == CL_LOGN) {
    return ks_decompose_cluster(c, a, s, a.count * c->L < LOLA_CL_SMALL_UNITS);
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
    return ks_modup_cluster(c, a, skip_diag, s, a.count * per < LOLA_CL_SMALL_UNITS);
  }
  LOLA_DISPATCH_CFG(CfgM, c->logn, kn_ks_modup, a.count * per, s, c->dev, a, (int)skip_diag);
  return post_launch(c, s);
}

int ks_intt_p(Ctx* c, const KsDev& a, cudaStream_t s) {
  ProfScope ps(c, KI_KS_IP_P, s, a.count * 2);
  if ((kClusterMask & 4u) && c->logn == CL_LOGN) {
    return ks_intt_p_cluster(c, a, s, a.count * 2 < LOLA_CL_SMALL_UNITS);
  }
  LOLA_DISPATCH(c->logn, kn_ks_intt_p, a.count * 2, s, c->dev, a);
  return post_launch(c, s);
}

int ks_moddown(Ctx* c, const KsDev& a, cudaStream_t s) {
  ProfScope ps(c, KI_KS_MODDOWN, s, a.count * 2 * c->L);
  if ((kClusterMask & 8u) && c->logn == CL_LOGN) {
    return ks_moddown_cluster(c, a, s, a.count * 2 * c->L < LOLA_CL_SMALL_UNITS);
  }
  LOLA_DISPATCH_CFG(CfgM, c->logn, kn_ks_moddown, a.count * 2 * c->L, s, c->dev, a);
  return post_launch(c, s);
}

}  // namespace k
}  // namespace lola
