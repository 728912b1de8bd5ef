// Key-switching transforms, one CTA per limb (any ring degree), and the
// key-switch dispatch, which sends the n = 16384 launches to the 2-CTA
// cluster versions of ntt_cluster.cu.
#include "ntt_common.cuh"

namespace lola {

// ------------------------------------------------------------- key switching
// A: the Galois automorphism in NTT form is a permutation of positions.
//    Load c1 limb i coalesced and scatter it through the inverse permutation
//    into shared memory; write the permuted limb (the diagonal block D[i][i])
//    back coalesced; inverse-transform it into digit i.  (tau_g(c0) is
//    never materialised: the inner product gathers it.)
template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::T) kn_ks_decompose(const CtxDev* __restrict__ C, KsDev a) {
  extern __shared__ uint64_t sm[];
  constexpr int N = Cfg<LOGN>::N, T = Cfg<LOGN>::T, LOGE = Cfg<LOGN>::LOGE;
  const int L = C->L, LK = C->L + C->K, dnum = C->dnum;
  const size_t ct = blockIdx.x / L;
  const int i = blockIdx.x % L;
  const uint32_t g = a.d_gal ? a.d_gal[ct / a.gal_div] : a.gal;
  const uint32_t ginv = inv_odd32(g) & ((2u << LOGN) - 1);
  const int tid = threadIdx.x;
  const uint64_t* src1 = a.c1 + (ct * 2 * L + L + i) * (size_t)N;
  uint64_t* diag = a.D + ((ct * dnum + i / C->alpha) * LK + i) * (size_t)N;
  uint64_t* dig = a.dig + (ct * L + i) * (size_t)N;
  const PrimeDev& P = C->pr[i];
  uint64_t v[N / T];
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

// B: digit g (one or two primes) reduced mod prime j, forward transform -> D[g][j]
template <int LOGN, bool GROUPED>
__device__ __forceinline__ void ks_modup_body(const CtxDev* __restrict__ C, const KsDev& a, int skip_diag) {
  extern __shared__ uint64_t sm[];
  constexpr int N = CfgM<LOGN>::N;
  const int L = C->L, LK = C->L + C->K, dnum = C->dnum;
  const int per = (int)C->mu_n[skip_diag];
  const size_t ct = blockIdx.x / per;
  const int r = blockIdx.x % per;
  const int g = C->mu_g[skip_diag][r], j = C->mu_j[skip_diag][r];
  uint64_t* dst = a.D + ((ct * dnum + g) * LK + j) * (size_t)N;
  const PrimeDev& P = C->pr[j];
  ntt_forward<LOGN, CfgM<LOGN>::LOGE>(sm, TW_F(C, j), P.q, P.f64,
                                      modup_digit<GROUPED>(C, a.dig + ct * L * (size_t)N, g, j, N),
                                      [&](int k, uint64_t v) { dst[k] = v; });
}

template <int LOGN>
__global__ void __launch_bounds__(CfgM<LOGN>::T) kn_ks_modup(const CtxDev* __restrict__ C, KsDev a, int skip_diag) {
  ks_modup_body<LOGN, false>(C, a, skip_diag);
}

template <int LOGN>
__global__ void __launch_bounds__(CfgM<LOGN>::T) kn_ks_modup2(const CtxDev* __restrict__ C, KsDev a, int skip_diag) {
  ks_modup_body<LOGN, true>(C, a, skip_diag);
}

// D: inverse transform of the special-prime inner products (both components,
//    each special prime) into x_P [ct][2][K][n]
template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::T) kn_ks_intt_p(const CtxDev* __restrict__ C, KsDev a) {
  extern __shared__ uint64_t sm[];
  constexpr int N = Cfg<LOGN>::N;
  const int LK = C->L + C->K, K = C->K;
  const size_t ct = blockIdx.x / (2 * K);
  const int r = blockIdx.x % (2 * K);
  const int comp = r / K, sp = r % K, ip = C->iP + sp;
  const PrimeDev& P = C->pr[ip];
  const uint64_t* src = a.acc + ct * a.acc_stride + (size_t)(comp * LK + ip) * N;
  uint64_t* dst = a.xP + ((ct * 2 + comp) * K + sp) * (size_t)N;
  ntt_inverse<LOGN, Cfg<LOGN>::LOGE>(sm, TW_I(C, ip), P.q, P.ninv, P.ninv_s, [&](int k) { return src[k]; },
                                      [&](int k, uint64_t v) { dst[k] = v; });
}


// E: output limb out[comp][j] = ACC'[comp][j] - NTT(x~ P^-1 mod q_j), with
//    x~ = centered(x mod P); the inner-product kernel left ACC' = ACC P^-1 +
//    addend + accumulator (the keys carry P^-1).  The loader (ModDownLoad)
//    forms x~ P^-1 mod q_j from the special-prime limbs in coefficient form;
//    its value stays below 6q, which the forward butterflies accept.
template <int LOGN, bool K2>
__device__ __forceinline__ void ks_moddown_body(const CtxDev* __restrict__ C, const KsDev& a) {
  extern __shared__ uint64_t sm[];
  constexpr int N = CfgM<LOGN>::N;
  const int L = C->L, LK = C->L + C->K;
  const size_t ct = blockIdx.x / (2 * L);
  const int r = blockIdx.x % (2 * L);
  const int comp = r / L, j = r % L;
  const uint64_t* accp = a.acc + ct * a.acc_stride + (size_t)(comp * LK + j) * N;
  const PrimeDev& P = C->pr[j];
  uint64_t* dst = a.out + ((ct * 2 + comp) * L + j) * (size_t)N;
  ntt_forward<LOGN, CfgM<LOGN>::LOGE>(sm, TW_F(C, j), P.q, P.f64, moddown_load<K2>(C, a.xP, ct, comp, j, N),
                                      ModDownStore{accp, dst, P.q});
}

template <int LOGN>
__global__ void __launch_bounds__(CfgM<LOGN>::T) kn_ks_moddown(const CtxDev* __restrict__ C, KsDev a) {
  ks_moddown_body<LOGN, false>(C, a);
}

template <int LOGN>
__global__ void __launch_bounds__(CfgM<LOGN>::T) kn_ks_moddown2(const CtxDev* __restrict__ C, KsDev a) {
  ks_moddown_body<LOGN, true>(C, a);
}

// Modulus switching (drop q_l, l = L1 - 1, from ciphertexts of L1 primes):
// F: inverse transform of limb l of each component into coefficients.
template <int LOGN>
__global__ void __launch_bounds__(Cfg<LOGN>::T) kn_ms_top(const CtxDev* __restrict__ C, const uint64_t* __restrict__ in,
                                                         uint64_t* __restrict__ top, int L1) {
  extern __shared__ uint64_t sm[];
  constexpr int N = Cfg<LOGN>::N;
  const int l = L1 - 1;
  const size_t cp = blockIdx.x;   // (ciphertext, component)
  const PrimeDev& P = C->pr[l];
  const uint64_t* src = in + (cp * L1 + l) * (size_t)N;
  uint64_t* dst = top + cp * (size_t)N;
  ntt_inverse<LOGN, Cfg<LOGN>::LOGE>(sm, TW_I(C, l), P.q, P.ninv, P.ninv_s, [&](int k) { return src[k]; },
                                      [&](int k, uint64_t v) { dst[k] = v; });
}

// G: out limb j < l = (c_j - NTT_j(x~)) q_l^-1 = c_j q_l^-1 - NTT_j(x~ q_l^-1),
//    x~ = centered(x mod q_l).  The loader forms x~ q_l^-1 mod q_j from the
//    raw x in [0, q_l) as mod-down does (x q_l^-1, minus 1 = q_l q_l^-1 when
//    x > (q_l - 1) / 2); the storer fetches c_j ahead of its stores.
struct MsConst {
  uint64_t inv[MAXL], inv_s[MAXL];   // q_l^-1 mod q_j and its Shoup companion
};
struct MsStore {
  const uint64_t* c;
  uint64_t* dst;
  uint64_t q, w, ws;
  __device__ __forceinline__ uint64_t fetch(int k) const { return c[k]; }
  __device__ __forceinline__ void operator()(int k, uint64_t v, uint64_t f) const {
    dst[k] = sub_mod(shoup_mul(f, w, ws, q), v, q);
  }
};

template <int LOGN>
__global__ void __launch_bounds__(CfgM<LOGN>::T) kn_ms_down(const CtxDev* __restrict__ C, const uint64_t* __restrict__ in,
                                                           const uint64_t* __restrict__ top, uint64_t* __restrict__ out,
                                                           int L1, MsConst mc) {
  extern __shared__ uint64_t sm[];
  constexpr int N = CfgM<LOGN>::N;
  const int l = L1 - 1;
  const size_t cp = blockIdx.x / l;
  const int j = blockIdx.x % l;
  const PrimeDev& P = C->pr[j];
  const uint64_t half = (C->pr[l].q - 1) / 2, q2m1 = 2 * P.q - 1;
  const uint64_t w = mc.inv[j], ws = mc.inv_s[j];
  const uint64_t* x = top + cp * (size_t)N;
  ntt_forward<LOGN, CfgM<LOGN>::LOGE>(
      sm, TW_F(C, j), P.q, P.f64,
      [&](int k) {
        const uint64_t v = x[k];
        return shoup_mul_lazy(v, w, ws, P.q) + (v > half ? q2m1 : 0);
      },
      MsStore{in + (cp * L1 + j) * (size_t)N, out + (cp * l + j) * (size_t)N, P.q, w, ws});
}

namespace k {
int mod_switch_drop(Ctx* c, const uint64_t* in, uint64_t* top, uint64_t* out, size_t count, uint32_t L1,
                    cudaStream_t s) {
  if (L1 < 2 || L1 > c->L) return fail(LOLA_E_PARAM, "mod switch: bad level");
  if (!count) return LOLA_OK;
  const uint32_t l = L1 - 1;
  MsConst mc{};
  const uint64_t ql = c->primes[l];
  for (uint32_t j = 0; j < l; ++j) {
    const uint64_t q = c->primes[j];
    mc.inv[j] = invmod_h(ql % q, q);
    mc.inv_s[j] = shoup_h(mc.inv[j], q);
  }
  {
    ProfScope ps(c, KI_MOD_SWITCH, s, count * 2);
    LOLA_DISPATCH(c->logn, kn_ms_top, count * 2, s, c->dev, in, top, (int)L1);
    const int rc = post_launch(c, s);
    if (rc != LOLA_OK) return rc;
  }
  ProfScope ps(c, KI_MOD_SWITCH, s, count * 2 * l);
  LOLA_DISPATCH_CFG(CfgM, c->logn, kn_ms_down, count * 2 * l, s, c->dev, in, top, out, (int)L1, mc);
  return post_launch(c, s);
}

// which key-switch transforms run as 2-CTA clusters at n = 16384 (bit 0
// decompose, 1 mod-up, 2 INTT mod P, 3 mod-down)
#ifndef LOLA_CLUSTER_MASK
#define LOLA_CLUSTER_MASK 0xE
#endif
static constexpr unsigned kClusterMask = LOLA_CLUSTER_MASK;

// the library's default geometry: clusters at n = 16384 for the kernels in
// kClusterMask, with 16 words per thread below LOLA_CL_SMALL_UNITS
int default_geometry(const Ctx* c, int kernel, size_t units) {
  if (c->logn != CL_LOGN || !(kClusterMask & (1u << kernel))) return TV_CTA;
  return units < LOLA_CL_SMALL_UNITS ? TV_CLUSTER16 : TV_CLUSTER32;
}

// geometry of one launch: the tuned table, else the default
static int geometry(const Ctx* c, int kernel, size_t units) {
  if (c->logn != CL_LOGN) return TV_CTA;
  const Tune& t = c->root->tune;
  if (t.on) return t.v[kernel][tune_bucket(units)];
  return default_geometry(c, kernel, units);
}

int ks_decompose(Ctx* c, const KsDev& a, cudaStream_t s) {
  const size_t units = a.count * c->L;
  ProfScope ps(c, KI_KS_DECOMPOSE, s, units);
  const int g = geometry(c, 0, units);
  if (g != TV_CTA) return ks_decompose_cluster(c, a, s, g);
  LOLA_DISPATCH(c->logn, kn_ks_decompose, units, s, c->dev, a);
  return post_launch(c, s);
}

int ks_modup(Ctx* c, const KsDev& a, bool skip_diag, cudaStream_t s) {
  const size_t per = c->host.mu_n[skip_diag ? 1 : 0];
  if (!per) return LOLA_OK;
  const size_t units = a.count * per;
  ProfScope ps(c, KI_KS_MODUP, s, units);
  const int g = geometry(c, 1, units);
  if (g != TV_CTA) return ks_modup_cluster(c, a, skip_diag, s, g);
  if (c->alpha > 1)
    LOLA_DISPATCH_CFG(CfgM, c->logn, kn_ks_modup2, units, s, c->dev, a, (int)skip_diag);
  else
    LOLA_DISPATCH_CFG(CfgM, c->logn, kn_ks_modup, units, s, c->dev, a, (int)skip_diag);
  return post_launch(c, s);
}

int ks_intt_p(Ctx* c, const KsDev& a, cudaStream_t s) {
  const size_t units = a.count * 2 * c->K;
  ProfScope ps(c, KI_KS_IP_P, s, units);
  const int g = geometry(c, 2, units);
  if (g != TV_CTA) return ks_intt_p_cluster(c, a, s, g);
  LOLA_DISPATCH(c->logn, kn_ks_intt_p, units, s, c->dev, a);
  return post_launch(c, s);
}

int ks_moddown(Ctx* c, const KsDev& a, cudaStream_t s) {
  const size_t units = a.count * 2 * c->L;
  ProfScope ps(c, KI_KS_MODDOWN, s, units);
  const int g = geometry(c, 3, units);
  if (g != TV_CTA) return ks_moddown_cluster(c, a, s, g);
  if (c->K > 1)
    LOLA_DISPATCH_CFG(CfgM, c->logn, kn_ks_moddown2, units, s, c->dev, a);
  else
    LOLA_DISPATCH_CFG(CfgM, c->logn, kn_ks_moddown, units, s, c->dev, a);
  return post_launch(c, s);
}

}  // namespace k
}  // namespace lola
