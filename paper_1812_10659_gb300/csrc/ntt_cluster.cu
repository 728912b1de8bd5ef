// Thread-block cluster versions of the key-switching transforms at
// n = 16384: one limb transform per cluster of C = 2^LOGC CTAs, each CTA
// holding 1/C of the limb (geometry and launch macro in ntt_common.cuh).
#include "ntt_common.cuh"

namespace lola {

template <int CL_LOGE, int LOGC, bool GROUPED>
__device__ __forceinline__ void kc_ks_modup_body(const CtxDev* __restrict__ C, const KsDev& a, int skip_diag) {
  extern __shared__ uint64_t sm[];
  constexpr int N = 1 << CL_LOGN;
  const int L = C->L, LK = C->L + C->K, dnum = C->dnum;
  const int per = (int)C->mu_n[skip_diag];
  const size_t unit = blockIdx.x >> LOGC;
  const size_t ct = unit / per;
  const int r = unit % per;
  const int g = C->mu_g[skip_diag][r], j = C->mu_j[skip_diag][r];
  uint64_t* dst = a.D + ((ct * dnum + g) * LK + j) * (size_t)N;
  const PrimeDev& P = C->pr[j];
  ncl::ntt_forward_cluster<CL_LOGN, CL_LOGE, LOGC>(sm, C->tw_fwd + (size_t)j * (2u << CL_LOGN), P.q, P.f64,
                                                   modup_digit<GROUPED>(C, a.dig + ct * L * (size_t)N, g, j, N),
                                                   [&](int k, uint64_t v) { dst[k] = v; });
}

template <int CL_LOGE, int LOGC>
__global__ void __cluster_dims__(1 << LOGC, 1, 1) __launch_bounds__(cl_threads<CL_LOGE, LOGC>(), 2)
    kc_ks_modup(const CtxDev* __restrict__ C, KsDev a, int skip_diag) {
  kc_ks_modup_body<CL_LOGE, LOGC, false>(C, a, skip_diag);
}

template <int CL_LOGE, int LOGC>
__global__ void __cluster_dims__(1 << LOGC, 1, 1) __launch_bounds__(cl_threads<CL_LOGE, LOGC>(), 2)
    kc_ks_modup2(const CtxDev* __restrict__ C, KsDev a, int skip_diag) {
  kc_ks_modup_body<CL_LOGE, LOGC, true>(C, a, skip_diag);
}

template <int CL_LOGE, int LOGC>
__global__ void __cluster_dims__(1 << LOGC, 1, 1) __launch_bounds__(cl_threads<CL_LOGE, LOGC>(), 2)
    kc_ks_intt_p(const CtxDev* __restrict__ C, KsDev a) {
  extern __shared__ uint64_t sm[];
  constexpr int N = 1 << CL_LOGN;
  const int LK = C->L + C->K, K = C->K;
  const size_t unit = blockIdx.x >> LOGC;
  const size_t ct = unit / (2 * K);
  const int r = unit % (2 * K);
  const int comp = r / K, sp = r % K, ip = C->iP + sp;
  const PrimeDev& P = C->pr[ip];
  const uint64_t* src = a.acc + ct * a.acc_stride + (size_t)(comp * LK + ip) * N;
  uint64_t* dst = a.xP + ((ct * 2 + comp) * K + sp) * (size_t)N;
  ncl::ntt_inverse_cluster<CL_LOGN, CL_LOGE, LOGC>(sm, C->tw_inv + (size_t)ip * (2u << CL_LOGN), P.q, P.ninv,
                                                   P.ninv_s, [&](int k) { return src[k]; },
                                                   [&](int k, uint64_t v) { dst[k] = v; });
}

template <int CL_LOGE, int LOGC, bool K2>
__device__ __forceinline__ void kc_ks_moddown_body(const CtxDev* __restrict__ C, const KsDev& a) {
  extern __shared__ uint64_t sm[];
  constexpr int N = 1 << CL_LOGN;
  const int L = C->L, LK = C->L + C->K;
  const size_t unit = blockIdx.x >> LOGC;
  const size_t ct = unit / (2 * L);
  const int r = unit % (2 * L);
  const int comp = r / L, j = r % L;
  const uint64_t* accp = a.acc + ct * a.acc_stride + (size_t)(comp * LK + j) * N;
  const PrimeDev& P = C->pr[j];
  uint64_t* dst = a.out + ((ct * 2 + comp) * L + j) * (size_t)N;
  ncl::ntt_forward_cluster<CL_LOGN, CL_LOGE, LOGC>(sm, C->tw_fwd + (size_t)j * (2u << CL_LOGN), P.q, P.f64,
                                                   moddown_load<K2>(C, a.xP, ct, comp, j, N),
                                                   ModDownStore{accp, dst, P.q});
}

template <int CL_LOGE, int LOGC>
__global__ void __cluster_dims__(1 << LOGC, 1, 1) __launch_bounds__(cl_threads<CL_LOGE, LOGC>(), 2)
    kc_ks_moddown(const CtxDev* __restrict__ C, KsDev a) {
  kc_ks_moddown_body<CL_LOGE, LOGC, false>(C, a);
}

template <int CL_LOGE, int LOGC>
__global__ void __cluster_dims__(1 << LOGC, 1, 1) __launch_bounds__(cl_threads<CL_LOGE, LOGC>(), 2)
    kc_ks_moddown2(const CtxDev* __restrict__ C, KsDev a) {
  kc_ks_moddown_body<CL_LOGE, LOGC, true>(C, a);
}

// Decompose (Galois permutation of c1 limb i, diagonal limb, inverse
// transform into digit i) over a cluster.  tau_g maps each chunk of the
// limb (its top LOGC position bits) onto one chunk: those bits are bits
// 1..LOGC of the odd exponent e = 2 brev(k) + 1, and bits 0..LOGC of e g
// depend only on bits 0..LOGC of e and of g.  So CTA h loads the one source
// chunk whose image is chunk h and scatters into its own shared memory
// only; the transform's last pass is the one exchange.
template <int CL_LOGE, int LOGC>
__global__ void __cluster_dims__(1 << LOGC, 1, 1) __launch_bounds__(cl_threads<CL_LOGE, LOGC>(), 2)
    kc_ks_decompose(const CtxDev* __restrict__ C, KsDev a) {
  extern __shared__ uint64_t sm[];
  namespace cg = cooperative_groups;
  constexpr int N = 1 << CL_LOGN, LOGE = CL_LOGE, LOGNL = CL_LOGN - LOGC, NC = 1 << LOGNL;
  constexpr int T = N >> (LOGE + LOGC);
  const int h = (int)cg::this_cluster().block_rank();
  const int L = C->L, LK = C->L + C->K, dnum = C->dnum;
  const size_t unit = blockIdx.x >> LOGC;
  const size_t ct = unit / L;
  const int i = unit % L;
  const uint32_t g = a.d_gal ? a.d_gal[ct / a.gal_div] : a.gal;
  const uint32_t ginv = inv_odd32(g) & ((2u << CL_LOGN) - 1);
  const int tid = threadIdx.x;
  const uint64_t* src1 = a.c1 + (ct * 2 * L + L + i) * (size_t)N;
  uint64_t* diag = a.D + ((ct * dnum + i / C->alpha) * LK + i) * (size_t)N;
  uint64_t* dig = a.dig + (ct * L + i) * (size_t)N;
  const PrimeDev& P = C->pr[i];
  // the source chunk of this CTA's chunk: that of the first position's source
  const int src_chunk = (int)(gal_src((uint32_t)h << LOGNL, g, CL_LOGN) >> LOGNL);
  uint64_t v[NC / T];
#pragma unroll
  for (int k = 0; k < NC / T; ++k) v[k] = src1[(src_chunk << LOGNL) + tid + k * T];
#pragma unroll
  for (int k = 0; k < NC / T; ++k) {
    const uint32_t d = gal_dst((uint32_t)((src_chunk << LOGNL) + tid + k * T), ginv, CL_LOGN);   // in chunk h
    sm[swz<LOGE>(d & (NC - 1))] = v[k];
  }
  __syncthreads();
#pragma unroll 4
  for (int k = 0; k < NC / T; ++k) {
    const int li = tid + k * T;
    diag[(h << LOGNL) + li] = sm[swz<LOGE>(li)];
  }
  ncl::ntt_inverse_cluster_smem<CL_LOGN, LOGE, LOGC>(sm, C->tw_inv + (size_t)i * (2u << CL_LOGN), P.q, P.ninv,
                                                     P.ninv_s, [&](int k2, uint64_t v2) { dig[k2] = v2; });
}

// Plain forward / inverse transforms over a cluster (small launches at
// n = 16384: a single-request evaluation or a batch of a few ciphertexts,
// where one CTA per limb would leave most SMs idle).  In place is allowed:
// every CTA finishes its global loads before the cluster barrier that
// precedes the first store.
template <int CL_LOGE, int LOGC>
__global__ void __cluster_dims__(1 << LOGC, 1, 1) __launch_bounds__(cl_threads<CL_LOGE, LOGC>(), 2)
    kc_fwd(const CtxDev* __restrict__ C, const uint64_t* in, uint64_t* out, uint32_t limbs, PrimeMap pm) {
  extern __shared__ uint64_t sm[];
  constexpr int N = 1 << CL_LOGN;
  const size_t poly = blockIdx.x >> LOGC;
  const int p = pm.p[poly % limbs];
  const uint64_t* src = in + poly * N;
  uint64_t* dst = out + poly * N;
  ncl::ntt_forward_cluster<CL_LOGN, CL_LOGE, LOGC>(sm, C->tw_fwd + (size_t)p * (2u << CL_LOGN), C->pr[p].q,
                                                   C->pr[p].f64, [&](int i) { return src[i]; },
                                                   [&](int i, uint64_t v) { dst[i] = v; });
}

template <int CL_LOGE, int LOGC>
__global__ void __cluster_dims__(1 << LOGC, 1, 1) __launch_bounds__(cl_threads<CL_LOGE, LOGC>(), 2)
    kc_inv(const CtxDev* __restrict__ C, const uint64_t* in, uint64_t* out, uint32_t limbs, PrimeMap pm,
           int mont_fix) {
  extern __shared__ uint64_t sm[];
  constexpr int N = 1 << CL_LOGN;
  const size_t poly = blockIdx.x >> LOGC;
  const int p = pm.p[poly % limbs];
  const PrimeDev& P = C->pr[p];
  const uint64_t* src = in + poly * N;
  uint64_t* dst = out + poly * N;
  const uint64_t c = mont_fix ? P.ninvr : P.ninv, cs = mont_fix ? P.ninvr_s : P.ninv_s;
  ncl::ntt_inverse_cluster<CL_LOGN, CL_LOGE, LOGC>(sm, C->tw_inv + (size_t)p * (2u << CL_LOGN), P.q, c, cs,
                                                   [&](int i) { return src[i]; },
                                                   [&](int i, uint64_t v) { dst[i] = v; });
}

namespace k {
#define LOLA_CLUSTER_VARIANTS(KERNEL, units, s, ...)                                                       \
  do {                                                                                                     \
    switch (variant) {                                                                                     \
      case TV_CLUSTER16: LOLA_LAUNCH_CLUSTER((KERNEL<4, 1>), 1, units, (cl_threads<4, 1>()), s, __VA_ARGS__); break; \
      case TV_CLUSTER32: LOLA_LAUNCH_CLUSTER((KERNEL<5, 1>), 1, units, (cl_threads<5, 1>()), s, __VA_ARGS__); break; \
      case TV_CLUSTER4_16: LOLA_LAUNCH_CLUSTER((KERNEL<4, 2>), 2, units, (cl_threads<4, 2>()), s, __VA_ARGS__); break; \
      default: return fail(LOLA_E_PARAM, "unknown cluster geometry");                                     \
    }                                                                                                      \
  } while (0)

int ks_decompose_cluster(Ctx* c, const KsDev& a, cudaStream_t s, int variant) {
  LOLA_CLUSTER_VARIANTS(kc_ks_decompose, a.count * c->L, s, c->dev, a);
  return post_launch(c, s);
}

int ks_modup_cluster(Ctx* c, const KsDev& a, bool skip_diag, cudaStream_t s, int variant) {
  const size_t per = c->host.mu_n[skip_diag ? 1 : 0];
  if (c->alpha > 1)
    LOLA_CLUSTER_VARIANTS(kc_ks_modup2, a.count * per, s, c->dev, a, (int)skip_diag);
  else
    LOLA_CLUSTER_VARIANTS(kc_ks_modup, a.count * per, s, c->dev, a, (int)skip_diag);
  return post_launch(c, s);
}

int ks_intt_p_cluster(Ctx* c, const KsDev& a, cudaStream_t s, int variant) {
  LOLA_CLUSTER_VARIANTS(kc_ks_intt_p, a.count * 2 * c->K, s, c->dev, a);
  return post_launch(c, s);
}

int ntt_fwd_cluster(Ctx* c, const uint64_t* in, uint64_t* out, size_t n_polys, uint32_t limbs, const PrimeMap& pm,
                    cudaStream_t s, int variant) {
  LOLA_CLUSTER_VARIANTS(kc_fwd, n_polys, s, c->dev, in, out, limbs, pm);
  return post_launch(c, s);
}

int ntt_inv_cluster(Ctx* c, const uint64_t* in, uint64_t* out, size_t n_polys, uint32_t limbs, const PrimeMap& pm,
                    bool mont_fix, cudaStream_t s, int variant) {
  LOLA_CLUSTER_VARIANTS(kc_inv, n_polys, s, c->dev, in, out, limbs, pm, (int)mont_fix);
  return post_launch(c, s);
}

int ks_moddown_cluster(Ctx* c, const KsDev& a, cudaStream_t s, int variant) {
  if (c->K > 1)
    LOLA_CLUSTER_VARIANTS(kc_ks_moddown2, a.count * 2 * c->L, s, c->dev, a);
  else
    LOLA_CLUSTER_VARIANTS(kc_ks_moddown, a.count * 2 * c->L, s, c->dev, a);
  return post_launch(c, s);
}
}  // namespace k
}  // namespace lola
