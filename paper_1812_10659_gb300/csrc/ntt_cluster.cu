// Thread-block cluster versions of the key-switching transforms at
// n = 16384: one limb transform per cluster of C = 2^LOGC CTAs, each CTA
// holding 1/C of the limb (geometry and launch macro in ntt_common.cuh).
#include "ntt_common.cuh"

namespace lola {

template <int CL_LOGE, int LOGC>
__global__ void __cluster_dims__(1 << LOGC, 1, 1) __launch_bounds__(cl_threads<CL_LOGE, LOGC>(), 2)
    kc_ks_modup(const CtxDev* __restrict__ C, KsDev a, int skip_diag) {
  extern __shared__ uint64_t sm[];
  constexpr int N = 1 << CL_LOGN;
  const int L = C->L, LK = C->L + C->K;
  const int per = skip_diag ? L * (LK - 1) : L * LK;
  const size_t unit = blockIdx.x >> LOGC;
  const size_t ct = unit / per;
  const int r = unit % per;
  const int i = r / (skip_diag ? LK - 1 : LK);
  int j = r % (skip_diag ? LK - 1 : LK);
  if (skip_diag && j >= i) ++j;
  const uint64_t* dig = a.dig + (ct * L + i) * (size_t)N;
  uint64_t* dst = a.D + ((ct * L + i) * LK + j) * (size_t)N;
  const PrimeDev& P = C->pr[j];
  const bool raw = C->modup_raw != 0;
  ncl::ntt_forward_cluster<CL_LOGN, CL_LOGE, LOGC>(sm, C->tw_fwd + (size_t)j * (2u << CL_LOGN), P.q, P.f64,
                                                   [&](int k) { return raw ? dig[k] : reduce64(dig[k], P.q, P.f64); },
                                                   [&](int k, uint64_t v) { dst[k] = v; });
}

template <int CL_LOGE, int LOGC>
__global__ void __cluster_dims__(1 << LOGC, 1, 1) __launch_bounds__(cl_threads<CL_LOGE, LOGC>(), 2)
    kc_ks_intt_p(const CtxDev* __restrict__ C, KsDev a) {
  extern __shared__ uint64_t sm[];
  constexpr int N = 1 << CL_LOGN;
  const int LK = C->L + C->K, ip = C->iP;
  const size_t unit = blockIdx.x >> LOGC;
  const size_t ct = unit >> 1;
  const int comp = unit & 1;
  const PrimeDev& P = C->pr[ip];
  const uint64_t* src = a.acc + ct * a.acc_stride + (size_t)(comp * LK + ip) * N;
  uint64_t* dst = a.xP + (ct * 2 + comp) * (size_t)N;
  ncl::ntt_inverse_cluster<CL_LOGN, CL_LOGE, LOGC>(sm, C->tw_inv + (size_t)ip * (2u << CL_LOGN), P.q, P.ninv,
                                                   P.ninv_s, [&](int k) { return src[k]; },
                                                   [&](int k, uint64_t v) { dst[k] = v; });
}

template <int CL_LOGE, int LOGC>
__global__ void __cluster_dims__(1 << LOGC, 1, 1) __launch_bounds__(cl_threads<CL_LOGE, LOGC>(), 2)
    kc_ks_moddown(const CtxDev* __restrict__ C, KsDev a) {
  extern __shared__ uint64_t sm[];
  constexpr int N = 1 << CL_LOGN;
  const int L = C->L, LK = C->L + C->K;
  const size_t unit = blockIdx.x >> LOGC;
  const size_t ct = unit / (2 * L);
  const int r = unit % (2 * L);
  const int comp = r / L, j = r % L;
  const uint64_t* accp = a.acc + ct * a.acc_stride + (size_t)(comp * LK + j) * N;
  const PrimeDev& P = C->pr[j];
  const uint64_t Phalf = (C->pr[C->iP].q - 1) / 2, q2m1 = 2 * P.q - 1;
  const uint64_t Pinv = C->PinvQ[j], Pinv_s = C->PinvQ_s[j];
  const uint64_t* x = a.xP + (ct * 2 + comp) * (size_t)N;
  uint64_t* dst = a.out + ((ct * 2 + comp) * L + j) * (size_t)N;
  ncl::ntt_forward_cluster<CL_LOGN, CL_LOGE, LOGC>(
      sm, C->tw_fwd + (size_t)j * (2u << CL_LOGN), P.q, P.f64,
      [&](int k) {
        const uint64_t v = x[k];
        return shoup_mul_lazy(v, Pinv, Pinv_s, P.q) + (v > Phalf ? q2m1 : 0);
      },
      ModDownStore{accp, dst, P.q});
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
  const int L = C->L, LK = C->L + C->K;
  const size_t unit = blockIdx.x >> LOGC;
  const size_t ct = unit / L;
  const int i = unit % L;
  const uint32_t g = a.d_gal ? a.d_gal[ct / a.gal_div] : a.gal;
  const uint32_t ginv = inv_odd32(g) & ((2u << CL_LOGN) - 1);
  const int tid = threadIdx.x;
  const uint64_t* src1 = a.c1 + (ct * 2 * L + L + i) * (size_t)N;
  uint64_t* diag = a.D + ((ct * L + i) * LK + i) * (size_t)N;
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
  const uint32_t LK = c->L + c->K;
  const size_t per = skip_diag ? (size_t)c->L * (LK - 1) : (size_t)c->L * LK;
  LOLA_CLUSTER_VARIANTS(kc_ks_modup, a.count * per, s, c->dev, a, (int)skip_diag);
  return post_launch(c, s);
}

int ks_intt_p_cluster(Ctx* c, const KsDev& a, cudaStream_t s, int variant) {
  LOLA_CLUSTER_VARIANTS(kc_ks_intt_p, a.count * 2, s, c->dev, a);
  return post_launch(c, s);
}

int ks_moddown_cluster(Ctx* c, const KsDev& a, cudaStream_t s, int variant) {
  LOLA_CLUSTER_VARIANTS(kc_ks_moddown, a.count * 2 * c->L, s, c->dev, a);
  return post_launch(c, s);
}
}  // namespace k
}  // namespace lola
