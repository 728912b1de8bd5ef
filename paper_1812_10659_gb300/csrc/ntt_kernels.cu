// Plain NTT-family kernels: every kernel here runs one negacyclic transform
// per CTA (ntt.cuh) with a kernel-specific loader (what feeds the transform)
// and storer (what happens to each output word).  Fusing the neighbouring
// element-wise work into the transform's first load / last store is what
// keeps each limb to one HBM read and one HBM write.
#include "ntt_common.cuh"

namespace lola {

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
  if (c->logn == CL_LOGN && n_polys < LOLA_NTT_CL2_UNITS)
    return ntt_fwd_cluster(c, in, out, n_polys, limbs, pm, s,
                           n_polys < LOLA_NTT_CL4_UNITS ? TV_CLUSTER4_16 : TV_CLUSTER16);
  LOLA_DISPATCH_CFG(CfgM, c->logn, kn_fwd, n_polys, s, c->dev, in, out, limbs, pm);
  return post_launch(c, s);
}

int ntt_inv_map(Ctx* c, const uint64_t* in, uint64_t* out, size_t n_polys, uint32_t limbs, const PrimeMap& pm,
                bool mont_fix, cudaStream_t s) {
  if (!n_polys) return LOLA_OK;
  ProfScope ps(c, KI_NTT_INV, s, n_polys);
  if (c->logn == CL_LOGN && n_polys < LOLA_NTT_CL2_UNITS)
    return ntt_inv_cluster(c, in, out, n_polys, limbs, pm, mont_fix, s,
                           n_polys < LOLA_NTT_CL4_UNITS ? TV_CLUSTER4_16 : TV_CLUSTER16);
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

}  // namespace k
}  // namespace lola
