// Kernel-side argument structs and the launcher API used by the host code.
#pragma once
#include <stdint.h>

#include "internal.h"

namespace lola {

__device__ __forceinline__ uint32_t brev_n(uint32_t k, int logn) { return __brev(k) >> (32 - logn); }

// NTT position whose value lands at position k under a(x) -> a(x^g): the
// forward transform leaves a(psi^(2 brev(k) + 1)) at position k, and
// tau_g(a)(psi^e) = a(psi^(e g)).
__device__ __forceinline__ uint32_t gal_src(uint32_t k, uint32_t g, int logn) {
  const uint32_t e = 2 * brev_n(k, logn) + 1;
  const uint32_t e2 = (uint32_t)(((uint64_t)e * g) & ((2ull << logn) - 1));
  return brev_n((e2 - 1) >> 1, logn);
}

// Inverse of the map above: the position k whose gal_src is i (ginv = g^-1 mod 2n).
__device__ __forceinline__ uint32_t gal_dst(uint32_t i, uint32_t ginv, int logn) { return gal_src(i, ginv, logn); }

// g^-1 mod 2^32 for odd g (Newton iteration), reduced mod 2n by the caller's mask
__device__ __forceinline__ uint32_t inv_odd32(uint32_t g) {
  uint32_t x = g;
  for (int i = 0; i < 5; ++i) x *= 2u - g * x;
  return x;
}

struct PrimeMap {
  uint8_t p[32];  // limb l of a polynomial uses prime index p[l]
};

// Arguments of the key-switching kernels (one batch of `count` ciphertexts).
struct KsDev {
  const uint64_t* c0;     // comp-0 addend in ciphertext layout, not permuted (relinearisation: e0)
  const uint64_t* c1;     // ciphertext whose c1 is switched (rotation), NTT form
  const uint64_t* add1;   // comp-1 addend (relinearisation: e1 in ciphertext layout) or null
  const uint64_t* accum;  // optional ciphertext added to the result (rotate-and-sum) or null
  uint64_t* out;          // [count][2][L][n]
  uint64_t* dig;          // scratch / input digits [count][L][n] coefficient form
  uint64_t* D;            // scratch [count][L][L+K][n]
  uint64_t* xP;           // scratch [count][2][n]
  uint64_t* acc;          // inner products: ACC(ct, comp, j) = acc + ct * acc_stride + (comp * (L+K) + j) * n
  size_t acc_stride;      // (in place over D's first two digit rows when L >= 2)
  size_t count;
  const uint32_t* d_gal;  // per-entry Galois element or null (use gal)
  uint32_t gal;
  const uint64_t* const* d_keys;  // per-entry key base or null (use key)
  const uint64_t* key;
  uint32_t gal_div;       // ciphertext i uses entry i / gal_div
  // hoisted rotations: entry i reads D and c0 of source ciphertext i % src_mod
  // (0: i) through tau_g in the NTT domain (D and c0 not permuted beforehand)
  uint32_t src_mod;
  uint32_t ip_gather;
  // rotation: the inner product adds tau_g(c0) by gathering c0 itself
  uint32_t c0_gather;
  // rotate-sum (ks_ip_sum): Galois elements per entry; entry e's elements and
  // keys are d_gal / d_keys [e gsum, e gsum + gsum)
  uint32_t gsum;
};

namespace k {
// Modulus switching, one prime (ntt_keyswitch.cu): in [count][2][L1][n] ->
// out [count][2][L1 - 1][n], dropping q_{L1-1}; top: scratch [count][2][n].
// c is the full context.
int mod_switch_drop(Ctx* c, const uint64_t* in, uint64_t* top, uint64_t* out, size_t count, uint32_t L1,
                    cudaStream_t s);
// launch geometry (TuneVariant) the key-switch transform `kernel` (0 decompose,
// 1 mod-up, 2 INTT mod P, 3 mod-down) uses for `units` limb transforms
// without a tuning table (ntt_keyswitch.cu)
int default_geometry(const Ctx* c, int kernel, size_t units);
// NTT family (ntt_kernels.cu)
int ntt_fwd_map(Ctx* c, const uint64_t* in, uint64_t* out, size_t n_limbpolys, uint32_t limbs, const PrimeMap& pm,
                cudaStream_t s);
int ntt_inv_map(Ctx* c, const uint64_t* in, uint64_t* out, size_t n_limbpolys, uint32_t limbs, const PrimeMap& pm,
                bool mont_fix, cudaStream_t s);
int ntt_fwd(Ctx* c, uint64_t* data, size_t n_polys, uint32_t limbs, uint32_t prime0, cudaStream_t s);
int ntt_inv(Ctx* c, uint64_t* data, size_t n_polys, uint32_t limbs, uint32_t prime0, bool mont_fix,
            cudaStream_t s);
int ntt_fwd_from_signed(Ctx* c, const int64_t* in, uint64_t* out, size_t n_polys, uint32_t limbs, uint32_t prime0,
                        cudaStream_t s);
int encode_lift(Ctx* c, const uint64_t* in, const uint32_t* d_tidx, uint64_t* out, size_t n_polys, uint32_t limbs,
                bool mont, cudaStream_t s);
int slots_to_coeff(Ctx* c, const uint64_t* slots, const uint32_t* d_tidx, uint64_t* coeff, size_t n_polys,
                   cudaStream_t s);
int coeff_to_slots(Ctx* c, const uint64_t* coeff, const uint32_t* d_tidx, uint64_t* slots, size_t n_polys,
                   cudaStream_t s);
int enc_msg(Ctx* c, const uint64_t* m, const int64_t* e1, const uint32_t* d_tidx, uint64_t* out, size_t n_polys,
            cudaStream_t s);
int ks_decompose(Ctx* c, const KsDev& a, cudaStream_t s);
int ks_modup(Ctx* c, const KsDev& a, bool skip_diag, cudaStream_t s);
int ks_intt_p(Ctx* c, const KsDev& a, cudaStream_t s);
int ks_moddown(Ctx* c, const KsDev& a, cudaStream_t s);

// element-wise / basis conversion (elem_kernels.cu)
int ks_ip(Ctx* c, const KsDev& a, bool final_out, cudaStream_t s);   // inner product over digits
int ks_ip_sum(Ctx* c, const KsDev& a, bool final_out, cudaStream_t s);   // the same over a rotate-sum's elements
int add(Ctx* c, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t count, cudaStream_t s);
int sub(Ctx* c, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t count, cudaStream_t s);
// mode: MONT_TO x -> x 2^64; MONT_FROM x -> x 2^-64; MONT_FROM_KSK a stored
// switching key back to its plain value (undoes the 2^64 P^-1 factor)
enum { MONT_TO = 0, MONT_FROM = 1, MONT_FROM_KSK = 2 };
int to_mont_map(Ctx* c, uint64_t* data, size_t n_limbpolys, uint32_t limbs, const PrimeMap& pm, cudaStream_t s,
                int mode = MONT_TO);
int axpy_mont_map(Ctx* c, const uint64_t* a, const uint64_t* b, const uint64_t* w_mont, uint64_t* out,
                  size_t n_limbpolys, uint32_t limbs, const PrimeMap& pm, cudaStream_t s);
int neg_axpe(Ctx* c, const uint64_t* a, const uint64_t* s_mont, const uint64_t* e, uint64_t* out, uint32_t limbs,
             cudaStream_t s);
int keygen_switch(Ctx* c, const uint64_t* a, const uint64_t* e, const uint64_t* s_mont, const uint64_t* sfrom,
                  uint64_t* out, cudaStream_t s);
int gal_permute(Ctx* c, const uint64_t* in, uint64_t* out, size_t n_limbpolys, uint32_t g, cudaStream_t s);
// per_msg_in: message r of `in` times plaintext r (else one input for all r)
int mul_plain_multi(Ctx* c, const uint64_t* in, const uint64_t* pt, uint64_t* out, uint32_t R, uint32_t B,
                    cudaStream_t s, bool per_msg_in = false);
// out = (aux or 0) + sum of `msgs` messages of `per` ciphertexts each at src
int sum_msgs(Ctx* c, const uint64_t* src, uint32_t msgs, const uint64_t* aux, uint64_t* out, size_t per,
             cudaStream_t s);
int mac_scalar(Ctx* c, const uint64_t* in, uint32_t R, const uint64_t* w, const uint64_t* ws, uint64_t* out,
               uint32_t maps, uint32_t B, cudaStream_t s);
int lift_q_to_b(Ctx* c, const uint64_t* xq, uint64_t* xb, size_t n_polys, cudaStream_t s);
int tensor(Ctx* c, const uint64_t* xq, const uint64_t* xb, const uint64_t* yq, const uint64_t* yb, uint64_t* T,
           size_t count, cudaStream_t s);
int scale_round(Ctx* c, const uint64_t* T, const uint32_t* d_tidx, uint32_t tidx_div, uint64_t* E, uint64_t* DIG,
                size_t count, cudaStream_t s);
int decrypt_round(Ctx* c, const uint64_t* x, const uint32_t* d_tidx, uint64_t* m, size_t n_polys, cudaStream_t s);
int enc_combine(Ctx* c, const uint64_t* M1, const uint64_t* E2, const uint64_t* U, const uint64_t* pk, uint64_t* out,
                size_t count, cudaStream_t s);
int dec_phase(Ctx* c, const uint64_t* ct, const uint64_t* s_mont, uint64_t* out, size_t count, cudaStream_t s);
}  // namespace k

}  // namespace lola
