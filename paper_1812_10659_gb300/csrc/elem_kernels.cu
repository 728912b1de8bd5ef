// Element-wise kernels (HBM-bound) and exact RNS basis conversions.
//
// Ciphertext words are addressed as [ct][comp][limb][n]; the prime of a word
// is its limb index in the ciphertext basis.  All kernels are grid-stride
// loops over words (or over coefficient positions for the basis
// conversions, which need every limb of one coefficient at once).
#include <type_traits>

#include "internal.h"
#include "kernels.h"
#include "mac.cuh"

namespace lola {

static int post(Ctx* c) {
  c->root->launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LOLA_E_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return LOLA_OK;
}

static unsigned grid_for(size_t items, int threads) {
  size_t g = (items + threads - 1) / threads;
  const size_t cap = 152 * 16;   // enough CTAs to fill every SM several times
  return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

// ------------------------------------------------------------- key switching

// Inner product over the digits, both key components at once:
//   ACC[comp][j] = sum_i D[i][j] * key[comp][i][j]   (keys are Montgomery-scaled)
// Products are summed in 128 bits and reduced once (every 8 terms: 8 q^2 < q 2^64
// for q < 2^61).  Each thread owns two adjacent coefficients of one (ct, j).
// final_out (K = 0): write the switched ciphertext limb directly, plus addends.
// Otherwise write ACC; the caller may place ACC over D's digit rows 0 and 1:
// a thread reads every D word it overwrites before writing it.
// Hoisted rotations (ip_gather): D and c0 are those of the unrotated source
// ciphertext ct % src_mod; position k of tau_g(D) is D[gal_src(k)], and the
// pair (k, k+1) maps to the aligned pair holding gal_src(k) and
// gal_src(k) ^ 1, so each pair is still one 16-byte load (swapped when
// gal_src(k) is odd).
// DT > 0: the digit count as a compile-time constant (fully unrolled digit
// loop, all loads of a thread issued together); 0: read it from the context.
// Digits: one per ciphertext prime, or one per group of alpha primes (D is
// [ct][digits][L+K][n]; key row g of component c at (c kdnum + g) kLK).
// At most 64 registers, so that 32 warps per SM keep loads in flight.
template <int DT>
__global__ void __launch_bounds__(256, 4) ke_ks_ip(const CtxDev* __restrict__ C, KsDev a, int final_out) {
  const int L = C->L, LK = L + C->K, logn = C->logn;
  const int dn = DT > 0 ? DT : (int)C->dnum;
  const size_t n = C->n, half = n >> 1;
  const int J = final_out ? L : LK;
  const size_t total = a.count * J * half;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t k = 2 * (w % half);
    const size_t r = w / half;
    const int j = r % J;
    const size_t ct = r / J;
    const PrimeDev& P = C->pr[j];
    const uint64_t* key = a.d_keys ? a.d_keys[ct / a.gal_div] : a.key;
    // the keys have kL digits over kL + K primes (the full context's): prime
    // j of this context is key prime j, the special primes follow kL
    const size_t kLK = C->kLK, jk = j < L ? (size_t)j : (size_t)C->kL + (j - L);
    const size_t krow1 = (size_t)C->kdnum * kLK;
    const size_t src = a.src_mod ? ct % a.src_mod : ct;
    size_t kd = k;                                // gathered pair of tau_g (D and/or c0)
    bool swp = false;
    const bool gather_c0 = a.ip_gather || a.c0_gather;
    if (gather_c0) {
      const uint32_t g = a.d_gal ? a.d_gal[ct / a.gal_div] : a.gal;
      const uint32_t m = gal_src((uint32_t)k, g, logn);
      kd = m & ~1u;
      swp = (m & 1u) != 0;
    }
    const size_t kD = a.ip_gather ? kd : k;
    const bool swpD = a.ip_gather && swp;
    uint64_t acc0[2] = {0, 0}, acc1[2] = {0, 0};
    unsigned __int128 s0[2] = {0, 0}, s1[2] = {0, 0};
#pragma unroll
    for (int i = 0; i < (DT > 0 ? DT : dn); ++i) {
      ulonglong2 d = *(const ulonglong2*)(a.D + ((src * dn + i) * LK + j) * n + kD);
      if (swpD) d = make_ulonglong2(d.y, d.x);
      const ulonglong2 k0 = __ldg((const ulonglong2*)(key + ((size_t)i * kLK + jk) * n + k));
      const ulonglong2 k1 = __ldg((const ulonglong2*)(key + (krow1 + (size_t)i * kLK + jk) * n + k));
      s0[0] += (unsigned __int128)d.x * k0.x;
      s0[1] += (unsigned __int128)d.y * k0.y;
      s1[0] += (unsigned __int128)d.x * k1.x;
      s1[1] += (unsigned __int128)d.y * k1.y;
      if ((i & 7) == 7 || i == dn - 1) {
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          acc0[e] = add_mod(acc0[e], redc128(s0[e], P.q, P.qinv), P.q);
          acc1[e] = add_mod(acc1[e], redc128(s1[e], P.q, P.qinv), P.q);
          s0[e] = s1[e] = 0;
        }
      }
    }
    if (final_out) {
      uint64_t* o0 = a.out + ((ct * 2 + 0) * L + j) * n;
      uint64_t* o1 = a.out + ((ct * 2 + 1) * L + j) * n;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const size_t kk = k + e;
        uint64_t v0 = acc0[e], v1 = acc1[e];
        if (gather_c0) v0 = add_mod(v0, a.c0[(src * 2 * L + j) * n + (kd + (e ^ (int)swp))], P.q);
        else if (a.c0) v0 = add_mod(v0, a.c0[(ct * 2 * L + j) * n + kk], P.q);
        if (a.add1) v1 = add_mod(v1, a.add1[(ct * 2 * L + L + j) * n + kk], P.q);
        if (a.accum) {
          v0 = add_mod(v0, a.accum[((ct * 2 + 0) * L + j) * n + kk], P.q);
          v1 = add_mod(v1, a.accum[((ct * 2 + 1) * L + j) * n + kk], P.q);
        }
        o0[kk] = v0;
        o1[kk] = v1;
      }
    } else {
      if (j < L) {
        // the keys carry P^-1 on these primes, so ACC here is already the
        // inner product times P^-1; fold the addends:
        //   out = ACC P^-1 + addend + accum - NTT(x~) P^-1
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const size_t kk = k + e;
          uint64_t s0v = 0, s1v = 0;
          if (gather_c0) s0v = a.c0[(src * 2 * L + j) * n + (kd + (e ^ (int)swp))];
          else if (a.c0) s0v = a.c0[(ct * 2 * L + j) * n + kk];
          if (a.add1) s1v = a.add1[(ct * 2 * L + L + j) * n + kk];
          if (a.accum) {
            s0v = add_mod(s0v, a.accum[((ct * 2 + 0) * L + j) * n + kk], P.q);
            s1v = add_mod(s1v, a.accum[((ct * 2 + 1) * L + j) * n + kk], P.q);
          }
          acc0[e] = add_mod(acc0[e], s0v, P.q);
          acc1[e] = add_mod(acc1[e], s1v, P.q);
        }
      }
      uint64_t* A0 = a.acc + ct * a.acc_stride + (size_t)j * n + k;
      uint64_t* A1 = a.acc + ct * a.acc_stride + (size_t)(LK + j) * n + k;
      *(ulonglong2*)A0 = make_ulonglong2(acc0[0], acc0[1]);
      *(ulonglong2*)A1 = make_ulonglong2(acc1[0], acc1[1]);
    }
  }
}

// Inner product of a rotate-sum (x plus its rotations by G Galois elements,
// one key switch): D holds the raised digits of x's own c1 (decomposed
// without an automorphism).  For every element g of the entry the digits are
// gathered through tau_g as in the hoisted rotations and multiplied by g's
// key; all G * digits products go into one inner product mod q_j, so the one
// mod-down that follows rounds once.  The addends are x itself (a.accum: c0
// and c1) and tau_g(c0) of every element.  Entry
// ct / gal_div uses elements and keys [e G, e G + G) of d_gal / d_keys.
// ACC must not overlap D: other threads gather D words at any position.
// The digit and key words are below q (mod-up and key generation reduce
// them), so each product is below q^2.  Up to 128 registers (the gathered
// and key loads of all digits are issued together; at 64 they spill).
template <int DT>
__global__ void __launch_bounds__(256, 2) ke_ks_ip_sum(const CtxDev* __restrict__ C, KsDev a, int final_out) {
  const int L = C->L, LK = L + C->K, logn = C->logn;
  const int dn = DT > 0 ? DT : (int)C->dnum;
  const int G = (int)a.gsum;
  const size_t n = C->n, half = n >> 1;
  const int J = final_out ? L : LK;
  const size_t total = a.count * J * half;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t k = 2 * (w % half);
    const size_t r = w / half;
    const int j = r % J;
    const size_t ct = r / J;
    const PrimeDev& P = C->pr[j];
    const size_t kLK = C->kLK, jk = j < L ? (size_t)j : (size_t)C->kL + (j - L);
    const size_t krow1 = (size_t)C->kdnum * kLK;
    const size_t e0 = (ct / a.gal_div) * (size_t)G;
    // one 128-bit sum (hi:lo) per component and coefficient over all G x
    // digits products, kept below q 2^64 by subtracting q from hi after every
    // digit group of at most 8 products (each below q^2, 8 q < 2^64), then
    // one REDC: the same residue as reducing every element on its own
    uint64_t lo0[2] = {0, 0}, hi0[2] = {0, 0}, lo1[2] = {0, 0}, hi1[2] = {0, 0}, c0s[2] = {0, 0};
    for (int gi = 0; gi < G; ++gi) {
      const uint64_t* key = a.d_keys[e0 + gi];
      const uint32_t m = gal_src((uint32_t)k, a.d_gal[e0 + gi], logn);
      const size_t kd = m & ~1u;                  // the aligned pair holding m (swapped when m is odd)
      const bool swp = (m & 1u) != 0;
#pragma unroll
      for (int i = 0; i < (DT > 0 ? DT : dn); ++i) {
        const ulonglong2 dv = *(const ulonglong2*)(a.D + ((ct * dn + i) * LK + j) * n + kd);
        const ulonglong2 k0 = __ldg((const ulonglong2*)(key + ((size_t)i * kLK + jk) * n + k));
        const ulonglong2 k1 = __ldg((const ulonglong2*)(key + (krow1 + (size_t)i * kLK + jk) * n + k));
        const uint64_t d0 = swp ? dv.y : dv.x, d1 = swp ? dv.x : dv.y;
        mac128(lo0[0], hi0[0], d0, k0.x);
        mac128(lo0[1], hi0[1], d1, k0.y);
        mac128(lo1[0], hi1[0], d0, k1.x);
        mac128(lo1[1], hi1[1], d1, k1.y);
        if ((i & 7) == 7 || i == dn - 1) {
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            hi0[e] = csub(hi0[e], P.q);
            hi1[e] = csub(hi1[e], P.q);
          }
        }
      }
      if (j < L) {
        const ulonglong2 cg = *(const ulonglong2*)(a.c0 + (ct * 2 * L + j) * n + kd);
        c0s[0] = add_mod(c0s[0], swp ? cg.y : cg.x, P.q);
        c0s[1] = add_mod(c0s[1], swp ? cg.x : cg.y, P.q);
      }
    }
    uint64_t acc0[2], acc1[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      acc0[e] = redc128(((unsigned __int128)hi0[e] << 64) | lo0[e], P.q, P.qinv);
      acc1[e] = redc128(((unsigned __int128)hi1[e] << 64) | lo1[e], P.q, P.qinv);
    }
    if (j < L) {
      // x itself and the gathered tau_g(c0); on the ciphertext primes the
      // keys carry P^-1, so ACC + addends is what the mod-down expects
      const ulonglong2 x0 = *(const ulonglong2*)(a.accum + ((ct * 2 + 0) * L + j) * n + k);
      const ulonglong2 x1 = *(const ulonglong2*)(a.accum + ((ct * 2 + 1) * L + j) * n + k);
      acc0[0] = add_mod(add_mod(acc0[0], c0s[0], P.q), x0.x, P.q);
      acc0[1] = add_mod(add_mod(acc0[1], c0s[1], P.q), x0.y, P.q);
      acc1[0] = add_mod(acc1[0], x1.x, P.q);
      acc1[1] = add_mod(acc1[1], x1.y, P.q);
    }
    if (final_out) {
      *(ulonglong2*)(a.out + ((ct * 2 + 0) * L + j) * n + k) = make_ulonglong2(acc0[0], acc0[1]);
      *(ulonglong2*)(a.out + ((ct * 2 + 1) * L + j) * n + k) = make_ulonglong2(acc1[0], acc1[1]);
    } else {
      *(ulonglong2*)(a.acc + ct * a.acc_stride + (size_t)j * n + k) = make_ulonglong2(acc0[0], acc0[1]);
      *(ulonglong2*)(a.acc + ct * a.acc_stride + (size_t)(LK + j) * n + k) = make_ulonglong2(acc1[0], acc1[1]);
    }
  }
}

// ------------------------------------------------------------- element-wise
// words of a batch of ciphertexts; limb = (w / n) % L
// out = (aux ? aux : 0) + sum of `msgs` blocks of `total` words at src, src + total, ...
__global__ void ke_sum_msgs(const CtxDev* __restrict__ C, const uint64_t* src, uint32_t msgs, const uint64_t* aux,
                            uint64_t* out, size_t total) {
  const int L = C->L, logn = C->logn;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const uint64_t q = C->pr[(w >> logn) % L].q;
    uint64_t acc = aux ? aux[w] : 0;
    for (uint32_t m = 0; m < msgs; ++m) acc = add_mod(acc, src[(size_t)m * total + w], q);
    out[w] = acc;
  }
}

__global__ void ke_add(const CtxDev* __restrict__ C, const uint64_t* a, const uint64_t* b, uint64_t* out,
                       size_t total, int sub) {
  const int L = C->L, logn = C->logn;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const uint64_t q = C->pr[(w >> logn) % L].q;
    out[w] = sub ? sub_mod(a[w], b[w], q) : add_mod(a[w], b[w], q);
  }
}

// x -> x * 2^64 mod q per limb of [poly][limbs][n]
// (inverse = true: x -> x * 2^-64 mod q)
__global__ void ke_to_mont(const CtxDev* __restrict__ C, uint64_t* x, size_t total, uint32_t limbs, PrimeMap pm,
                           int mode) {
  const int logn = C->logn;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const int pi = pm.p[(w >> logn) % limbs];
    const PrimeDev& P = C->pr[pi];
    x[w] = mont_mul(x[w], mode == k::MONT_TO ? P.r2 : mode == k::MONT_FROM ? 1 : C->KskOut[pi], P.q, P.qinv);
  }
}

// out = a + b * w (w in Montgomery form, one [limbs][n] block broadcast over polys)
__global__ void ke_axpy_mont(const CtxDev* __restrict__ C, const uint64_t* a, const uint64_t* b, const uint64_t* w,
                             uint64_t* out, size_t total, uint32_t limbs, PrimeMap pm) {
  const int logn = C->logn;
  const size_t blk = (size_t)limbs << logn;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const PrimeDev& P = C->pr[pm.p[(i >> logn) % limbs]];
    const uint64_t v = mont_mul(b[i], w[i % blk], P.q, P.qinv);
    out[i] = a ? add_mod(a[i], v, P.q) : v;
  }
}

// out = -(a * s + e) per limb (public key): s in Montgomery form
__global__ void ke_neg_axpe(const CtxDev* __restrict__ C, const uint64_t* a, const uint64_t* s_mont,
                            const uint64_t* e, uint64_t* out, size_t total) {
  const int logn = C->logn;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const PrimeDev& P = C->pr[i >> logn];
    out[i] = neg_mod(add_mod(mont_mul(a[i], s_mont[i], P.q, P.qinv), e[i], P.q), P.q);
  }
}

// switching key rows: a, e: [L][LK][n] (e broadcast per digit over primes),
// out: [2][L][LK][n] Montgomery form of (b, a) times P^-1 on the ciphertext primes,
// b_ij = -a_ij s_j + e_ij + [i == j] (P mod q_j) s'_j
__global__ void ke_keygen_switch(const CtxDev* __restrict__ C, const uint64_t* a, const uint64_t* e,
                                 const uint64_t* s_mont, const uint64_t* sfrom, uint64_t* out) {
  const int L = C->L, LK = C->L + C->K, logn = C->logn;
  const size_t n = C->n;
  const size_t total = (size_t)C->dnum * LK * n;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t k = w & (n - 1);
    const int j = (w >> logn) % LK;
    const int g = (int)((w >> logn) / LK);
    const PrimeDev& P = C->pr[j];
    uint64_t b = neg_mod(mont_mul(a[w], s_mont[(size_t)j * n + k], P.q, P.qinv), P.q);
    b = add_mod(b, e[w], P.q);
    // [P]_{q_j} s' on the primes of digit g's group
    if (j < L && j / (int)C->alpha == g)
      b = add_mod(b, mont_mul(sfrom[(size_t)j * n + k], C->PmontQ[j], P.q, P.qinv), P.q);
    out[w] = mont_mul(b, C->KskR2[j], P.q, P.qinv);
    out[total + w] = mont_mul(a[w], C->KskR2[j], P.q, P.qinv);
  }
}

// NTT-domain Galois permutation of [poly][limbs][n]
__global__ void ke_gal_permute(const CtxDev* __restrict__ C, const uint64_t* in, uint64_t* out, size_t total,
                               uint32_t g) {
  const int logn = C->logn;
  const size_t n = C->n;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t base = w & ~(n - 1);
    out[w] = in[base + gal_src((uint32_t)(w & (n - 1)), g, logn)];
  }
}

// ct x plaintext for R plaintexts at once: out[r][b][t] = in[b][t] (.) pt[r][t]
// in: [B][kt][2][L][n] (per_msg_in: [R][B][kt][2][L][n], message r times
// plaintext r); pt: [R][kt][L][n] Montgomery; out: [R][B][kt][2][L][n]
__global__ void ke_mul_plain_multi(const CtxDev* __restrict__ C, const uint64_t* in, const uint64_t* pt,
                                   uint64_t* out, uint32_t R, uint32_t B, int per_msg_in) {
  const int L = C->L, logn = C->logn, kt = C->kt;
  const size_t n = C->n;
  const size_t ctw = 2 * (size_t)L * n;
  const size_t total = (size_t)R * B * kt * ctw;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t k = w & (n - 1);
    const int j = (w >> logn) % L;
    const size_t ctg = w / ctw;             // r * B * kt + b * kt + t
    const int t = ctg % kt;
    const size_t r = ctg / ((size_t)B * kt);
    const size_t in_ct = per_msg_in ? ctg : ctg % ((size_t)B * kt);
    const size_t comp = (w / ((size_t)L * n)) & 1;
    const PrimeDev& P = C->pr[j];
    const uint64_t x = in[in_ct * ctw + (comp * L + j) * n + k];
    const uint64_t p = pt[((r * kt + t) * L + j) * n + k];
    out[w] = mont_mul(x, p, P.q, P.qinv);
  }
}

// convolution row-major: out[m][b][t] = sum_r w[r][t][j][m] in[r][b][t]
// in: [R][B][kt][2][L][n]; w, ws: [R][kt][L][maps] scalars (Shoup).  A
// thread accumulates MB maps for WPT adjacent input words (one 8- or 16-byte
// load per input), so every input word is read once per block of MB maps
// and each weight load serves WPT words.
#ifndef LOLA_MAC_WPT
#define LOLA_MAC_WPT 2
#endif
template <int MB, int WPT>
__global__ void ke_mac_scalar(const CtxDev* __restrict__ C, const uint64_t* in, uint32_t R, const uint64_t* w,
                              const uint64_t* ws, uint64_t* out, uint32_t maps, uint32_t B) {
  using VecT = typename std::conditional<WPT == 2, ulonglong2, unsigned long long>::type;
  const int L = C->L, logn = C->logn, kt = C->kt;
  const size_t n = C->n;
  const size_t ctw = 2 * (size_t)L * n;
  const size_t per_msg = (size_t)B * kt * ctw;
  const size_t per_thr = per_msg / WPT;
  const size_t total = (size_t)((maps + MB - 1) / MB) * per_thr;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const uint32_t m0 = (uint32_t)(i / per_thr) * MB;
    const size_t off = (i % per_thr) * WPT;
    const int j = (off >> logn) % L;
    const int t = (off / ctw) % kt;
    const uint64_t q = C->pr[j].q;
    uint64_t acc[MB][WPT];
#pragma unroll
    for (int mm = 0; mm < MB; ++mm)
#pragma unroll
      for (int e = 0; e < WPT; ++e) acc[mm][e] = 0;
    for (uint32_t r = 0; r < R; ++r) {
      const VecT xv = *(const VecT*)(in + r * per_msg + off);
      uint64_t x[WPT];
      if constexpr (WPT == 2) {
        x[0] = xv.x;
        x[1] = xv.y;
      } else {
        x[0] = xv;
      }
      const size_t wb = (((size_t)r * kt + t) * L + j) * maps + m0;
#pragma unroll
      for (int mm = 0; mm < MB; ++mm)
        if (m0 + mm < maps) {
          const uint64_t wv = __ldg(w + wb + mm), wsv = __ldg(ws + wb + mm);
#pragma unroll
          for (int e = 0; e < WPT; ++e) acc[mm][e] = add_mod(acc[mm][e], shoup_mul(x[e], wv, wsv, q), q);
        }
    }
#pragma unroll
    for (int mm = 0; mm < MB; ++mm)
      if (m0 + mm < maps) {
        if constexpr (WPT == 2) {
          *(ulonglong2*)(out + (m0 + mm) * per_msg + off) = make_ulonglong2(acc[mm][0], acc[mm][1]);
        } else {
          out[(m0 + mm) * per_msg + off] = acc[mm][0];
        }
      }
  }
}

// ------------------------------------------------------ exact basis conversion
// Mixed-radix digits of x given by residues x_i (i < k) over basis `b` of the
// MRC table; returns whether x > (prod b - 1) / 2 (the centered lift is x - prod b).
template <int KMAX>
__device__ __forceinline__ bool mrc_digits(const CtxDev* C, const MrcDev& T, int first_prime, int k,
                                           const uint64_t (&x)[KMAX], uint64_t (&v)[KMAX]) {
#pragma unroll
  for (int i = 0; i < KMAX; ++i) {
    if (i < k) {
      const PrimeDev& P = C->pr[first_prime + i];
      uint64_t u = x[i];
#pragma unroll
      for (int j = 0; j < KMAX; ++j) {
        if (j < i) {
          const uint64_t vj = reduce64(v[j], P.q, P.f64);
          u = shoup_mul(sub_mod(u, vj, P.q), T.inv[i][j], T.inv_s[i][j], P.q);
        }
      }
      v[i] = u;
    }
  }
  bool decided = false, gt = false;
#pragma unroll
  for (int i = KMAX - 1; i >= 0; --i) {
    if (i < k && !decided && v[i] != T.half[i]) {
      decided = true;
      gt = v[i] > T.half[i];
    }
  }
  return gt;
}

// lift centered x in Z_Q (residues over q_0..q_{L-1}) to the aux primes
// xq: [poly][L][n], xb: [poly][M][n]
template <int KQ>
__global__ void ke_lift_q_to_b(const CtxDev* __restrict__ C, const uint64_t* xq, uint64_t* xb, size_t n_polys) {
  const int L = C->L, M = C->M, logn = C->logn, iB = C->iB;
  const size_t n = C->n;
  const size_t total = n_polys * n;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t poly = w >> logn, k = w & (n - 1);
    uint64_t x[KQ], v[KQ];
#pragma unroll
    for (int i = 0; i < KQ; ++i) x[i] = i < L ? xq[(poly * L + i) * n + k] : 0;
    const bool neg = mrc_digits<KQ>(C, C->mrcQ, 0, L, x, v);
    for (int jb = 0; jb < M; ++jb) {
      const PrimeDev& P = C->pr[iB + jb];
      uint64_t acc = 0;
#pragma unroll
      for (int i = 0; i < KQ; ++i)
        if (i < L) acc = add_mod(acc, shoup_mul(reduce64(v[i], P.q, P.f64), C->wQB[i][jb], C->wQB_s[i][jb], P.q), P.q);
      if (neg) acc = sub_mod(acc, C->QmodB[jb], P.q);
      xb[(poly * M + jb) * n + k] = acc;
    }
  }
}

// tensor over Q u B (Montgomery products; the inverse transform that follows
// multiplies by 2^64 to undo the factor).  x/y: NTT form, Q part in
// ciphertext layout [ct][2][L][n], B part [ct][2][M][n].
// T: [ct][3][L+M][n]
__global__ void ke_tensor(const CtxDev* __restrict__ C, const uint64_t* xq, const uint64_t* xb, const uint64_t* yq,
                          const uint64_t* yb, uint64_t* T, size_t count) {
  const int L = C->L, M = C->M, LM = C->L + C->M, logn = C->logn, iB = C->iB;
  const size_t n = C->n;
  const size_t total = count * LM * n;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t k = w & (n - 1);
    const int l = (w >> logn) % LM;
    const size_t ct = (w >> logn) / LM;
    uint64_t x0, x1, y0, y1;
    int p;
    if (l < L) {
      p = l;
      x0 = xq[(ct * 2 * L + l) * n + k];
      x1 = xq[(ct * 2 * L + L + l) * n + k];
      y0 = yq[(ct * 2 * L + l) * n + k];
      y1 = yq[(ct * 2 * L + L + l) * n + k];
    } else {
      const int jb = l - L;
      p = iB + jb;
      x0 = xb[(ct * 2 * M + jb) * n + k];
      x1 = xb[(ct * 2 * M + M + jb) * n + k];
      y0 = yb[(ct * 2 * M + jb) * n + k];
      y1 = yb[(ct * 2 * M + M + jb) * n + k];
    }
    const PrimeDev& P = C->pr[p];
    const uint64_t d0 = mont_mul(x0, y0, P.q, P.qinv);
    const uint64_t d1 = add_mod(mont_mul(x0, y1, P.q, P.qinv), mont_mul(x1, y0, P.q, P.qinv), P.q);
    const uint64_t d2 = mont_mul(x1, y1, P.q, P.qinv);
    T[((ct * 3 + 0) * LM + l) * n + k] = d0;
    T[((ct * 3 + 1) * LM + l) * n + k] = d1;
    T[((ct * 3 + 2) * LM + l) * n + k] = d2;
  }
}

// BFV scaling, exact: for d given mod Q u B (coefficient form),
// r = [t d]_Q centered, y = (t d - r) / Q computed mod each b, then y lifted
// exactly from B to Q.  T: [ct][3][L+M][n]; parts 0 and 1 go to E
// ([ct][2][L][n], ciphertext layout), part 2 to DIG ([ct][L][n]).
template <int KQ, int KB>
__global__ void ke_scale_round(const CtxDev* __restrict__ C, const uint64_t* T, const uint32_t* tidx,
                               uint32_t tidx_div, uint64_t* E, uint64_t* DIG, size_t count) {
  const int L = C->L, M = C->M, LM = C->L + C->M, logn = C->logn, iB = C->iB;
  const size_t n = C->n;
  const size_t total = count * 3 * n;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t k = w & (n - 1);
    const size_t cp = w >> logn;         // ct * 3 + part
    const size_t ct = cp / 3;
    const int ti = tidx ? tidx[ct / tidx_div] : 0;
    const uint64_t* src = T + cp * LM * n + k;
    uint64_t r[KQ], v[KQ];
#pragma unroll
    for (int i = 0; i < KQ; ++i)
      r[i] = i < L ? shoup_mul(src[(size_t)i * n], C->tQ[ti][i], C->tQ_s[ti][i], C->pr[i].q) : 0;
    const bool rneg = mrc_digits<KQ>(C, C->mrcQ, 0, L, r, v);
    uint64_t y[KB], u[KB];
#pragma unroll
    for (int jb = 0; jb < KB; ++jb) {
      if (jb < M) {
        const PrimeDev& P = C->pr[iB + jb];
        uint64_t rb = 0;
#pragma unroll
        for (int i = 0; i < KQ; ++i)
          if (i < L) rb = add_mod(rb, shoup_mul(reduce64(v[i], P.q, P.f64), C->wQB[i][jb], C->wQB_s[i][jb], P.q), P.q);
        if (rneg) rb = sub_mod(rb, C->QmodB[jb], P.q);
        const uint64_t td = shoup_mul(src[(size_t)(L + jb) * n], C->tB[ti][jb], C->tB_s[ti][jb], P.q);
        y[jb] = shoup_mul(sub_mod(td, rb, P.q), C->QinvB[jb], C->QinvB_s[jb], P.q);
      } else {
        y[jb] = 0;
      }
    }
    const bool yneg = mrc_digits<KB>(C, C->mrcB, iB, M, y, u);
    const int part = (int)(cp % 3);
    uint64_t* dst = (part < 2 ? E + (ct * 2 + part) * L * n : DIG + ct * L * n) + k;
    for (int i = 0; i < L; ++i) {
      const PrimeDev& P = C->pr[i];
      uint64_t acc = 0;
#pragma unroll
      for (int jb = 0; jb < KB; ++jb)
        if (jb < M) acc = add_mod(acc, shoup_mul(reduce64(u[jb], P.q, P.f64), C->wBQ[jb][i], C->wBQ_s[jb][i], P.q), P.q);
      if (yneg) acc = sub_mod(acc, C->BmodQ[i], P.q);
      dst[(size_t)i * n] = acc;
    }
  }
}

// decryption rounding: x = [c0 + c1 s]_Q (coefficient form, [poly][L][n]) ->
// m = round(t x / Q) mod t = (-(r mod t) Q^-1 + [r > (Q-1)/2]) mod t, r = [t x]_Q
template <int KQ>
__global__ void ke_decrypt_round(const CtxDev* __restrict__ C, const uint64_t* x, const uint32_t* tidx,
                                 uint64_t* m, size_t n_polys) {
  const int L = C->L, logn = C->logn, iT = C->iT;
  const size_t n = C->n;
  const size_t total = n_polys * n;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t poly = w >> logn, k = w & (n - 1);
    const int ti = tidx[poly];
    uint64_t r[KQ], v[KQ];
#pragma unroll
    for (int i = 0; i < KQ; ++i)
      r[i] = i < L ? shoup_mul(x[(poly * L + i) * n + k], C->tQ[ti][i], C->tQ_s[ti][i], C->pr[i].q) : 0;
    const bool gt = mrc_digits<KQ>(C, C->mrcQ, 0, L, r, v);
    const PrimeDev& T = C->pr[iT + ti];
    uint64_t rt = 0;
#pragma unroll
    for (int i = 0; i < KQ; ++i)
      if (i < L) rt = add_mod(rt, shoup_mul(reduce64(v[i], T.q, T.f64), C->wQT[i][ti], C->wQT_s[i][ti], T.q), T.q);
    uint64_t mm = neg_mod(shoup_mul(rt, C->QinvT[ti], C->QinvT_s[ti], T.q), T.q);
    if (gt) mm = add_mod(mm, 1, T.q);
    m[w] = mm;
  }
}

// encryption combine: out[ct][0][j] = M1[ct][j] + U[ct][j] pk0_j ; out[ct][1][j] = E2[ct][j] + U[ct][j] pk1_j
__global__ void ke_enc_combine(const CtxDev* __restrict__ C, const uint64_t* M1, const uint64_t* E2,
                               const uint64_t* U, const uint64_t* pk, uint64_t* out, size_t count) {
  const int L = C->L, logn = C->logn;
  const size_t n = C->n;
  const size_t total = count * 2 * L * n;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t k = w & (n - 1);
    const size_t r = w >> logn;
    const int j = r % L;
    const int comp = (r / L) & 1;
    const size_t ct = r / (2 * L);
    const PrimeDev& P = C->pr[j];
    const size_t src = (ct * L + j) * n + k;
    const uint64_t prod = mont_mul(U[src], pk[((size_t)comp * L + j) * n + k], P.q, P.qinv);
    out[w] = add_mod(comp ? E2[src] : M1[src], prod, P.q);
  }
}

// decryption phase: x = c0 + c1 s (NTT form), out [ct][L][n]
__global__ void ke_dec_phase(const CtxDev* __restrict__ C, const uint64_t* ct_in, const uint64_t* s_mont,
                             uint64_t* out, size_t count) {
  const int L = C->L, logn = C->logn;
  const size_t n = C->n;
  const size_t total = count * L * n;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t k = w & (n - 1);
    const int j = (w >> logn) % L;
    const size_t ct = (w >> logn) / L;
    const PrimeDev& P = C->pr[j];
    const uint64_t c0 = ct_in[(ct * 2 * L + j) * n + k];
    const uint64_t c1 = ct_in[(ct * 2 * L + L + j) * n + k];
    out[w] = add_mod(c0, mont_mul(c1, s_mont[(size_t)j * n + k], P.q, P.qinv), P.q);
  }
}

// ------------------------------------------------------------------ launchers
namespace k {

#define ELEM_LAUNCH(kind, KERNEL, items, ...)                                       \
  do {                                                                             \
    ProfScope ps_(c, kind, s, (uint64_t)(items));                                  \
    KERNEL<<<grid_for(items, 256), 256, 0, s>>>(__VA_ARGS__);                       \
  } while (0)

int ks_ip(Ctx* c, const KsDev& a, bool final_out, cudaStream_t s) {
  const size_t pairs = a.count * (final_out ? c->L : c->L + c->K) * (c->n / 2);
  switch (c->dnum) {
    case 1: ELEM_LAUNCH(KI_KS_IP_Q, ke_ks_ip<1>, pairs, c->dev, a, (int)final_out); break;
    case 2: ELEM_LAUNCH(KI_KS_IP_Q, ke_ks_ip<2>, pairs, c->dev, a, (int)final_out); break;
    case 3: ELEM_LAUNCH(KI_KS_IP_Q, ke_ks_ip<3>, pairs, c->dev, a, (int)final_out); break;
    case 4: ELEM_LAUNCH(KI_KS_IP_Q, ke_ks_ip<4>, pairs, c->dev, a, (int)final_out); break;
    case 5: ELEM_LAUNCH(KI_KS_IP_Q, ke_ks_ip<5>, pairs, c->dev, a, (int)final_out); break;
    case 6: ELEM_LAUNCH(KI_KS_IP_Q, ke_ks_ip<6>, pairs, c->dev, a, (int)final_out); break;
    case 7: ELEM_LAUNCH(KI_KS_IP_Q, ke_ks_ip<7>, pairs, c->dev, a, (int)final_out); break;
    case 8: ELEM_LAUNCH(KI_KS_IP_Q, ke_ks_ip<8>, pairs, c->dev, a, (int)final_out); break;
    default: ELEM_LAUNCH(KI_KS_IP_Q, ke_ks_ip<0>, pairs, c->dev, a, (int)final_out); break;
  }
  return post(c);
}

// profiled units: 64 x 64-bit products (each pair of coefficients takes
// G x digits x 2 components x 2 of them)
int ks_ip_sum(Ctx* c, const KsDev& a, bool final_out, cudaStream_t s) {
  const size_t pairs = a.count * (final_out ? c->L : c->L + c->K) * (c->n / 2);
  ProfScope ps_(c, KI_KS_IP_SUM, s, (uint64_t)pairs * a.gsum * c->dnum * 4);
  const unsigned grid = grid_for(pairs, 256);
  switch (c->dnum) {
    case 1: ke_ks_ip_sum<1><<<grid, 256, 0, s>>>(c->dev, a, (int)final_out); break;
    case 2: ke_ks_ip_sum<2><<<grid, 256, 0, s>>>(c->dev, a, (int)final_out); break;
    case 3: ke_ks_ip_sum<3><<<grid, 256, 0, s>>>(c->dev, a, (int)final_out); break;
    case 4: ke_ks_ip_sum<4><<<grid, 256, 0, s>>>(c->dev, a, (int)final_out); break;
    case 5: ke_ks_ip_sum<5><<<grid, 256, 0, s>>>(c->dev, a, (int)final_out); break;
    case 6: ke_ks_ip_sum<6><<<grid, 256, 0, s>>>(c->dev, a, (int)final_out); break;
    default: ke_ks_ip_sum<0><<<grid, 256, 0, s>>>(c->dev, a, (int)final_out); break;
  }
  return post(c);
}

int add(Ctx* c, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t count, cudaStream_t s) {
  if (!count) return LOLA_OK;
  const size_t total = count * c->ct_words();
  ELEM_LAUNCH(KI_ADD, ke_add, total, c->dev, a, b, out, total, 0);
  return post(c);
}

int sub(Ctx* c, const uint64_t* a, const uint64_t* b, uint64_t* out, size_t count, cudaStream_t s) {
  if (!count) return LOLA_OK;
  const size_t total = count * c->ct_words();
  ELEM_LAUNCH(KI_ADD, ke_add, total, c->dev, a, b, out, total, 1);
  return post(c);
}

int to_mont_map(Ctx* c, uint64_t* data, size_t n_limbpolys, uint32_t limbs, const PrimeMap& pm, cudaStream_t s,
                int mode) {
  const size_t total = n_limbpolys * c->n;
  ELEM_LAUNCH(KI_MISC, ke_to_mont, total, c->dev, data, total, limbs, pm, mode);
  return post(c);
}

int axpy_mont_map(Ctx* c, const uint64_t* a, const uint64_t* b, const uint64_t* w_mont, uint64_t* out,
                  size_t n_limbpolys, uint32_t limbs, const PrimeMap& pm, cudaStream_t s) {
  const size_t total = n_limbpolys * c->n;
  ELEM_LAUNCH(KI_MISC, ke_axpy_mont, total, c->dev, a, b, w_mont, out, total, limbs, pm);
  return post(c);
}

int neg_axpe(Ctx* c, const uint64_t* a, const uint64_t* s_mont, const uint64_t* e, uint64_t* out, uint32_t limbs,
             cudaStream_t s) {
  const size_t total = (size_t)limbs * c->n;
  ELEM_LAUNCH(KI_MISC, ke_neg_axpe, total, c->dev, a, s_mont, e, out, total);
  return post(c);
}

int keygen_switch(Ctx* c, const uint64_t* a, const uint64_t* e, const uint64_t* s_mont, const uint64_t* sfrom,
                  uint64_t* out, cudaStream_t s) {
  const size_t total = (size_t)c->dnum * (c->L + c->K) * c->n;
  ELEM_LAUNCH(KI_MISC, ke_keygen_switch, total, c->dev, a, e, s_mont, sfrom, out);
  return post(c);
}

int gal_permute(Ctx* c, const uint64_t* in, uint64_t* out, size_t n_limbpolys, uint32_t g, cudaStream_t s) {
  const size_t total = n_limbpolys * c->n;
  ELEM_LAUNCH(KI_MISC, ke_gal_permute, total, c->dev, in, out, total, g);
  return post(c);
}

int mul_plain_multi(Ctx* c, const uint64_t* in, const uint64_t* pt, uint64_t* out, uint32_t R, uint32_t B,
                    cudaStream_t s, bool per_msg_in) {
  const size_t total = (size_t)R * B * c->kt * c->ct_words();
  if (!total) return LOLA_OK;
  ELEM_LAUNCH(KI_MUL_PLAIN, ke_mul_plain_multi, total, c->dev, in, pt, out, R, B, (int)per_msg_in);
  return post(c);
}

int sum_msgs(Ctx* c, const uint64_t* src, uint32_t msgs, const uint64_t* aux, uint64_t* out, size_t per,
             cudaStream_t s) {
  const size_t total = per * c->ct_words();
  if (!total) return LOLA_OK;
  ELEM_LAUNCH(KI_ADD, ke_sum_msgs, total, c->dev, src, msgs, aux, out, total);
  return post(c);
}

int mac_scalar(Ctx* c, const uint64_t* in, uint32_t R, const uint64_t* w, const uint64_t* ws, uint64_t* out,
               uint32_t maps, uint32_t B, cudaStream_t s) {
  const size_t per_msg = (size_t)B * c->kt * c->ct_words();
  if (!maps || !per_msg) return LOLA_OK;
  ProfScope ps_(c, KI_MAC_SCALAR, s, (uint64_t)maps * per_msg);   // units: output words
  constexpr int WPT = LOLA_MAC_WPT;        // n is a power of two >= 16, so WPT divides every limb
  if (maps <= 4) {
    const size_t items = per_msg / WPT * ((maps + 3) / 4);
    ke_mac_scalar<4, WPT><<<grid_for(items, 256), 256, 0, s>>>(c->dev, in, R, w, ws, out, maps, B);
  } else {
    const size_t items = per_msg / WPT * ((maps + 7) / 8);
    ke_mac_scalar<8, WPT><<<grid_for(items, 256), 256, 0, s>>>(c->dev, in, R, w, ws, out, maps, B);
  }
  return post(c);
}

template <int KQ>
static int lift_dispatch(Ctx* c, const uint64_t* xq, uint64_t* xb, size_t n_polys, cudaStream_t s) {
  ELEM_LAUNCH(KI_LIFT_Q_TO_B, ke_lift_q_to_b<KQ>, n_polys * c->n, c->dev, xq, xb, n_polys);
  return post(c);
}

int lift_q_to_b(Ctx* c, const uint64_t* xq, uint64_t* xb, size_t n_polys, cudaStream_t s) {
  if (c->L <= 4) return lift_dispatch<4>(c, xq, xb, n_polys, s);
  if (c->L <= 8) return lift_dispatch<8>(c, xq, xb, n_polys, s);
  return lift_dispatch<12>(c, xq, xb, n_polys, s);
}

int tensor(Ctx* c, const uint64_t* xq, const uint64_t* xb, const uint64_t* yq, const uint64_t* yb, uint64_t* T,
           size_t count, cudaStream_t s) {
  ELEM_LAUNCH(KI_TENSOR, ke_tensor, count * (c->L + c->M) * c->n, c->dev, xq, xb, yq, yb, T, count);
  return post(c);
}

template <int KQ, int KB>
static int scale_dispatch(Ctx* c, const uint64_t* T, const uint32_t* tidx, uint32_t div, uint64_t* E, uint64_t* DIG,
                          size_t count, cudaStream_t s) {
  ELEM_LAUNCH(KI_SCALE_ROUND, (ke_scale_round<KQ, KB>), count * 3 * c->n, c->dev, T, tidx, div, E, DIG, count);
  return post(c);
}

int scale_round(Ctx* c, const uint64_t* T, const uint32_t* d_tidx, uint32_t tidx_div, uint64_t* E, uint64_t* DIG,
                size_t count, cudaStream_t s) {
  if (c->L <= 4 && c->M <= 4) return scale_dispatch<4, 4>(c, T, d_tidx, tidx_div, E, DIG, count, s);
  if (c->L <= 8 && c->M <= 8) return scale_dispatch<8, 8>(c, T, d_tidx, tidx_div, E, DIG, count, s);
  return scale_dispatch<12, 16>(c, T, d_tidx, tidx_div, E, DIG, count, s);
}

int decrypt_round(Ctx* c, const uint64_t* x, const uint32_t* d_tidx, uint64_t* m, size_t n_polys, cudaStream_t s) {
  if (c->L <= 4) {
    ELEM_LAUNCH(KI_DECRYPT_ROUND, ke_decrypt_round<4>, n_polys * c->n, c->dev, x, d_tidx, m, n_polys);
  } else if (c->L <= 8) {
    ELEM_LAUNCH(KI_DECRYPT_ROUND, ke_decrypt_round<8>, n_polys * c->n, c->dev, x, d_tidx, m, n_polys);
  } else {
    ELEM_LAUNCH(KI_DECRYPT_ROUND, ke_decrypt_round<12>, n_polys * c->n, c->dev, x, d_tidx, m, n_polys);
  }
  return post(c);
}

int enc_combine(Ctx* c, const uint64_t* M1, const uint64_t* E2, const uint64_t* U, const uint64_t* pk, uint64_t* out,
                size_t count, cudaStream_t s) {
  ELEM_LAUNCH(KI_MISC, ke_enc_combine, count * c->ct_words(), c->dev, M1, E2, U, pk, out, count);
  return post(c);
}

int dec_phase(Ctx* c, const uint64_t* ct, const uint64_t* s_mont, uint64_t* out, size_t count, cudaStream_t s) {
  ELEM_LAUNCH(KI_MISC, ke_dec_phase, count * c->L * c->n, c->dev, ct, s_mont, out, count);
  return post(c);
}

}  // namespace k
}  // namespace lola
