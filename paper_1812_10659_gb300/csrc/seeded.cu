// Seeded symmetric encryption (a library facility; the paper's encryption
// is SEAL's public-key BFV).  The client holds the secret key (it encrypts
// and decrypts, Sec. 1), so it may encrypt with it: c1 = a uniform, c0 =
// Delta m + e - a s.  a is generated from a seed, so the client sends c0
// and the seed and the server regenerates c1 in the evaluation domain:
// half the bytes on the wire and on the host-to-device copy.
//
// Definition of a (per ciphertext id, per ciphertext prime q_j): its
// evaluation at psi_j^(2i+1) (psi_j the smallest primitive 2n-th root of
// unity mod q_j) is ((w_{2i+1} << 64) | w_{2i}) mod q_j, with w the word
// stream (seed, tag 9, id, j): word w is lane (w mod 4) of Philox4x64-10
// (Salmon et al., SC'11) on counter (w div 4, 9, id, j) under key (seed, 0).
// The forward transform leaves the evaluation at psi^(2 brev(p) + 1) at
// position p, so position p holds evaluation i = brev(p); positions p and
// p + n/2 hold evaluations 2b and 2b + 1, the four words of Philox block b.
#include "he.h"
#include "sampler.h"

namespace lola {
namespace {

__device__ __forceinline__ void philox_dev(uint64_t c[4], uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t m0 = 0xD2E7470EE14C6C93ull, m1 = 0xCA5A826395121157ull;
    const uint64_t lo0 = m0 * c[0], hi0 = __umul64hi(m0, c[0]);
    const uint64_t lo1 = m1 * c[2], hi1 = __umul64hi(m1, c[2]);
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B97F4A7C15ull;
    k1 += 0xBB67AE8584CAA73Bull;
  }
}

// (hi 2^64 + lo) mod q: hi 2^64 = mont_mul(hi mod q, 2^128 mod q)
__device__ __forceinline__ uint64_t wide_mod(uint64_t hi, uint64_t lo, const PrimeDev& P) {
  const uint64_t h = mont_mul(reduce64(hi, P.q, P.f64), P.r2, P.q, P.qinv);
  return add_mod(h, reduce64(lo, P.q, P.f64), P.q);
}

// c1 limbs (NTT form) of `count` ciphertexts [ct][2][L][n] with ids id0 + ct
__global__ void ke_seeded_c1(const CtxDev* __restrict__ C, uint64_t* __restrict__ out, size_t count, uint64_t seed,
                             uint64_t id0) {
  const int L = C->L, logn = C->logn;
  const size_t n = C->n, half = n / 2;
  const size_t total = count * L * half;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t p = w % half;
    const size_t r = w / half;
    const int j = r % L;
    const size_t ct = r / L;
    const PrimeDev& P = C->pr[j];
    const uint32_t i = brev_n((uint32_t)p, logn);   // even: p < n/2 has a zero top bit
    uint64_t c[4] = {i >> 1, TAG_SYM_A, id0 + ct, (uint64_t)j};
    philox_dev(c, seed, 0);
    uint64_t* dst = out + (ct * 2 * L + L + j) * n;
    dst[p] = wide_mod(c[1], c[0], P);
    dst[p + half] = wide_mod(c[3], c[2], P);
  }
}

// c0 = M - c1 s (NTT form), M = NTT(Delta m + e) [ct][L][n]
__global__ void ke_sym_c0(const CtxDev* __restrict__ C, const uint64_t* __restrict__ M,
                          const uint64_t* __restrict__ s_mont, uint64_t* __restrict__ ct, size_t count) {
  const int L = C->L, logn = C->logn;
  const size_t n = C->n;
  const size_t total = count * L * n;
  for (size_t w = blockIdx.x * (size_t)blockDim.x + threadIdx.x; w < total; w += (size_t)gridDim.x * blockDim.x) {
    const size_t k = w & (n - 1);
    const int j = (w >> logn) % L;
    const size_t c = (w >> logn) / L;
    const PrimeDev& P = C->pr[j];
    const uint64_t a = ct[(c * 2 * L + L + j) * n + k];
    ct[(c * 2 * L + j) * n + k] = sub_mod(M[w], mont_mul(a, s_mont[(size_t)j * n + k], P.q, P.qinv), P.q);
  }
}

unsigned grid_items(size_t items) {
  const size_t b = (items + 255) / 256;
  return (unsigned)std::min<size_t>(b, 152 * 16);
}

}  // namespace

int seeded_c1(Ctx* c, uint64_t* d_ct, size_t count, uint64_t seed, uint64_t id0, cudaStream_t s) {
  if (!count) return LOLA_OK;
  const size_t items = count * c->L * (c->n / 2);
  {
    ProfScope ps(c, KI_MISC, s, items);
    ke_seeded_c1<<<grid_items(items), 256, 0, s>>>(c->dev, d_ct, count, seed, id0);
  }
  c->root->launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(LOLA_E_CUDA, std::string("seeded c1: ") + cudaGetErrorString(e));
  return LOLA_OK;
}

int encrypt_symmetric(Ctx* c, const KeySet* ks, const int64_t* slots, size_t n_msg, uint64_t seed, uint64_t* d_out,
                      cudaStream_t s) {
  if (!ks->has_secret) return fail(LOLA_E_STATE, "symmetric encryption needs the secret key");
  const size_t n = c->n, L = c->L, kt = c->kt;
  const size_t count = n_msg * kt;
  if (!count) return LOLA_OK;
  std::vector<uint64_t> red(count * n);
  std::vector<uint32_t> tidx(count);
  std::vector<int64_t> e(count * n);
  for (size_t m = 0; m < n_msg; ++m)
    for (size_t ti = 0; ti < kt; ++ti) {
      const size_t id = m * kt + ti;
      const int64_t t = (int64_t)c->primes[c->iT() + ti];
      tidx[id] = (uint32_t)ti;
      for (size_t j = 0; j < n; ++j) {
        int64_t v = slots[m * n + j] % t;
        red[id * n + j] = (uint64_t)(v < 0 ? v + t : v);
      }
      sample_gaussian(seed, TAG_SYM_E, id, 0, e.data() + id * n, n);
    }
  DevBuf dsl, dco, dti, de, dM;
  int rc;
  if ((rc = dsl.alloc(count * n * 8)) || (rc = dco.alloc(count * n * 8)) || (rc = dti.alloc(count * 4)) ||
      (rc = de.alloc(count * n * 8)) || (rc = dM.alloc(count * L * n * 8)))
    return rc;
  LOLA_CUDA_TRY(cudaMemcpyAsync(dsl.p, red.data(), count * n * 8, cudaMemcpyHostToDevice, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(dti.p, tidx.data(), count * 4, cudaMemcpyHostToDevice, s));
  LOLA_CUDA_TRY(cudaMemcpyAsync(de.p, e.data(), count * n * 8, cudaMemcpyHostToDevice, s));
  if ((rc = k::slots_to_coeff(c, dsl.u64(), (const uint32_t*)dti.p, dco.u64(), count, s))) return rc;
  if ((rc = k::enc_msg(c, dco.u64(), (const int64_t*)de.p, (const uint32_t*)dti.p, dM.u64(), count, s))) return rc;
  if ((rc = seeded_c1(c, d_out, count, seed, 0, s))) return rc;
  {
    const size_t items = count * L * n;
    ProfScope ps(c, KI_MISC, s, items);
    ke_sym_c0<<<grid_items(items), 256, 0, s>>>(c->dev, dM.u64(), ks->s_mont.u64(), d_out, count);
  }
  c->root->launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return fail(LOLA_E_CUDA, std::string("symmetric encryption: ") + cudaGetErrorString(err));
  LOLA_CUDA_TRY(cudaStreamSynchronize(s));
  return LOLA_OK;
}

}  // namespace lola
