// BFV operations composed from the kernels (host orchestration).
#pragma once
#include "internal.h"
#include "kernels.h"

namespace lola {

int ctx_create(const lola_params* p, int device, Ctx** out);
void ctx_destroy(Ctx* c);
int profile_enable(Ctx* c, int kind, int on);
int profile_read(Ctx* c, int kind, double* ms, uint64_t* launches, uint64_t* units);
const char* last_error();

struct EvalKeys {
  std::shared_ptr<SwitchKey> relin;
  std::map<uint32_t, std::shared_ptr<SwitchKey>> galois;   // Galois element -> key
};

struct KeySet {
  Ctx* ctx = nullptr;
  bool has_secret = false, has_public = false;
  std::vector<int64_t> s_coeff;      // ternary secret (host)
  DevBuf s_ntt;                      // [L+K][n] NTT form
  DevBuf s_mont;                     // [L+K][n] NTT form, Montgomery
  DevBuf pk;                         // [2][L][n] NTT form, Montgomery
  std::shared_ptr<EvalKeys> ev;
  const SwitchKey* galois_key(uint32_t g) const {
    auto it = ev->galois.find(g);
    return it == ev->galois.end() ? nullptr : it->second.get();
  }
};

int keygen(Ctx* c, uint64_t seed, const int32_t* steps, size_t n_steps, uint32_t flags, KeySet** secret,
           KeySet** eval);
int keys_export(Ctx* c, const KeySet* ks, int what, int32_t step, uint64_t* host, size_t* words);

int encrypt(Ctx* c, const KeySet* ks, const int64_t* slots, size_t n_msg, uint64_t seed, uint64_t* d_out,
            cudaStream_t s);
int decrypt_residues(Ctx* c, const KeySet* ks, const uint64_t* d_ct, size_t n_msg, uint64_t* host_slots,
                     cudaStream_t s);
// Seeded symmetric encryption (seeded.cu): c1 regenerated from (seed, id)
// in the evaluation domain, c0 = Delta m + e - c1 s.  seeded_c1 writes the
// c1 limbs of `count` ciphertexts [ct][2][L][n] with ids id0, id0 + 1, ...
int encrypt_symmetric(Ctx* c, const KeySet* ks, const int64_t* slots, size_t n_msg, uint64_t seed, uint64_t* d_out,
                      cudaStream_t s);
int seeded_c1(Ctx* c, uint64_t* d_ct, size_t count, uint64_t seed, uint64_t id0, cudaStream_t s);
int to_coeff(Ctx* c, const uint64_t* d_ct, uint64_t* d_out, size_t count, cudaStream_t s);
int from_coeff(Ctx* c, const uint64_t* d_in, uint64_t* d_out, size_t count, cudaStream_t s);

// Rotation / Galois key switch of `count` ciphertexts.  Either a uniform
// Galois element + key, or per-entry arrays on the device (entry i / div).
struct RotSpec {
  const uint32_t* d_gal = nullptr;
  uint32_t gal = 0;
  const uint64_t* const* d_keys = nullptr;
  const uint64_t* key = nullptr;
  uint32_t div = 1;
};
size_t rotate_scratch_words(const Ctx* c, size_t count);
size_t rotate_hoisted_scratch_words(const Ctx* c, size_t count, size_t S);
int rotate_hoisted(Ctx* c, const uint64_t* in, uint64_t* out, size_t count, size_t S, const uint32_t* d_gal,
                   const uint64_t* const* d_keys, uint64_t* scratch, cudaStream_t s);
int rotate(Ctx* c, const uint64_t* in, uint64_t* out, const uint64_t* accum, size_t count, const RotSpec& r,
           uint64_t* scratch, cudaStream_t s);
// Rotate-sum: out = in + sum over G Galois elements of tau_g(in), one key
// switch per ciphertext (the digits raised once, one inner product over all
// elements, one mod-down).  Entry e = i / gal_div of the `count` ciphertexts
// uses elements and keys [e G, e G + G) of the device arrays d_gal / d_keys.
// out must not overlap in.
size_t rotate_sum_scratch_words(const Ctx* c, size_t count);
int rotate_sum(Ctx* c, const uint64_t* in, uint64_t* out, size_t count, uint32_t G, const uint32_t* d_gal,
               const uint64_t* const* d_keys, uint32_t gal_div, uint64_t* scratch, cudaStream_t s);

// Modulus switching of `count` ciphertexts [count][2][L_from][n] to
// [count][2][L_to][n] (L_to <= L_from <= c->L; the first primes of Q stay):
// the top prime is dropped L_from - L_to times, each time
// c'_j = (c_j - x~) q_l^-1 with x~ the centered residue mod the dropped q_l.
// in and out must not overlap.
size_t mod_switch_scratch_words(const Ctx* c, size_t count, uint32_t L_from, uint32_t L_to);
int mod_switch(Ctx* c, const uint64_t* in, uint64_t* out, size_t count, uint32_t L_from, uint32_t L_to,
               uint64_t* scratch, cudaStream_t s);

size_t multiply_scratch_words(const Ctx* c, size_t count, bool square);

// Time every launch geometry of the key-switch transforms per launch-size
// bucket on synthetic buffers and install the fastest in the root context.
int autotune(Ctx* c, cudaStream_t s);
int multiply(Ctx* c, const uint64_t* x, const uint64_t* y, uint64_t* out, size_t count, const uint32_t* d_tidx,
             uint32_t tidx_div, const uint64_t* relin_key, uint64_t* scratch, cudaStream_t s);

// encode slot vectors (host int64 [count][n], plaintext modulus index per
// entry) into NTT-form Montgomery plaintexts [count][L][n] on the device
int encode_plaintexts(Ctx* c, const int64_t* slots, const uint32_t* tidx, size_t count, uint64_t* d_out,
                      cudaStream_t s);

}  // namespace lola
