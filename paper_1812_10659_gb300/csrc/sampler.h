// Host-side randomness for key generation and encryption.
//
// One word stream per sampled polynomial: stream (seed, tag, a, b) is the
// sequence of 64-bit words where word w is lane (w mod 4) of the
// Philox4x64-10 block cipher (Salmon, Moraes, Dror, Shaw, SC'11) applied to
// counter (w div 4, tag, a, b) under key (seed, 0).  Distributions:
//   uniform mod q : take words until (w & (2^bitlen(q) - 1)) < q
//   ternary       : take words until w < 3 floor(2^64 / 3); w mod 3 -> {0, 1, -1}
//   Gaussian      : one word per coefficient, sigma = 3.2, |e| <= 19, by
//                   inversion of a cumulative table on the low 63 bits, sign
//                   from the top bit (table in gauss_cdt.h).
#pragma once
#include <stdint.h>

#include <vector>

namespace lola {

enum StreamTag : uint64_t {
  TAG_SECRET = 1, TAG_PK_A = 2, TAG_PK_E = 3, TAG_KSK_A = 4, TAG_KSK_E = 5,
  TAG_ENC_U = 6, TAG_ENC_E1 = 7, TAG_ENC_E2 = 8, TAG_SYM_A = 9, TAG_SYM_E = 10,
};

class PhiloxStream {
 public:
  PhiloxStream(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b) : seed_(seed), tag_(tag), a_(a), b_(b) {}
  uint64_t next();

 private:
  uint64_t seed_, tag_, a_, b_;
  uint64_t word_ = 0;
  uint64_t block_[4] = {0, 0, 0, 0};
  uint64_t block_id_ = ~0ull;
};

void philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);

void sample_uniform(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, uint64_t q, uint64_t* out, size_t n);
void sample_ternary(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, int64_t* out, size_t n);
void sample_gaussian(uint64_t seed, uint64_t tag, uint64_t a, uint64_t b, int64_t* out, size_t n);

}  // namespace lola
