// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lola.h"
#include "modarith.cuh"

namespace lola {

constexpr int MAXP = 40;    // primes per context: Q + P + aux + t
constexpr int MAXL = 12;    // ciphertext primes
constexpr int MAXB = 16;    // size bound of either mixed-radix basis (Q or aux)
constexpr int MAXT = 4;     // plaintext moduli

struct PrimeDev {
  uint64_t q, qinv, r2, f64;  // modulus, -q^-1 mod 2^64, 2^128 mod q, floor(2^64/q)
  uint64_t ninv, ninv_s;      // n^-1 and its Shoup companion
  uint64_t ninvr, ninvr_s;    // n^-1 * 2^64 mod q (undoes one Montgomery factor)
};

// Constants for exact mixed-radix (Garner) conversion out of a basis
// b_0..b_{k-1}: x = v_0 + v_1 b_0 + v_2 b_0 b_1 + ..., v_i in [0, b_i).
struct MrcDev {
  int k;                           // basis size
  uint64_t inv[MAXB][MAXB];        // inv[i][j] = b_j^-1 mod b_i (j < i)
  uint64_t inv_s[MAXB][MAXB];
  uint64_t half[MAXB];             // mixed-radix digits of (prod b - 1) / 2
};

// modup work items of one ciphertext: (digit, target prime) pairs
constexpr int MAXMU = MAXL * (MAXL + 2);

struct CtxDev {
  uint32_t n, logn, L, K, M, kt, np;
  uint32_t alpha, dnum;            // primes per key-switching digit, digits (ceil(L / alpha))
  int iP;                          // index of the first special prime (= L) when K > 0
  int iB;                          // first auxiliary prime index (= L + K)
  int iT;                          // first plaintext modulus index (= L + K + M)
  // 1 when every prime of Q and P is below 8x the smallest one: a digit
  // (< q_i) is then a valid forward-transform input for every q_j as it is
  uint32_t modup_raw;
  PrimeDev pr[MAXP];
  const uint64_t* tw_fwd;          // [np][n] pairs (w, floor(w 2^64 / q))
  const uint64_t* tw_inv;          // [np][n] pairs for psi^-1
  // --- exact lifts Q -> B and B -> Q ---
  MrcDev mrcQ;                     // over q_0..q_{L-1}
  MrcDev mrcB;                     // over the aux primes b_0..b_{M-1}
  uint64_t wQB[MAXB][MAXB];        // [k][j] prod_{l<k} q_l mod b_j
  uint64_t wQB_s[MAXB][MAXB];
  uint64_t QmodB[MAXB];            // Q mod b_j
  uint64_t wBQ[MAXB][MAXB];        // [k][i] prod_{l<k} b_l mod q_i
  uint64_t wBQ_s[MAXB][MAXB];
  uint64_t BmodQ[MAXB];            // prod B mod q_i
  uint64_t QinvB[MAXB], QinvB_s[MAXB];            // Q^-1 mod b_j
  uint64_t tQ[MAXT][MAXB], tQ_s[MAXT][MAXB];      // t mod q_i
  uint64_t tB[MAXT][MAXB], tB_s[MAXT][MAXB];      // t mod b_j
  // --- decryption ---
  uint64_t wQT[MAXB][MAXT], wQT_s[MAXB][MAXT];    // prod_{l<k} q_l mod t
  uint64_t QinvT[MAXT], QinvT_s[MAXT];            // Q^-1 mod t
  uint64_t deltaQ[MAXT][MAXB];                    // floor(Q/t) mod q_i
  uint64_t deltaQ_s[MAXT][MAXB];
  // --- key switching (P = product of the K special primes) ---
  uint64_t PmodQ[MAXB], PmodQ_s[MAXB];
  uint64_t PinvQ[MAXB], PinvQ_s[MAXB];            // P^-1 mod q_i
  // mod-up work items: [0] every (digit g, prime j), [1] those with q_j
  // outside digit g's group (the diagonal blocks come from decompose)
  uint32_t mu_n[2];
  uint8_t mu_g[2][MAXMU], mu_j[2][MAXMU];
  // digits of two primes (q_a, q_b = q_{a+1}, a = alpha g): q_a^-1 mod q_b
  // and q_a mod every prime of Q P (the digit is a + q_a ((b - a) q_a^-1 mod q_b))
  uint64_t grp_inv[MAXL], grp_inv_s[MAXL];
  uint64_t grp_qa[MAXL][MAXL + 2], grp_qa_s[MAXL][MAXL + 2];
  uint32_t modup_lazy_a;           // 1 when q_a < 6 q_j for all primes (a digit's q_a-part needs no reduction)
  // K = 2 mod-down: x = x1 + P1 v, v = (x2 - x1) P1^-1 mod P2; (P - 1) / 2 =
  // ph1 + P1 phv; P1 P^-1 mod q_i
  uint64_t P1invP2, P1invP2_s, ph1, phv;
  uint64_t P1PinvQ[MAXB], P1PinvQ_s[MAXB];
  uint64_t PmontQ[MAXB];                          // (P mod q_i) 2^64 mod q_i (P = 1 when K = 0)
  // switching keys are stored as k * P^-1 * 2^64 mod q_j on the L ciphertext
  // primes (k * 2^64 on the special prime), so the inner product already
  // carries the ModDown factor P^-1:
  uint64_t KskR2[MAXB];                           // 2^128 P^-1 mod q_j; 2^128 mod P on P
  uint64_t KskOut[MAXB];                          // P mod q_j; 1 on P (Montgomery factor back to k)
  // geometry of the switching keys, which belong to the full context: kdnum
  // digits of kL + K primes, the special primes at prime index kL (kL = L
  // except in a context reached by modulus switching)
  uint32_t kL, kLK, kdnum;
};

// host-side error reporting
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define LOLA_CUDA_TRY(expr)                                                          \
  do {                                                                               \
    cudaError_t _e = (expr);                                                         \
    if (_e != cudaSuccess)                                                           \
      return ::lola::fail(LOLA_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

}  // namespace lola
