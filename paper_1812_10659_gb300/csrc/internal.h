// Host-side objects behind the C-ABI handles.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "common.h"

namespace lola {

// ---------------------------------------------------------------- host math
typedef unsigned __int128 u128;
uint64_t mulmod_h(uint64_t a, uint64_t b, uint64_t q);
uint64_t powmod_h(uint64_t b, uint64_t e, uint64_t q);
uint64_t invmod_h(uint64_t a, uint64_t q);
bool is_prime_h(uint64_t x);
uint64_t shoup_h(uint64_t w, uint64_t q);            // floor(w 2^64 / q)
uint64_t smallest_root_2n(uint64_t q, uint32_t n);   // smallest primitive 2n-th root of unity

// ------------------------------------------------------------ device memory
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept;
  ~DevBuf();
  int alloc(size_t nbytes);           // LOLA_OK or LOLA_E_NOMEM
  uint64_t* u64() const { return (uint64_t*)p; }
};

// Kernel identities for profiling (lola_profile_* in the C-ABI).
enum KernelId {
  KI_NTT_FWD = 0, KI_NTT_INV, KI_NTT_SIGNED, KI_ENCODE_LIFT, KI_SLOTS_TO_COEFF, KI_COEFF_TO_SLOTS, KI_ENC_MSG,
  KI_KS_DECOMPOSE, KI_KS_MODUP, KI_KS_IP_P, KI_KS_MODDOWN, KI_KS_IP_Q,
  KI_ADD, KI_MUL_PLAIN, KI_MAC_SCALAR, KI_TENSOR, KI_LIFT_Q_TO_B, KI_SCALE_ROUND, KI_DECRYPT_ROUND, KI_MISC,
  KI_MOD_SWITCH, KI_KS_IP_SUM, KI_COUNT
};
const char* kernel_name(int id);

// Profiling: CUDA events around every launch of the enabled kernels, plus
// the work units each launch processed (limb-polynomials for transform
// kernels, 64-bit words for element-wise kernels).
struct Profiler {
  bool on[KI_COUNT] = {};
  double ms[KI_COUNT] = {};
  uint64_t launches[KI_COUNT] = {};
  uint64_t units[KI_COUNT] = {};
  struct Pending { cudaEvent_t a, b; uint64_t units; };
  std::vector<Pending> pending[KI_COUNT];
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
  bool any() const {
    for (int i = 0; i < KI_COUNT; ++i)
      if (on[i]) return true;
    return false;
  }
};

// Launch geometry of the key-switch transforms (decompose, mod-up, INTT mod
// P, mod-down) per launch-size bucket: one CTA per limb, or (n = 16384) a
// 2-CTA cluster per limb with 16 or 32 words per thread, or a 4-CTA cluster
// with 16 words per thread.  Chosen by timing (autotune) or by the built-in
// defaults when `on` is false.
constexpr int TUNE_KERNELS = 4;
constexpr int TUNE_BUCKETS = 6;     // limb transforms per launch: <64, <256, <1024, <4096, <16384, more
enum TuneVariant : uint8_t { TV_CTA = 0, TV_CLUSTER16 = 1, TV_CLUSTER32 = 2, TV_CLUSTER4_16 = 3, TV_COUNT = 4 };
struct Tune {
  bool on = false;
  uint8_t v[TUNE_KERNELS][TUNE_BUCKETS] = {};
  float us[TUNE_KERNELS][TUNE_BUCKETS][TV_COUNT] = {};   // measured microseconds per launch (0: not run)
};
int tune_bucket(size_t units);

// -------------------------------------------------------------------- context
struct Ctx {
  int device = 0;
  uint32_t n = 0, logn = 0, L = 0, K = 0, M = 0, kt = 0;
  uint32_t alpha = 1, dnum = 0;   // primes per key-switching digit, digits (ceil(L / alpha))
  std::vector<uint64_t> primes;   // [Q..][P][aux..][t..]
  CtxDev host;                    // host copy of the device constants
  CtxDev* dev = nullptr;          // device copy
  DevBuf d_const, d_tw, d_slotpos;   // d_slotpos[pos] = slot whose value sits at NTT position pos
  std::atomic<uint64_t> launches{0};
  Profiler prof;
  Tune tune;                      // root context's table applies to every level
  // device address of the library's static rotation scratch array (looked
  // up on the first lola_rotate_noalloc call with this context)
  std::atomic<uint64_t*> noalloc_scratch{nullptr};
  // Modulus switching: a context of the first L' < L ciphertext primes (same
  // special prime, plaintext moduli and keys) is a child of the full one.
  // Launch counts and profiles go to the root; children live in its map.
  Ctx* root = this;
  std::map<uint32_t, std::unique_ptr<Ctx>> levels;
  int iP() const { return (int)L; }
  int iB() const { return (int)(L + K); }
  int iT() const { return (int)(L + K + M); }
  size_t ct_words() const { return (size_t)2 * L * n; }
};

// The context of the first Lv ciphertext primes of `c` (c itself when Lv is
// its L); created on first use, owned by the root context.
int ctx_level(Ctx* c, uint32_t Lv, Ctx** out);

// Launch bookkeeping around one kernel launch.
void prof_begin(Ctx* c, int id, cudaStream_t s, cudaEvent_t* ev_pair);
void prof_end(Ctx* c, int id, cudaStream_t s, cudaEvent_t* ev_pair, uint64_t units);
struct ProfScope {
  Ctx* c; int id; cudaStream_t s; uint64_t units; cudaEvent_t ev[2] = {nullptr, nullptr};
  ProfScope(Ctx* c_, int id_, cudaStream_t s_, uint64_t u) : c(c_), id(id_), s(s_), units(u) { prof_begin(c, id, s, ev); }
  ~ProfScope() { prof_end(c, id, s, ev, units); }
};

// ---------------------------------------------------------------------- keys
struct SwitchKey {
  DevBuf buf;   // [2 (b, a)][dnum digits][L+K primes][n], NTT form, Montgomery (x 2^64)
};

// ---------------------------------------------------------------- ciphertexts
struct Ct {
  Ctx* ctx = nullptr;
  size_t n_msg = 0;
  uint32_t level = 0;   // ciphertext primes after modulus switching (0: all of ctx)
  DevBuf buf;           // [n_msg][kt][2][L][n] NTT form (capacity for the full L)
  size_t words() const { return n_msg * ctx->kt * ctx->ct_words(); }
  uint32_t L() const { return level ? level : ctx->L; }
  size_t used_words() const { return n_msg * ctx->kt * 2 * (size_t)L() * ctx->n; }
};

uint32_t galois_for_step(uint32_t n, int32_t step);   // step 0 = row swap

// Integer-unit microbenchmark `kind` (lola_alu_rate) on the context's device:
// operations per second and the best kernel time in ms (peak.cu).
int alu_rate(Ctx* c, int kind, double* per_second, double* ms);

}  // namespace lola
