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

// Profiling: CUDA events around launches of one kernel class.
struct Profiler {
  bool on[4] = {false, false, false, false};
  double ms[4] = {0, 0, 0, 0};
  uint64_t launches[4] = {0, 0, 0, 0};
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending[4];
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
};

enum KernelKind { KK_NTT = 0, KK_KSIP = 1, KK_ELEM = 2, KK_BASIS = 3 };

// -------------------------------------------------------------------- context
struct Ctx {
  int device = 0;
  uint32_t n = 0, logn = 0, L = 0, K = 0, M = 0, kt = 0;
  std::vector<uint64_t> primes;   // [Q..][P][aux..][t..]
  CtxDev host;                    // host copy of the device constants
  CtxDev* dev = nullptr;          // device copy
  DevBuf d_const, d_tw, d_slotpos;   // d_slotpos[pos] = slot whose value sits at NTT position pos
  std::atomic<uint64_t> launches{0};
  Profiler prof;
  int iP() const { return (int)L; }
  int iB() const { return (int)(L + K); }
  int iT() const { return (int)(L + K + M); }
  size_t ct_words() const { return (size_t)2 * L * n; }
};

// Launch bookkeeping: call before/after a kernel launch of class `kind`.
void prof_begin(Ctx* c, int kind, cudaStream_t s, cudaEvent_t* ev_pair);
void prof_end(Ctx* c, int kind, cudaStream_t s, cudaEvent_t* ev_pair);
struct ProfScope {
  Ctx* c; int kind; cudaStream_t s; cudaEvent_t ev[2] = {nullptr, nullptr};
  ProfScope(Ctx* c_, int k, cudaStream_t s_) : c(c_), kind(k), s(s_) { prof_begin(c, kind, s, ev); }
  ~ProfScope() { prof_end(c, kind, s, ev); }
};

// ---------------------------------------------------------------------- keys
struct SwitchKey {
  DevBuf buf;   // [2 (b, a)][L digits][L+K primes][n], NTT form, Montgomery (x 2^64)
};

// ---------------------------------------------------------------- ciphertexts
struct Ct {
  Ctx* ctx = nullptr;
  size_t n_msg = 0;
  DevBuf buf;           // [n_msg][kt][2][L][n] NTT form
  size_t words() const { return n_msg * ctx->kt * ctx->ct_words(); }
};

uint32_t galois_for_step(uint32_t n, int32_t step);   // step 0 = row swap

}  // namespace lola
