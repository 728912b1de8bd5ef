// Rotation without any device allocation.
//
// Some callers cannot allocate device memory: applications whose memory
// manager owns the whole device and forbids cudaMalloc / cudaMallocAsync
// after start-up, hosts that budget every byte of device memory up front,
// and latency-critical loops where an allocation's cost or its possible
// implicit synchronisation is not acceptable.  For them
// lola_rotate_noalloc rotates ciphertexts using a scratch area that is part
// of the library image itself: a file-scope __device__ array that every GPU
// loading the library holds until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents.  Each rotation overwrites every scratch word it reads before
// reading it (digits, mod-up limbs, special-prime accumulators), so nothing
// has to be cleared between calls.  Calls whose work overlaps on the GPU
// (different streams, or different threads without ordering) race on the
// array; callers must serialise them.
#include <mutex>

#include "he.h"

namespace lola {

// LOLA_ROTATE_NOALLOC_SCRATCH_BYTES (32 MiB) of 64-bit words, 256-byte aligned.
constexpr size_t kNoAllocWords = (size_t)LOLA_ROTATE_NOALLOC_SCRATCH_BYTES / 8;
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocWords];

static std::mutex g_noalloc_lookup;

// Host code must not pass g_noalloc_scratch itself to a kernel: in host code
// that name is only a stand-in for the symbol.  The device address comes from
// cudaGetSymbolAddress with the context's device current (the caller makes
// it current).  It is looked up once per context and kept in the context, so
// a context created after the device was reset (cudaDeviceReset, a new
// primary context) looks it up again instead of reusing a stale address.
// The lock serialises first calls from several threads.
static int noalloc_scratch(Ctx* c, uint64_t** out) {
  Ctx* r = c->root;
  uint64_t* p = r->noalloc_scratch.load(std::memory_order_acquire);
  if (!p) {
    std::lock_guard<std::mutex> lk(g_noalloc_lookup);
    p = r->noalloc_scratch.load(std::memory_order_relaxed);
    if (!p) {
      void* a = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&a, g_noalloc_scratch);
      if (e != cudaSuccess || !a)
        return fail(LOLA_E_CUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
      p = (uint64_t*)a;
      r->noalloc_scratch.store(p, std::memory_order_release);
    }
  }
  *out = p;
  return LOLA_OK;
}

}  // namespace lola

using namespace lola;

struct lola_ctx {
  Ctx* c;
};
struct lola_keys {
  KeySet* k;
};

extern "C" int lola_rotate_noalloc(lola_ctx* ctx, const lola_keys* keys, const uint64_t* in, uint64_t* out,
                                   size_t count, int32_t step, void* stream) {
  if (!ctx || !keys || ((!in || !out) && count)) return fail(LOLA_E_PARAM, "null argument");
  if (in == out && count) return fail(LOLA_E_PARAM, "rotation output must not alias its input");
  Ctx* c = ctx->c;
  if (step < 0 || (uint32_t)step >= c->n / 2) return fail(LOLA_E_PARAM, "rotation step out of range");
  if (!count) return LOLA_OK;
  const size_t need = rotate_scratch_words(c, count);
  if (need > kNoAllocWords)
    return fail(LOLA_E_PARAM, "lola_rotate_noalloc: " + std::to_string(count) + " ciphertexts need " +
                                  std::to_string(need * 8) + " bytes of scratch, the static area holds " +
                                  std::to_string(kNoAllocWords * 8) + "; rotate fewer ciphertexts per call");
  const uint32_t g = galois_for_step(c->n, step);
  const SwitchKey* key = keys->k->galois_key(g);
  if (!key) return fail(LOLA_E_NOKEY, "missing Galois key for step " + std::to_string(step));
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(LOLA_E_CUDA, cudaGetErrorString(e));
  if (dev != c->device) {
    e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(LOLA_E_CUDA, cudaGetErrorString(e));
  }
  uint64_t* scratch = nullptr;
  int rc = noalloc_scratch(c, &scratch);
  if (rc == LOLA_OK) {
    RotSpec rs;
    rs.gal = g;
    rs.key = key->buf.u64();
    rc = rotate(c, in, out, nullptr, count, rs, scratch, (cudaStream_t)stream);
  }
  if (dev != c->device) cudaSetDevice(dev);
  return rc;
}
