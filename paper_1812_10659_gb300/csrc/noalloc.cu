// Rotation without any device allocation.
//
// Some callers cannot allocate device memory: code running inside a CUDA
// stream capture that must not create allocation nodes, applications whose
// memory manager forbids cudaMalloc / cudaMallocAsync after start-up, or
// hosts that budget every byte of device memory up front.  For them
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
#include "he.h"

namespace lola {

// LOLA_ROTATE_NOALLOC_SCRATCH_BYTES (32 MiB) of 64-bit words, 256-byte aligned.
constexpr size_t kNoAllocWords = (size_t)LOLA_ROTATE_NOALLOC_SCRATCH_BYTES / 8;
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoAllocWords];

constexpr int kMaxDevices = 64;
static uint64_t* g_noalloc_ptr[kMaxDevices];   // device address per device, set on first use

// Host code must not pass g_noalloc_scratch itself to a kernel: in host code
// that name is only a stand-in for the symbol.  The device address comes from
// cudaGetSymbolAddress with the device current.
static int noalloc_scratch(int device, uint64_t** out) {
  if (device < 0 || device >= kMaxDevices) return fail(LOLA_E_PARAM, "device index out of range");
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail(LOLA_E_CUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
    g_noalloc_ptr[device] = (uint64_t*)p;
  }
  *out = g_noalloc_ptr[device];
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
  int rc = noalloc_scratch(c->device, &scratch);
  if (rc == LOLA_OK) {
    RotSpec rs;
    rs.gal = g;
    rs.key = key->buf.u64();
    rc = rotate(c, in, out, nullptr, count, rs, scratch, (cudaStream_t)stream);
  }
  if (dev != c->device) cudaSetDevice(dev);
  return rc;
}
