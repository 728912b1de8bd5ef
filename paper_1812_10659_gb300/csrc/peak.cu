// Microbenchmarks of the integer units the transforms are bound by, so that
// a transform kernel's rate can be stated as a fraction of a measured peak
// instead of one derived from unit counts.
//
// Each kernel runs a fixed number of operations per thread on register data
// (no memory traffic inside the loop), on 8 CTAs of 256 threads per SM; the
// host times it with CUDA events (best of three after a warm-up run).
//  * forward / inverse butterflies: the transforms' own butterflies (lazy
//    Harvey butterflies with the Shoup product, the forward one correcting
//    its "a" operand on even stages), 16 words and 8 twiddle pairs per thread
//    in registers, stages of decreasing distance as in one pass;
//  * the same forward butterfly with the product left to the compiler's
//    64-bit arithmetic (for comparison with the 32-bit-halves product);
//  * mad.lo.u32, mad.wide.u32, mul.hi.u32: eight independent chains per
//    thread;
//  * mma.sync m16n8k32 s8 x s8 -> s32 (the integer tensor-core path an
//    int8-split matrix transform would use): four independent accumulators
//    per warp, 2 * 16 * 8 * 32 integer operations per instruction;
//  * the rotate-sum inner product's multiply-accumulate (64 x 64 -> 128-bit
//    products accumulated with carry, one REDC per 16).
#include <cuda_runtime.h>

#include "internal.h"
#include "mac.cuh"
#include "modarith.cuh"

namespace lola {

#define TRY_OK(x)                   \
  do {                              \
    int _rc = (x);                  \
    if (_rc != LOLA_OK) return _rc; \
  } while (0)

namespace {

constexpr int kThreads = 256, kCtasPerSm = 8;

// Shoup product for a prime of the form q = 2^60 - c 2^32 + 1 (c < 2^28):
// lo64(qh q) = ((h1 + (h0 << 28) - lo32(h0 c)) << 32) + h0 needs one 32-bit
// product instead of three.
__device__ __forceinline__ uint64_t shoup_mul_lazy_sparse(uint64_t x, uint64_t w, uint64_t wp, uint32_t c) {
  uint64_t r;
  asm("{\n\t"
      ".reg .u32 x0, x1, p0, p1, w0, w1, t, al, ah, bl, bh, h0, h1, l0, l1, s;\n\t"
      ".reg .u64 a, b, d, lo;\n\t"
      "mov.b64 {x0, x1}, %1;\n\t"
      "mov.b64 {w0, w1}, %2;\n\t"
      "mov.b64 {p0, p1}, %3;\n\t"
      "mul.hi.u32 t, x0, p0;\n\t"
      "cvt.u64.u32 d, t;\n\t"
      "mad.wide.u32 a, x0, p1, d;\n\t"
      "mov.b64 {al, ah}, a;\n\t"
      "cvt.u64.u32 d, al;\n\t"
      "mad.wide.u32 b, x1, p0, d;\n\t"
      "mov.b64 {bl, bh}, b;\n\t"
      "cvt.u64.u32 d, bh;\n\t"
      "mad.wide.u32 d, x1, p1, d;\n\t"
      "mov.b64 {h0, h1}, d;\n\t"
      "add.cc.u32 h0, h0, ah;\n\t"
      "addc.u32 h1, h1, 0;\n\t"
      "mul.wide.u32 lo, x0, w0;\n\t"
      "mov.b64 {l0, l1}, lo;\n\t"
      "mad.lo.u32 l1, x0, w1, l1;\n\t"
      "mad.lo.u32 l1, x1, w0, l1;\n\t"
      "mad.lo.u32 l1, h0, %4, l1;\n\t"
      "shl.b32 s, h0, 28;\n\t"
      "sub.cc.u32 l0, l0, h0;\n\t"
      "subc.u32 l1, l1, h1;\n\t"
      "sub.u32 l1, l1, s;\n\t"
      "mov.b64 %0, {l0, l1};\n\t"
      "}"
      : "=l"(r)
      : "l"(x), "l"(w), "l"(wp), "r"(c));
  return r;
}

// PR 0: compiler 64-bit; 1: 32-bit halves; 2: sparse prime (c = nq's high word use)
template <int PR>
__device__ __forceinline__ uint64_t prod(uint64_t x, uint64_t w, uint64_t wp, uint64_t q, uint64_t nq, uint32_t c) {
  if constexpr (PR == 1) return shoup_mul_lazy_ptx(x, w, wp, nq);
  else if constexpr (PR == 2) return shoup_mul_lazy_sparse(x, w, wp, c);
  else return x * w - __umul64hi(x, wp) * q;
}

template <int PR>
__global__ void __launch_bounds__(kThreads) kb_fwd_butterfly(const uint64_t* __restrict__ tw, uint64_t q, int iters,
                                                             uint64_t* __restrict__ sink, uint32_t c) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t x[16], w[8], wp[8];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = (uint64_t)(tid * 16 + k) % q;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    w[k] = tw[2 * k];
    wp[k] = tw[2 * k + 1];
  }
  const uint64_t q2 = 2 * q, q4 = 4 * q, nq = 0ull - q;
  const uint32_t q4hi = (uint32_t)(q4 >> 32);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int lbit = 3; lbit >= 0; --lbit) {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (k & (1 << lbit)) continue;
        const int ti = (k >> (lbit + 1)) & 7;
        uint64_t a = x[k];
        if ((lbit & 1) == 1 && (uint32_t)(a >> 32) > q4hi) a -= q4;   // every other stage
        const uint64_t t = prod<PR>(x[k | (1 << lbit)], w[ti], wp[ti], q, nq, c);
        x[k] = a + t;
        x[k | (1 << lbit)] = a - t + q2;
      }
    }
  }
  uint64_t acc = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) acc ^= x[k];
  sink[tid] = acc;
}

__global__ void __launch_bounds__(kThreads) kb_inv_butterfly(const uint64_t* __restrict__ tw, uint64_t q, int iters,
                                                             uint64_t* __restrict__ sink) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t x[16], w[8], wp[8];
#pragma unroll
  for (int k = 0; k < 16; ++k) x[k] = (uint64_t)(tid * 16 + k) % q;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    w[k] = tw[2 * k];
    wp[k] = tw[2 * k + 1];
  }
  const uint64_t q2 = 2 * q;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int lbit = 0; lbit < 4; ++lbit) {
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        if (k & (1 << lbit)) continue;
        const int ti = (k >> (lbit + 1)) & 7;
        const uint64_t a = x[k], b = x[k | (1 << lbit)];
        uint64_t u = a + b;
        u = u >= q2 ? u - q2 : u;
        x[k] = u;
        x[k | (1 << lbit)] = shoup_mul_lazy(a - b + q2, w[ti], wp[ti], q);
      }
    }
  }
  uint64_t acc = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) acc ^= x[k];
  sink[tid] = acc;
}

// OP 0: mad.lo.u32, 1: mad.wide.u32, 2: mul.hi.u32 (eight chains per thread)
template <int OP>
__global__ void __launch_bounds__(kThreads) kb_imad(uint32_t c, int iters, uint64_t* __restrict__ sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t v[8];
  uint64_t v64[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    v[k] = tid * 8 + k + 1;
    v64[k] = v[k];
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if constexpr (OP == 0) {
          asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(v[k]) : "r"(c), "r"(v[(k + 1) & 7]));
        } else if constexpr (OP == 1) {
          asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(v64[k]) : "r"((uint32_t)v64[k]), "r"(c));
        } else {
          asm volatile("mul.hi.u32 %0, %0, %1;" : "+r"(v[k]) : "r"(c | 0x80000000u));
        }
      }
    }
  }
  uint64_t acc = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) acc += v[k] + v64[k];
  sink[tid] = acc;
}

__global__ void __launch_bounds__(kThreads) kb_mma_s8(int iters, uint64_t* __restrict__ sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t a[4], b[2];
  int32_t d[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k) a[k] = 0x01010101u * ((tid + k) & 3);
  b[0] = 0x01020102u;
  b[1] = 0x02010201u;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < 4; ++k) d[j][k] = 0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      asm volatile(
          "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
          "{%0, %1, %2, %3};"
          : "+r"(d[j][0]), "+r"(d[j][1]), "+r"(d[j][2]), "+r"(d[j][3])
          : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
    }
  }
  uint64_t acc = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc += (uint32_t)d[j][k];
  sink[tid] = acc;
}

// The rotate-sum inner product's operation: 64 x 64 -> 128-bit products
// accumulated with carry (mac128), two key components and two coefficients
// per thread, four products per sum between conditional subtractions of q
// from the high word, one REDC and modular add per 16 products (four
// elements of four digits, as ke_ks_ip_sum runs them).  Every 16 products the
// digits take the reduced sums in (one masked XOR each), so nothing is
// hoisted out of the loop.
__global__ void __launch_bounds__(kThreads) kb_mac64(uint64_t q, uint64_t qinv, int iters,
                                                     uint64_t* __restrict__ sink) {
  const uint64_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t mask = (1ull << 59) - 1;
  uint64_t d[2][4], k0[4], k1[4], a0[2] = {0, 0}, a1[2] = {0, 0};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    d[0][i] = (tid * 8 + i) % q;
    d[1][i] = (tid * 8 + 4 + i) % q;
    k0[i] = (0x9E3779B97F4A7C15ull * (i + 1)) % q;
    k1[i] = (0xBB67AE8584CAA73Bull * (i + 1)) % q;
  }
  for (int it = 0; it < iters; it += 4) {
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      uint64_t lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          mac128(lo0, hi0, d[e][i], k0[i]);
          mac128(lo1, hi1, d[e][i], k1[i]);
        }
        hi0 = csub(hi0, q);
        hi1 = csub(hi1, q);
      }
      a0[e] = add_mod(a0[e], redc128(((unsigned __int128)hi0 << 64) | lo0, q, qinv), q);
      a1[e] = add_mod(a1[e], redc128(((unsigned __int128)hi1 << 64) | lo1, q, qinv), q);
#pragma unroll
      for (int i = 0; i < 4; ++i) d[e][i] ^= a0[e] & mask;   // d stays below 2^60
    }
  }
  sink[tid] = a0[0] ^ a0[1] ^ a1[0] ^ a1[1];
}

}  // namespace

// operations per thread per loop iteration of each kind
static double ops_per_iter(int kind) {
  switch (kind) {
    case 0: case 1: case 2: case 7: return 32; // butterflies (4 stages x 8)
    case 3: case 4: case 5: return 64;         // instructions (8 rounds x 8 chains)
    case 6: return 4.0 * 2 * 16 * 8 * 32 / 32; // int8 operations per thread (4 mma per warp)
    case 8: return 16;                         // 64 x 64-bit products (2 coefficients x 2 components x 4)
                                               // per iteration (the kernel counts iterations of 4 elements)
    default: return 0;
  }
}

int alu_rate(Ctx* c, int kind, double* per_second, double* ms_out) {
  if (kind < 0 || kind > 8) return fail(LOLA_E_PARAM, "unknown ALU benchmark kind");
  LOLA_CUDA_TRY(cudaSetDevice(c->device));
  int sms = 0;
  LOLA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
  const int blocks = sms * kCtasPerSm;
  const int iters = (kind <= 2 || kind == 7) ? 2048 : (kind <= 5 ? 16384 : (kind == 8 ? 4096 : 8192));
  DevBuf sink, tw;
  TRY_OK(sink.alloc((size_t)blocks * kThreads * 8));
  TRY_OK(tw.alloc(16 * 8));
  // twiddles of the first ciphertext prime: the first 8 (w, w') pairs of its
  // forward table; kind 7 uses the prime 2^60 - 96 2^32 + 1 and twiddles 3^k
  // below it, whatever the context's primes
  const uint32_t sparse_c = 96;
  uint64_t q = c->primes[0];
  if (kind == 7) {
    q = (1ull << 60) - ((uint64_t)sparse_c << 32) + 1;
    uint64_t h[16], w = 1;
    for (int k = 0; k < 8; ++k) {
      w = mulmod_h(w, 3, q);
      h[2 * k] = w;
      h[2 * k + 1] = shoup_h(w, q);
    }
    LOLA_CUDA_TRY(cudaMemcpy(tw.p, h, 16 * 8, cudaMemcpyHostToDevice));
  } else {
    LOLA_CUDA_TRY(cudaMemcpy(tw.p, c->host.tw_fwd + 2 * 8, 16 * 8, cudaMemcpyDeviceToDevice));
  }
  cudaEvent_t e0, e1;
  LOLA_CUDA_TRY(cudaEventCreate(&e0));
  LOLA_CUDA_TRY(cudaEventCreate(&e1));
  float best = 0;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, nullptr);
    switch (kind) {
      case 0: kb_fwd_butterfly<1><<<blocks, kThreads>>>(tw.u64(), q, iters, sink.u64(), 0); break;
      case 1: kb_inv_butterfly<<<blocks, kThreads>>>(tw.u64(), q, iters, sink.u64()); break;
      case 2: kb_fwd_butterfly<0><<<blocks, kThreads>>>(tw.u64(), q, iters, sink.u64(), 0); break;
      case 7: kb_fwd_butterfly<2><<<blocks, kThreads>>>(tw.u64(), q, iters, sink.u64(), sparse_c); break;
      case 3: kb_imad<0><<<blocks, kThreads>>>(0x9E3779B9u, iters, sink.u64()); break;
      case 4: kb_imad<1><<<blocks, kThreads>>>(0x9E3779B9u, iters, sink.u64()); break;
      case 5: kb_imad<2><<<blocks, kThreads>>>(0x9E3779B9u, iters, sink.u64()); break;
      case 6: kb_mma_s8<<<blocks, kThreads>>>(iters, sink.u64()); break;
      case 8: kb_mac64<<<blocks, kThreads>>>(q, c->host.pr[0].qinv, iters, sink.u64()); break;
    }
    cudaEventRecord(e1, nullptr);
    cudaError_t err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return fail(LOLA_E_CUDA, std::string("ALU benchmark: ") + cudaGetErrorString(err));
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0 || ms < best)) best = ms;   // rep 0 is the warm-up
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->root->launches.fetch_add(4, std::memory_order_relaxed);
  const double ops = (double)blocks * kThreads * iters * ops_per_iter(kind);
  if (per_second) *per_second = ops / (best * 1e-3);
  if (ms_out) *ms_out = best;
  return LOLA_OK;
}

}  // namespace lola
