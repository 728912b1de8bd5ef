// 128-bit multiply-accumulate of the key-switch inner products.
#pragma once
#include <stdint.h>

namespace lola {

// (hi:lo) += a * b for 64-bit a, b: the low product added with carry-out,
// the high product added with the carry in (one asm block, so the carry
// flag stays between the two instructions).
__device__ __forceinline__ void mac128(uint64_t& lo, uint64_t& hi, uint64_t a, uint64_t b) {
  asm("mad.lo.cc.u64 %0, %2, %3, %0;\n\t"
      "madc.hi.u64 %1, %2, %3, %1;"
      : "+l"(lo), "+l"(hi)
      : "l"(a), "l"(b));
}

}  // namespace lola
