// Division of 32-bit unsigned integers by a run-time invariant divisor with
// one multiply-high, two shifts and two adds: the method of Granlund and
// Montgomery, "Division by invariant integers using multiplication" (PLDI
// 1994), Fig. 4.1.  For a divisor d >= 1 with l = ceil(log2 d):
//   m = floor(2^32 * (2^l - d) / d) + 1,  sh1 = min(l, 1),  sh2 = max(l - 1, 0)
//   t = mulhi(m, n);  n / d = (t + ((n - t) >> sh1)) >> sh2
// exactly, for every 0 <= n < 2^32.
#pragma once

#include <stdint.h>

#ifdef __CUDACC__
#define MS_HD __host__ __device__ __forceinline__
#else
#define MS_HD inline
#endif

namespace msseg {

struct FastDivU32 {
  uint32_t d = 1, m = 1, sh1 = 0, sh2 = 0;

  FastDivU32() = default;
  explicit FastDivU32(uint32_t divisor) : d(divisor ? divisor : 1) {
    uint32_t l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    m = (uint32_t)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    sh1 = l < 1 ? l : 1;
    sh2 = l > 1 ? l - 1 : 0;
  }

  MS_HD uint32_t div(uint32_t n) const {
#ifdef __CUDA_ARCH__
    const uint32_t t = __umulhi(m, n);
#else
    const uint32_t t = (uint32_t)(((uint64_t)m * n) >> 32);
#endif
    return (t + ((n - t) >> sh1)) >> sh2;
  }
  MS_HD void divmod(uint32_t n, uint32_t *q, uint32_t *r) const {
    *q = div(n);
    *r = n - *q * d;
  }
};

}  // namespace msseg
