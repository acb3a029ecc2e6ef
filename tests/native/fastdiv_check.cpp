// Exhaustive-in-part check of FastDivU32 against the hardware divide: every
// divisor below 2^12 and a spread of larger ones, each against boundary and
// pseudo-random dividends.  Prints "ok" or the first mismatch.
#include <stdint.h>
#include <stdio.h>

#include "../../paper_2303_15491_gb300/csrc/fastdiv.h"

static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint32_t next() {  // xorshift64*
  state ^= state >> 12;
  state ^= state << 25;
  state ^= state >> 27;
  return (uint32_t)((state * 0x2545F4914F6CDD1Dull) >> 32);
}

static int check(uint32_t d, uint32_t n) {
  msseg::FastDivU32 f(d);
  if (f.div(n) != n / d) {
    printf("mismatch d=%u n=%u got %u want %u\n", d, n, f.div(n), n / d);
    return 1;
  }
  return 0;
}

int main() {
  const uint32_t edge[] = {0u, 1u, 2u, 3u, 0x7fffffffu, 0x80000000u, 0xfffffffeu, 0xffffffffu};
  for (uint32_t d = 1; d < 4096; ++d) {
    for (uint32_t e : edge)
      if (check(d, e)) return 1;
    for (int k = 1; k < 4; ++k)
      for (int64_t off = -2; off <= 2; ++off) {
        const int64_t n = (int64_t)d * k * 977 + off;
        if (n >= 0 && n <= 0xffffffffll && check(d, (uint32_t)n)) return 1;
      }
    for (int i = 0; i < 256; ++i)
      if (check(d, next())) return 1;
  }
  for (int i = 0; i < 200000; ++i) {
    uint32_t d = next() >> (next() % 32);
    if (d == 0) d = 1;
    for (uint32_t e : edge)
      if (check(d, e)) return 1;
    if (check(d, next()) || check(d, d) || check(d, d - 1) || check(d, d * 2u)) return 1;
  }
  printf("ok\n");
  return 0;
}
