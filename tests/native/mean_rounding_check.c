/* The geometry pass's point coordinates (ms_simplex.cu, narrow path): a
 * coordinate is the mean of n corners (n = 1..4), k of them one step above
 * the cell's coordinate o, i.e. (n o + k) / n rounded to nearest even.  The
 * kernel takes fl(o) + fl(k / n), and for k / n = 2/3 at o = 1 the constant
 * fl(5/3) (bits 0x3FD55555).  This checks, for every o below 2^21 and every
 * (n, k), that the result is the float nearest (n o + k) / n.  No quotient is
 * halfway between two floats: for n = 1, 2, 4 it is itself a float, and for
 * n = 3 it is either an integer or not a dyadic rational, while halfway points
 * are dyadic.  Prints "ok". */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

int main(void) {
  long bad = 0;
  const uint32_t five_thirds_bits = 0x3FD55555u;
  float five_thirds;
  memcpy(&five_thirds, &five_thirds_bits, sizeof five_thirds);
  if (five_thirds != (float)(5.0 / 3.0)) ++bad;
  for (uint32_t n = 1; n <= 4; ++n) {
    for (uint32_t k = 0; k <= n; ++k) {
      const float frac = (float)k / (float)n;
      for (uint32_t o = 0; o < (1u << 21); ++o) {
        const float q = (o == 1 && n == 3 && k == 2) ? five_thirds : (float)o + frac;
        const double s = (double)n * o + k; /* exact */
        /* nearest: n q is no farther from s than n times either neighbour */
        const double e = fabs((double)n * q - s);
        if (e > fabs((double)n * nextafterf(q, INFINITY) - s) ||
            e > fabs((double)n * nextafterf(q, -INFINITY) - s))
          ++bad;
      }
    }
  }
  if (bad) {
    printf("bad %ld\n", bad);
    return 1;
  }
  printf("ok\n");
  return 0;
}
