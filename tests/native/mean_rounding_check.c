/* The geometry pass's point coordinates (ms_simplex.cu, mean_of): for a sum s
 * of n corner coordinates (n = 1..4, s < 2^23), s is converted exactly
 * through the mantissa of 2^23 and divided as q = s * R with R = 1/n rounded,
 * then corrected once with the FMA residual (Markstein): q' = q + (s - q n) R.
 * This checks, for every s below 2^23, that the conversion is exact and q'
 * is the float nearest s / n.  No quotient is halfway between two floats:
 * for n = 1, 2, 4 it is itself a float, and for n = 3 it is either an
 * integer or not a dyadic rational, while halfway points are dyadic.
 * Prints "ok". */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

static float via_mantissa(uint32_t s) {
  const uint32_t bits = 0x4B000000u | s;
  float f;
  memcpy(&f, &bits, sizeof f);
  return f - 8388608.0f;
}

int main(void) {
  long bad = 0;
  for (uint32_t n = 1; n <= 4; ++n) {
    const float R = 1.0f / (float)n, c = (float)n;
    for (uint32_t s = 0; s < (1u << 23); ++s) {
      const float f = via_mantissa(s);
      if (f != (float)s) ++bad;
      const float q = f * R;
      const float q1 = fmaf(fmaf(-q, c, f), R, q);
      /* nearest: n q1 is no farther from s than n times either neighbour */
      const double e = fabs((double)n * q1 - s);
      if (e > fabs((double)n * nextafterf(q1, INFINITY) - s) ||
          e > fabs((double)n * nextafterf(q1, -INFINITY) - s))
        ++bad;
    }
  }
  if (bad) {
    printf("bad %ld\n", bad);
    return 1;
  }
  printf("ok\n");
  return 0;
}
