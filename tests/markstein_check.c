/* Markstein's corrected quotient (P. Markstein, IBM J. Res. Dev. 34, 1990):
 * with r = RN(1/c), q = RN(d * r), the residual e = d - q * c is exact and
 * RN(q + e * r), taken with one FMA, is RN(d / c).  The heat-trace kernel of
 * the reduced forms divides its Welford updates this way.  Checks random d
 * over a wide exponent range against IEEE division for c = 1..cmax; prints
 * the sample and mismatch counts. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint64_t next(void) {
  state ^= state << 13;
  state ^= state >> 7;
  state ^= state << 17;
  return state;
}

int main(int argc, char **argv) {
  const int cmax = argc > 1 ? atoi(argv[1]) : 512;
  const long per = argc > 2 ? atol(argv[2]) : 4000;
  long n = 0, bad = 0;
  for (int c = 1; c <= cmax; ++c) {
    const double r = 1.0 / (double)c;
    for (long i = 0; i < per; ++i) {
      const uint64_t b = next();
      double d = ldexp((double)(b >> 11) / 9007199254740992.0 + 0.5, (int)(next() % 601) - 300);
      if (b & 1) d = -d;
      const double q = d * r;
      const double e = fma(-q, (double)c, d);
      const double got = fma(e, r, q);
      const double want = d / (double)c;
      if (memcmp(&got, &want, sizeof got) != 0) ++bad;
      ++n;
    }
  }
  printf("%ld %ld\n", n, bad);
  return 0;
}
