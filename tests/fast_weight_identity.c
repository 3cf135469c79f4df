/* Exhaustive check of the identity behind the warp kernels' fast weight form.
 *
 * For every fp32 a in [0.5, 4094.5) (so sx = a - 0.5 lies in [0, 4094)):
 *   definition: sx = fl(a - 0.5); x0 = floor(sx); f = fl(sx - x0); t = f * 2048;
 *               k = floor(t); q = k + (t - k >= 0.5)      (11-bit weight, half up)
 *   fast form:  T = floor(fl(2048 a - 1023.5))            (one rounding, as one fma)
 *   identity:   T == 2048 * x0 + q
 * 2048 a - 1023.5 is computed exactly in double and rounded once to float, which is
 * what an fma does. Exit status 0 iff no value breaks the identity. */
#include <stdio.h>
#include <math.h>
#include <stdint.h>
#include <string.h>
int main(void) {
  float lo = 0.5f, hi = 4094.5f;
  uint32_t ulo, uhi; memcpy(&ulo, &lo, 4); memcpy(&uhi, &hi, 4);
  long bad = 0, n = 0;
  for (uint32_t u = ulo; u < uhi; ++u) {
    float a; memcpy(&a, &u, 4);
    float sx = a - 0.5f;
    long x0 = (long)floorf(sx);
    float f = sx - (float)x0;
    float t = f * 2048.0f;
    long k = (long)floorf(t);
    long q = k + ((t - (float)k) >= 0.5f);
    double e = (double)a * 2048.0 - 1023.5;
    float ef = (float)e;
    long T = (long)floorf(ef);
    if ((double)ef != e) { bad++; if (bad < 5) printf("inexact fma at a=%.9g\n", a); }
    if (T != 2048 * x0 + q) { bad++; if (bad < 10) printf("mismatch a=%.9g T=%ld ref=%ld\n", a, T, 2048*x0+q); }
    n++;
  }
  printf("checked %ld values, %ld bad\n", n, bad);
  return bad != 0;
}
