/* Exhaustive check of the identities behind the warp kernels' fast coordinate forms.
 *
 * For every fp32 a in [0.5, 4094.5) (so sx = a - 0.5 lies in [0, 4094)):
 *   definition: sx = fl(a - 0.5); x0 = floor(sx); f = fl(sx - x0); t = f * 2048;
 *               k = floor(t); q = k + (t - k >= 0.5)      (11-bit weight, half up)
 *   u8 form:    T = floor(fl(2048 a - 1023.5))            (one rounding, as one fma)
 *               T == 2048 * x0 + q; and the fma rounded toward minus infinity with
 *               addend 2^23 - 1023.5 gives the float 2^23 + T, whose bits are
 *               0x4B000000 + T (no float-to-int conversion needed)
 *   f32 form:   fl = fl_down(a + (2^23 - 0.5)) is the float 2^23 + x0 (bits 0x4B000000 + x0);
 *               fl(a - fl(fl - (2^23 - 0.5))) == fl(sx - x0), the fp32 weight of x0 + 1
 * 2048 a - 1023.5 is also computed exactly in double and must be a float (so rounding
 * it once, as an fma does, changes nothing). The downward-rounded operations run with
 * the host's rounding mode set to FE_DOWNWARD, in chunks, everything else to nearest.
 * Exit status 0 iff no value breaks an identity. */
#include <fenv.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#pragma STDC FENV_ACCESS ON

#define CHUNK 1048576
static float rd_t[CHUNK], rd_f[CHUNK];

static uint32_t bits(float v) { uint32_t u; memcpy(&u, &v, 4); return u; }

int main(void) {
  float lo = 0.5f, hi = 4094.5f;
  uint32_t ulo = bits(lo), uhi = bits(hi);
  long bad = 0, n = 0;
  for (uint32_t u0 = ulo; u0 < uhi; u0 += CHUNK) {
    uint32_t u1 = uhi - u0 < CHUNK ? uhi : u0 + CHUNK;
    fesetround(FE_DOWNWARD);
    for (uint32_t u = u0; u < u1; ++u) {
      float a; memcpy(&a, &u, 4);
      rd_t[u - u0] = fmaf(a, 2048.0f, 8387584.5f);
      volatile float k = 8388607.5f;
      rd_f[u - u0] = a + k;
    }
    fesetround(FE_TONEAREST);
    for (uint32_t u = u0; u < u1; ++u) {
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
      if ((long)bits(rd_t[u - u0]) != 0x4B000000L + T) {
        bad++; if (bad < 10) printf("rounded-down fma a=%.9g bits=%08x T=%ld\n", a, bits(rd_t[u - u0]), T);
      }
      float fl = rd_f[u - u0];
      if ((long)bits(fl) != 0x4B000000L + x0) {
        bad++; if (bad < 10) printf("rounded-down add a=%.9g bits=%08x x0=%ld\n", a, bits(fl), x0);
      }
      volatile float kk = 8388607.5f;
      float fx = a - (fl - kk);
      if (bits(fx) != bits(f)) { bad++; if (bad < 10) printf("f32 weight a=%.9g %.9g vs %.9g\n", a, fx, f); }
      n++;
    }
  }
  printf("checked %ld values, %ld bad\n", n, bad);
  return bad != 0;
}
