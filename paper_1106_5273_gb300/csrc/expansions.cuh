// FP32 normalized regular harmonics for P2M / L2P (see harmonics.cuh).
#pragma once
#include "common.cuh"

namespace fmm {

// R~_n^m(x,y,z), n < p, m >= 0, written to re[cidx], im[cidx].
__device__ inline void regular_table_f(float x, float y, float z, int p, float* re, float* im) {
  const float r2 = x * x + y * y + z * z;
  re[0] = 1.f;
  im[0] = 0.f;
  for (int m = 1; m < p; ++m) {
    int pc = (m - 1) * m / 2 + (m - 1), c = m * (m + 1) / 2 + m;
    float f = sqrtf((2.f * m - 1.f) / (2.f * m));
    re[c] = f * (re[pc] * x - im[pc] * y);
    im[c] = f * (re[pc] * y + im[pc] * x);
  }
  for (int m = 0; m < p; ++m) {
    for (int n = m + 1; n < p; ++n) {
      int c = n * (n + 1) / 2 + m, c1 = (n - 1) * n / 2 + m;
      float inv = rsqrtf((float)((n + m) * (n - m)));
      float a = (2.f * n - 1.f) * z;
      float vr = a * re[c1], vi = a * im[c1];
      if (n - 2 >= m) {
        int c2 = (n - 2) * (n - 1) / 2 + m;
        float b = r2 * sqrtf((float)((n + m - 1) * (n - m - 1)));
        vr -= b * re[c2];
        vi -= b * im[c2];
      }
      re[c] = vr * inv;
      im[c] = vi * inv;
    }
  }
}

}  // namespace fmm
