// Noise models of arXiv 2505.14372 §3.1: per-pixel loss l(I) and the factor
// dl such that the detector seed is 2 dl A (float, cancellation-free forms).
//   0 amplitude / Anscombe: l = 1/2 (sqrt(I+c+eps) - sqrt(E+c+eps))^2
//   1 Poisson:              l = I - E - E log((I+eps)/(E+eps))
//   2 Gaussian:             l = (I - E)^2 / (2 c^2), c = sigma
//   3 ePIE modulus update (§3.1's optimal wavefront update, §3.3.1): l as 0;
//     2 dl = sqrt(E+c) / (eps + sqrt(I+c)) - 1, so the seed is the
//     detector-plane update chi itself.
#pragma once
#include "launch.h"

namespace ptycho {

__device__ __forceinline__ void noise_model(int model, float eps, float c, float I, float E, float& l, float& dl) {
  if (model == 0 || model == kModelEpie) {
    const float sa = sqrtf(I + c + eps), sb = sqrtf(E + c + eps);
    const float diff = (I - E) / (sa + sb);
    l = 0.5f * diff * diff;
    if (model == 0) dl = 0.5f * (1.0f - sb / sa);
    else dl = 0.5f * (sqrtf(E + c) / (eps + sqrtf(I + c)) - 1.0f);
  } else if (model == 1) {
    l = (I - E) - E * log1pf((I - E) / (E + eps));
    dl = 1.0f - E / (I + eps);
  } else {
    const float r = (I - E) / (c * c);
    l = 0.5f * r * (I - E);
    dl = r;
  }
}

}  // namespace ptycho
