// Constitutive law of Sec. 2 on six-component tensors (11, 22, 33, 23, 13, 12), FP32:
// isotropic linear elasticity, and for plastic phases the von Mises yield function with
// linear isotropic hardening, associative flow and a closed-form radial return from the
// internal variables (eps_p, alpha) of the last converged increment. Shared by the SIMT and the
// tensor-core row kernels.
#pragma once

#include "rf_internal.cuh"

namespace rfk {

struct LawOut {
  float s[6];
  float ep[6];
  float alpha;
  bool yielded;
};

template <bool PLASTIC>
__device__ __forceinline__ void stress6(const float* e, const DevPhase& p, const float* ep,
                                        float alpha, LawOut& o) {
  bool elastic = true;
  if constexpr (PLASTIC) elastic = !p.plastic;
  if (elastic) {
    float tr = e[0] + e[1] + e[2];
    float lt = p.lam * tr;
#pragma unroll
    for (int i = 0; i < 3; ++i) o.s[i] = lt + 2.f * p.mu * e[i];
#pragma unroll
    for (int i = 3; i < 6; ++i) o.s[i] = 2.f * p.mu * e[i];
    o.yielded = false;
#pragma unroll
    for (int i = 0; i < 6; ++i) o.ep[i] = ep[i];
    o.alpha = alpha;
    return;
  }
  // trial state with the internal variables of the last converged increment
  float ee[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) ee[i] = e[i] - ep[i];
  float tre = ee[0] + ee[1] + ee[2];
  float m = tre * (1.f / 3.f);
  float s[6] = {2.f * p.mu * (ee[0] - m), 2.f * p.mu * (ee[1] - m), 2.f * p.mu * (ee[2] - m),
                2.f * p.mu * ee[3], 2.f * p.mu * ee[4], 2.f * p.mu * ee[5]};
  float ss = s[0] * s[0] + s[1] * s[1] + s[2] * s[2] +
             2.f * (s[3] * s[3] + s[4] * s[4] + s[5] * s[5]);
  float seq = sqrtf(1.5f * ss);
  float phi = seq - (p.sy + p.H * alpha);
  float pm = (p.lam + (2.f / 3.f) * p.mu) * tre;
  if (phi > 0.f) {
    // radial return: dgamma = phi / (3 mu + H), flow direction 3/2 s / sigma_eq
    float dg = phi / (3.f * p.mu + p.H);
    float fl = 1.5f * dg / seq;
    float f = 1.f - 3.f * p.mu * dg / seq;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      o.ep[i] = ep[i] + fl * s[i];
      s[i] *= f;
    }
    o.alpha = alpha + dg;
    o.yielded = true;
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) o.ep[i] = ep[i];
    o.alpha = alpha;
    o.yielded = false;
  }
  o.s[0] = s[0] + pm;
  o.s[1] = s[1] + pm;
  o.s[2] = s[2] + pm;
  o.s[3] = s[3];
  o.s[4] = s[4];
  o.s[5] = s[5];
}

}  // namespace rfk
