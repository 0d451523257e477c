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
    // radial return: dgamma = phi / (3 mu + H), flow direction 3/2 s / sigma_eq (seq > 0 here:
    // phi > 0 and sigma_y0 > 0); one division per voxel
    const float rs = 1.f / seq;
    float dg = phi * p.r3muH;
    float fl = 1.5f * dg * rs;
    float f = 1.f - 3.f * p.mu * dg * rs;
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

// J2 state, component maps and deterministic block reductions
template <int NC>
__device__ __forceinline__ void load_state(const float* st, long long N, long long g, float* ep,
                                           float& alpha) {
  if (NC == 3) {
    ep[0] = st[g];
    ep[1] = st[N + g];
    ep[5] = st[2 * N + g];
    ep[2] = -(ep[0] + ep[1]);
    ep[3] = ep[4] = 0.f;
    alpha = st[3 * N + g];
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) ep[i] = st[i * N + g];
    alpha = st[6 * N + g];
  }
}

template <int NC>
__device__ __forceinline__ void store_state(float* st, long long N, long long g, const float* ep,
                                            float alpha) {
  if (NC == 3) {
    st[g] = ep[0];
    st[N + g] = ep[1];
    st[2 * N + g] = ep[5];
    st[3 * N + g] = alpha;
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) st[i * N + g] = ep[i];
    st[6 * N + g] = alpha;
  }
}

template <int NC>
__device__ __forceinline__ void comp_to6(const float* e, float* e6) {
  if (NC == 3) {
    e6[0] = e[0];
    e6[1] = e[1];
    e6[2] = 0.f;
    e6[3] = 0.f;
    e6[4] = 0.f;
    e6[5] = e[2];
  } else {
#pragma unroll
    for (int i = 0; i < 6; ++i) e6[i] = e[i];
  }
}

template <int NC>
__device__ __forceinline__ int comp6(int c) {
  return NC == 3 ? (c == 2 ? 5 : c) : c;
}

__device__ __forceinline__ double block_sum_d(double v, double* red) {
  // deterministic: fixed shuffle tree inside warps, fixed order across warps
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) t += red[i];
  }
  __syncthreads();
  return t;
}

__device__ __forceinline__ double block_max_d(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) t = fmax(t, red[i]);
  }
  __syncthreads();
  return t;
}

// Green operator of the isotropic reference medium applied to a symmetric tensor (Sec. 3):
//   (Gamma : t)_ij = (n_i (t n)_j + n_j (t n)_i) / (2 mu0) - c n_i n_j (n . t . n),
//   c = (lam0 + mu0) / (mu0 (lam0 + 2 mu0)), n = q / |q|.
__device__ __forceinline__ void gamma6(const float4& n, const float* t, float inv2mu0, float cg,
                                       float* o) {
  // t: (11, 22, 33, 23, 13, 12)
  const float v0 = t[0] * n.x + t[5] * n.y + t[4] * n.z;
  const float v1 = t[5] * n.x + t[1] * n.y + t[3] * n.z;
  const float v2 = t[4] * n.x + t[3] * n.y + t[2] * n.z;
  const float nvn = n.x * v0 + n.y * v1 + n.z * v2;
  o[0] = 2.f * n.x * v0 * inv2mu0 - cg * n.x * n.x * nvn;
  o[1] = 2.f * n.y * v1 * inv2mu0 - cg * n.y * n.y * nvn;
  o[2] = 2.f * n.z * v2 * inv2mu0 - cg * n.z * n.z * nvn;
  o[3] = (n.y * v2 + n.z * v1) * inv2mu0 - cg * n.y * n.z * nvn;
  o[4] = (n.x * v2 + n.z * v0) * inv2mu0 - cg * n.x * n.z * nvn;
  o[5] = (n.x * v1 + n.y * v0) * inv2mu0 - cg * n.x * n.y * nvn;
}

// Macroscopic strain E under mixed control from the zero frequency of tau (tv = tau^(0) of the
// NC components, <tau> = tau^(0) / N): E_i = target_i where the strain is prescribed; where the
// average stress is prescribed, (C0 : E)_i = target_i - <tau>_i with the other components held
// (the averaged Lippmann-Schwinger equation <sigma> = C0 : <eps> + <tau>), solved in FP64 by
// Gaussian elimination with partial pivoting. C0 acts on six-vectors with tensor shear:
// normal rows lam0 + 2 mu0 delta_ij, shear columns 2 mu0. In plane strain E_33 = E_23 = E_13 = 0.
template <int NC>
__device__ __noinline__ void mixed_macro(const float2* tv, double Nd, const Status* st, double* E) {
  double t6[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
  for (int c = 0; c < NC; ++c) t6[comp6<NC>(c)] = (double)tv[c].x / Nd;
  const double l = st->lam0, m = st->mu0;
  auto A = [&](int a, int b) -> double {
    if (a < 3 && b < 3) return l + (a == b ? 2.0 * m : 0.0);
    return a == b ? 2.0 * m : 0.0;
  };
  int P[6], np = 0;
  for (int i = 0; i < 6; ++i) {
    E[i] = st->control[i] ? 0.0 : st->target[i];
    if (NC == 3 && i >= 2 && i <= 4) E[i] = 0.0;
    if (st->control[i]) P[np++] = i;
  }
  double M[6][7];
  for (int r = 0; r < np; ++r) {
    double rhs = st->target[P[r]] - t6[P[r]];
    for (int j = 0; j < 6; ++j)
      if (!st->control[j]) rhs -= A(P[r], j) * E[j];
    for (int q = 0; q < np; ++q) M[r][q] = A(P[r], P[q]);
    M[r][np] = rhs;
  }
  for (int k = 0; k < np; ++k) {
    int piv = k;
    for (int r = k + 1; r < np; ++r)
      if (fabs(M[r][k]) > fabs(M[piv][k])) piv = r;
    if (piv != k)
      for (int q = 0; q <= np; ++q) {
        const double t = M[k][q];
        M[k][q] = M[piv][q];
        M[piv][q] = t;
      }
    for (int r = k + 1; r < np; ++r) {
      const double f = M[r][k] / M[k][k];
      for (int q = k; q <= np; ++q) M[r][q] -= f * M[k][q];
    }
  }
  for (int k = np - 1; k >= 0; --k) {
    double v = M[k][np];
    for (int q = k + 1; q < np; ++q) v -= M[k][q] * E[P[q]];
    E[P[k]] = v / M[k][k];
  }
}

// New strain coefficients at one half-pattern frequency (Sec. 4 step c) from tau^ of its NC
// components: N ebar at the zero frequency (kind 1), 0 where the operator is null (kind 2),
// otherwise eps^ = -Gamma0 : tau^ applied to the real and to the imaginary parts.
template <int NC>
__device__ __forceinline__ void green_update(int kind, const float4& n, const float2* tv,
                                             const double* ebar, double Nd, float inv2mu0,
                                             float cg, float* er, float* ei) {
  if (kind == 1) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      er[c] = (float)(Nd * ebar[comp6<NC>(c)]);
      ei[c] = 0.f;
    }
  } else if (kind == 2) {
#pragma unroll
    for (int c = 0; c < NC; ++c) er[c] = ei[c] = 0.f;
  } else {
    float tr[NC], ti[NC], t6[6], o6[6];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      tr[c] = tv[c].x;
      ti[c] = tv[c].y;
    }
    comp_to6<NC>(tr, t6);
    gamma6(n, t6, inv2mu0, cg, o6);
#pragma unroll
    for (int c = 0; c < NC; ++c) er[c] = -o6[comp6<NC>(c)];
    comp_to6<NC>(ti, t6);
    gamma6(n, t6, inv2mu0, cg, o6);
#pragma unroll
    for (int c = 0; c < NC; ++c) ei[c] = -o6[comp6<NC>(c)];
  }
}

}  // namespace rfk
