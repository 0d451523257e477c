// Batched FFTs in shared memory for lengths L = 2^b or 3 * 2^b (FP32), shared by the FFT
// transform mode and the batched solver.
//
// Out-of-place Stockham stages: radix-16 stages in registers (the 16-point kernel as 4 x 4)
// while four factors of two remain, then one radix-4 and one radix-2 stage as needed, then one
// radix-3 stage when 3 divides L. A stage of radix R with sub-transform size Ns reads element
// j + r L / R (r < R), multiplies it by exp(sign 2 pi i r k / (R Ns)) with k = j mod Ns, takes
// the R-point DFT and writes output q to (j / Ns) R Ns + k + q Ns. Sequence p occupies
// [p L, (p + 1) L) of both buffers; element i lives at sw(i) = i + i / 16 (one pad entry after
// every 16: stride-16 stores then hit different banks, unit-stride accesses stay
// conflict-free). Because sw(x + m n) = sw(x) + m (n + n / 16) whenever n is a multiple of 16
// (or the m-run stays inside one 16-entry block), a stage addresses its R operands from one
// swizzled base with a fixed stride. Buffers hold span_of(n) entries for n elements.
#pragma once

#include <cuda_runtime.h>

namespace rfk {
namespace fftc {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ int sw(int i) { return i + (i >> 4); }
// distance between sw(x) and sw(x + n) for n a multiple of 16
__device__ __forceinline__ int sw_stride(int n) { return n + (n >> 4); }

// entries a buffer needs to hold n elements (even, so that buffers placed back to back keep
// 16-byte alignment)
__host__ __device__ inline int span_of(int n) { return (n + (n >> 4) + 2) & ~1; }

__host__ __device__ constexpr int ilog2(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

// twiddle entries a length needs (fewer than L)
__host__ __device__ inline int twiddle_count(int L) {
  const int p2 = (L % 3 == 0) ? L / 3 : L;
  int n = 0, Ns = 1;
  for (int R : {16, 4, 2}) {
    while (Ns * R <= p2) {
      n += (R - 1) * Ns;
      Ns *= R;
      if (R != 16) break;
    }
  }
  if (p2 != L) n += 2 * Ns;
  return n;
}

// Twiddle buffer of one length L: tab[t] = exp(+2 pi i t / L) for t < L, then (from entry
// stage_offset(L), 16-byte aligned when the buffer is) the stage-major table below, padded to an
// even count. Buffers of several lengths placed back to back keep that alignment.
__host__ __device__ inline int stage_offset(int L) { return (L + 1) & ~1; }
__host__ __device__ inline int stage_len(int L) {
  const int n = (twiddle_count(L) + 1) & ~1;
  return n < 2 ? 2 : n;
}
__host__ __device__ inline int table_len(int L) { return stage_offset(L) + stage_len(L); }

// Stage-major twiddles from tab[t] = exp(+2 pi i t / L): a stage of radix R and size Ns stores
// exp(+2 pi i r k / (R Ns)), r = 1..R-1, k < Ns, as R - 1 arrays contiguous in k (neighbouring
// threads read neighbouring words). The whole block calls it; tw may be global or shared.
__device__ inline void stage_twiddles(const float2* tab, int L, float2* tw) {
  const int p2 = (L % 3 == 0) ? L / 3 : L;
  int off = 0, Ns = 1;
  for (int R : {16, 4, 2}) {
    while (Ns * R <= p2) {
      const int step = L / (R * Ns);
      for (int i = threadIdx.x; i < (R - 1) * Ns; i += blockDim.x) {
        const int r = 1 + i / Ns, k = i - (r - 1) * Ns;
        tw[off + i] = tab[r * k * step];
      }
      off += (R - 1) * Ns;
      Ns *= R;
      if (R != 16) break;   // at most one radix-4 and one radix-2 stage
    }
  }
  if (p2 != L) {
    const int step = L / (3 * Ns);   // = 1
    for (int i = threadIdx.x; i < 2 * Ns; i += blockDim.x) {
      const int r = 1 + i / Ns, k = i - (r - 1) * Ns;
      tw[off + i] = tab[r * k * step];
    }
  }
}

// Copies the stage-major table of a twiddle buffer into shared memory (tw 16-byte aligned, room
// for stage_len(L) entries): independent 16-byte loads issued back to back, then the stores.
__device__ __forceinline__ void copy_twiddles(const float2* __restrict__ buf, int L, float2* tw) {
  const float4* src = reinterpret_cast<const float4*>(buf + stage_offset(L));
  float4* dst = reinterpret_cast<float4*>(tw);
  const int n4 = stage_len(L) / 2;
  for (int i0 = threadIdx.x; i0 < n4; i0 += 4 * blockDim.x) {
    float4 v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < n4) v[u] = __ldg(src + i);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * blockDim.x;
      if (i < n4) dst[i] = v[u];
    }
  }
}

// v0..v3 <- their 4-point DFT with kernel exp(sign 2 pi i r q / 4)
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3, int sign) {
  const float2 s02 = make_float2(a0.x + a2.x, a0.y + a2.y);
  const float2 d02 = make_float2(a0.x - a2.x, a0.y - a2.y);
  const float2 s13 = make_float2(a1.x + a3.x, a1.y + a3.y);
  const float2 d13 = make_float2(a1.x - a3.x, a1.y - a3.y);
  const float2 id13 = sign < 0 ? make_float2(d13.y, -d13.x) : make_float2(-d13.y, d13.x);
  a0 = make_float2(s02.x + s13.x, s02.y + s13.y);
  a1 = make_float2(d02.x + id13.x, d02.y + id13.y);
  a2 = make_float2(s02.x - s13.x, s02.y - s13.y);
  a3 = make_float2(d02.x - id13.x, d02.y - id13.y);
}

// 16-point DFT in registers as 4 x 4 (n = n1 + 4 n2, q = q2 + 4 q1): 4-point DFTs over n2,
// the twiddles exp(sign 2 pi i n1 q2 / 16), 4-point DFTs over n1. X[q] lands in
// v[4 (q & 3) + (q >> 2)].
__device__ __forceinline__ void dft16(float2* v, int sign) {
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) dft4(v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12], sign);
  // cos and sin of 2 pi m / 16 for m = 1, 2, 3 (exact constants of the 16-point kernel)
  const float c1 = 0.92387953251128674f, s1 = 0.38268343236508978f, h = 0.70710678118654752f;
  const float sg = sign < 0 ? -1.f : 1.f;
  const float2 w[10] = {make_float2(1.f, 0.f),  make_float2(c1, sg * s1), make_float2(h, sg * h),
                        make_float2(s1, sg * c1), make_float2(0.f, sg),    make_float2(-s1, sg * c1),
                        make_float2(-h, sg * h),  make_float2(-c1, sg * s1), make_float2(-1.f, 0.f),
                        make_float2(-c1, -sg * s1)};
#pragma unroll
  for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
    for (int q2 = 1; q2 < 4; ++q2) v[n1 + 4 * q2] = cmul(v[n1 + 4 * q2], w[n1 * q2]);
#pragma unroll
  for (int q2 = 0; q2 < 4; ++q2) dft4(v[4 * q2], v[4 * q2 + 1], v[4 * q2 + 2], v[4 * q2 + 3], sign);
}

// (p, j) of item u of a stage with q butterflies per sequence
__device__ __forceinline__ void split_item(int u, int q, bool pow2, int lq, int& p, int& j) {
  if (pow2) {
    p = u >> lq;
    j = u & (q - 1);
  } else {
    p = u / q;
    j = u - p * q;
  }
}

// Batched FFT of P sequences of length L (sign -1 forward, +1 inverse, unnormalised). Returns
// the buffer holding the result. The whole block calls it.
__device__ inline float2* fft_block(float2* in, float2* out, const float2* tw, int L, int P,
                                    int sign) {
  const bool three = (L % 3 == 0);
  const int p2 = three ? L / 3 : L;
  const int lb = ilog2(p2);
  const bool pow2 = !three;
  int off = 0;
  int ls = 0;   // log2 Ns
  while (ls + 4 <= lb) {   // radix-16
    const int Ns = 1 << ls, q = L >> 4;
    const bool lin = (q & 15) == 0;
    const int pq = sw_stride(q), pn = sw_stride(Ns);
    for (int u = threadIdx.x; u < P * q; u += blockDim.x) {
      int p, j;
      split_item(u, q, pow2, ilog2(L) - 4, p, j);
      const int base_in = p * L + j;
      float2 v[16];
      if (lin) {
        const float2* src = in + sw(base_in);
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = src[r * pq];
      } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = in[sw(base_in + r * q)];
      }
      const int k = j & (Ns - 1);
      if (ls > 0) {
#pragma unroll
        for (int r = 1; r < 16; ++r) {
          float2 w = tw[off + (r - 1) * Ns + k];
          if (sign < 0) w.y = -w.y;
          v[r] = cmul(v[r], w);
        }
      }
      dft16(v, sign);
      // Ns is 1 (base a multiple of 16) or a multiple of 16: always one base and a stride
      float2* dst = out + sw(p * L + ((j >> ls) << (ls + 4)) + k);
#pragma unroll
      for (int qq = 0; qq < 16; ++qq) dst[qq * pn] = v[4 * (qq & 3) + (qq >> 2)];
    }
    __syncthreads();
    float2* t = in;
    in = out;
    out = t;
    off += 15 * Ns;
    ls += 4;
  }
  if (ls + 2 <= lb) {   // one radix-4 stage
    const int Ns = 1 << ls, q = L >> 2;
    const bool lin = (q & 15) == 0;
    const bool lout = (Ns & 15) == 0 || (Ns == 1 && (L & 15) == 0);
    const int pq = sw_stride(q), pn = sw_stride(Ns);
    for (int u = threadIdx.x; u < P * q; u += blockDim.x) {
      int p, j;
      split_item(u, q, pow2, ilog2(L) - 2, p, j);
      const int base_in = p * L + j;
      float2 v0, v1, v2, v3;
      if (lin) {
        const float2* src = in + sw(base_in);
        v0 = src[0];
        v1 = src[pq];
        v2 = src[2 * pq];
        v3 = src[3 * pq];
      } else {
        v0 = in[sw(base_in)];
        v1 = in[sw(base_in + q)];
        v2 = in[sw(base_in + 2 * q)];
        v3 = in[sw(base_in + 3 * q)];
      }
      const int k = j & (Ns - 1);
      if (ls > 0) {
        float2 w1 = tw[off + k], w2 = tw[off + Ns + k], w3 = tw[off + 2 * Ns + k];
        if (sign < 0) {
          w1.y = -w1.y;
          w2.y = -w2.y;
          w3.y = -w3.y;
        }
        v1 = cmul(v1, w1);
        v2 = cmul(v2, w2);
        v3 = cmul(v3, w3);
      }
      dft4(v0, v1, v2, v3, sign);
      const int base = p * L + ((j >> ls) << (ls + 2)) + k;
      if (lout) {
        float2* dst = out + sw(base);
        dst[0] = v0;
        dst[pn] = v1;
        dst[2 * pn] = v2;
        dst[3 * pn] = v3;
      } else {
        out[sw(base)] = v0;
        out[sw(base + Ns)] = v1;
        out[sw(base + 2 * Ns)] = v2;
        out[sw(base + 3 * Ns)] = v3;
      }
    }
    __syncthreads();
    float2* t = in;
    in = out;
    out = t;
    off += 3 * Ns;
    ls += 2;
  }
  if (ls < lb) {   // one radix-2 stage
    const int Ns = 1 << ls, h = L >> 1;
    for (int u = threadIdx.x; u < P * h; u += blockDim.x) {
      int p, j;
      split_item(u, h, pow2, ilog2(L) - 1, p, j);
      const int base_in = p * L + j;
      float2 v0 = in[sw(base_in)], v1 = in[sw(base_in + h)];
      const int k = j & (Ns - 1);
      float2 w = tw[off + k];
      if (sign < 0) w.y = -w.y;
      v1 = cmul(v1, w);
      const int base = p * L + ((j >> ls) << (ls + 1)) + k;
      out[sw(base)] = make_float2(v0.x + v1.x, v0.y + v1.y);
      out[sw(base + Ns)] = make_float2(v0.x - v1.x, v0.y - v1.y);
    }
    __syncthreads();
    float2* t = in;
    in = out;
    out = t;
    off += Ns;
    ls += 1;
  }
  if (three) {   // one radix-3 stage, Ns = L / 3: k = j, outputs j, j + Ns, j + 2 Ns
    const int Ns = p2;
    const float hs = 0.86602540378443865f * (sign < 0 ? -1.f : 1.f);   // sign sqrt(3) / 2
    for (int u = threadIdx.x; u < P * Ns; u += blockDim.x) {
      const int p = u / Ns, j = u - p * Ns;
      const int base = p * L + j;
      float2 v0 = in[sw(base)], v1 = in[sw(base + Ns)], v2 = in[sw(base + 2 * Ns)];
      if (ls > 0) {
        float2 w1 = tw[off + j], w2 = tw[off + Ns + j];
        if (sign < 0) {
          w1.y = -w1.y;
          w2.y = -w2.y;
        }
        v1 = cmul(v1, w1);
        v2 = cmul(v2, w2);
      }
      // X0 = v0 + v1 + v2; X1,2 = v0 - (v1 + v2) / 2 +- i sign sqrt(3)/2 (v1 - v2)
      const float2 s = make_float2(v1.x + v2.x, v1.y + v2.y);
      const float2 d = make_float2(v1.x - v2.x, v1.y - v2.y);
      const float2 m = make_float2(v0.x - 0.5f * s.x, v0.y - 0.5f * s.y);
      out[sw(base)] = make_float2(v0.x + s.x, v0.y + s.y);
      out[sw(base + Ns)] = make_float2(m.x - hs * d.y, m.y + hs * d.x);
      out[sw(base + 2 * Ns)] = make_float2(m.x + hs * d.y, m.y - hs * d.x);
    }
    __syncthreads();
    in = out;
  }
  return in;
}

}  // namespace fftc
}  // namespace rfk
