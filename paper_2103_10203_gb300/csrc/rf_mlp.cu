// Learned warm start: a three-layer GELU perceptron maps 48 descriptors of an RVE's phase
// indicator to a real strain-transfer expansion over 27 angular/radial basis functions; the
// head evaluates the transfer at every slot (frequency of the kx >= 0 half of the pattern) and
// multiplies it with gamma(k) and the macroscopic strain direction, the structure of the
// scheme's first update (Sec. 4 step c on the plain start). Inference and training kernels.
//
// GEMM C[M][N] = sum_k A(m, k) B(k, n) on the tensor cores (tcgen05): one 128 x 128 output tile
// per CTA of 128 threads, accumulated in 128 FP32 tensor-memory columns. K is staged in
// 128-byte chunks (64 BF16 or 32 TF32 values per row) through two shared-memory buffers in the
// no-swizzle K-major core-matrix layout: all threads load and convert chunk g + 1 from FP32
// global memory while the MMAs of chunk g run; one thread issues the MMAs and commits them to
// the buffer's mbarrier. Either operand may be K-contiguous or M/N-contiguous in global memory
// (the transposes of the backward pass); the conversion step writes the canonical layout.
// Epilogues fuse bias, GELU (storing the pre-activation for the backward pass) and GELU'.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/rf_mlp.h"
#include "rf_internal.cuh"
#include "rf_tcgen05.cuh"

namespace rfk {
namespace mlp {

using tc::cm_off;
using tc::EBf16;
using tc::ETf32;
using tc::smem_u32;

constexpr int kTM = 128;                 // output rows per tile (tensor-memory lanes)
constexpr int kTN = 128;                 // output columns per tile (tensor-memory columns)
constexpr int kChunk = 128;              // K bytes per staged chunk row
constexpr int kTileBytes = kTM * kChunk; // 16 KB per operand chunk
constexpr size_t kGemmSmem = 4 * kTileBytes + 64;

enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_DGELU = 3 };

struct GemmArgs {
  const float* A;
  long long lda;     // A(m, k) = AK ? A[m lda + k] : A[k lda + m]
  const float* B;
  long long ldb;     // B(k, n) = BK ? B[n ldb + k] : B[k ldb + n]
  float* C;
  long long ldc;
  const float* bias; // [N]
  const float* Zin;  // EPI_DGELU: pre-activation [M][ldz]
  float* Zout;       // EPI_BIAS_GELU: pre-activation out (nullable)
  long long ldz;
  int M, N, K;
  int* err;
};

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.f + erff(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// four consecutive K values of one row into the core-matrix tile (kbyte a multiple of 4 E)
template <class E>
__device__ __forceinline__ void put4(unsigned char* tile, int row, int k, float4 v) {
  const uint32_t off = cm_off(row, k * E::kBytes, kChunk);
  if constexpr (E::kBytes == 2) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
    __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
    uint2 u;
    u.x = *reinterpret_cast<uint32_t*>(&a);
    u.y = *reinterpret_cast<uint32_t*>(&b);
    *reinterpret_cast<uint2*>(tile + off) = u;
  } else {
    uint4 u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u.x) : "f"(v.x));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u.y) : "f"(v.y));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u.z) : "f"(v.z));
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u.w) : "f"(v.w));
    *reinterpret_cast<uint4*>(tile + off) = u;
  }
}

template <class E>
__device__ __forceinline__ void put1(unsigned char* tile, int row, int k, float v) {
  const uint32_t off = cm_off(row, k * E::kBytes, kChunk);
  if constexpr (E::kBytes == 2) {
    *reinterpret_cast<__nv_bfloat16*>(tile + off) = __float2bfloat16_rn(v);
  } else {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(v));
    *reinterpret_cast<uint32_t*>(tile + off) = u;
  }
}

// Stage rows [r0, r0 + 128) x K chunk [k0, k0 + per) of an operand. KC: the operand is
// K-contiguous (element (row, k) at src[row ld + k]), else row-contiguous (src[k ld + row]).
// Out-of-range elements are zero. ld and the base are multiples of 4 floats (checked on the
// host), so every float4 below starts inside its row and is 16-byte aligned.
template <class E, bool KC>
__device__ __forceinline__ void stage(unsigned char* tile, const float* __restrict__ src,
                                      long long ld, int rows, int r0, int K, int k0) {
  constexpr int per = kChunk / E::kBytes;
  constexpr int items = kTM * per / 4 / 128;   // float4 per thread
  float4 v[items];
  if constexpr (KC) {
#pragma unroll
    for (int i = 0; i < items; ++i) {
      const int it = threadIdx.x + i * 128;
      const int r = it / (per / 4), k = k0 + 4 * (it % (per / 4));
      const int row = r0 + r;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row < rows && k < K) {
        x = __ldg(reinterpret_cast<const float4*>(src + (long long)row * ld + k));
        if (k + 1 >= K) x.y = 0.f;
        if (k + 2 >= K) x.z = 0.f;
        if (k + 3 >= K) x.w = 0.f;
      }
      v[i] = x;
    }
#pragma unroll
    for (int i = 0; i < items; ++i) {
      const int it = threadIdx.x + i * 128;
      put4<E>(tile, it / (per / 4), 4 * (it % (per / 4)), v[i]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < items; ++i) {
      const int it = threadIdx.x + i * 128;
      const int kk = it / (kTM / 4), r = 4 * (it % (kTM / 4));
      const int k = k0 + kk, row = r0 + r;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (k < K && row < rows) {
        x = __ldg(reinterpret_cast<const float4*>(src + (long long)k * ld + row));
        if (row + 1 >= rows) x.y = 0.f;
        if (row + 2 >= rows) x.z = 0.f;
        if (row + 3 >= rows) x.w = 0.f;
      }
      v[i] = x;
    }
#pragma unroll
    for (int i = 0; i < items; ++i) {
      const int it = threadIdx.x + i * 128;
      const int kk = it / (kTM / 4), r = 4 * (it % (kTM / 4));
      put1<E>(tile, r + 0, kk, v[i].x);
      put1<E>(tile, r + 1, kk, v[i].y);
      put1<E>(tile, r + 2, kk, v[i].z);
      put1<E>(tile, r + 3, kk, v[i].w);
    }
  }
}

template <class E, bool AK, bool BK, int EPI>
__global__ __launch_bounds__(128) void k_gemm(GemmArgs g) {
  constexpr int per = kChunk / E::kBytes;
  extern __shared__ __align__(1024) unsigned char smem[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + 4 * kTileBytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
  int* s_err = reinterpret_cast<int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int n0 = blockIdx.x * kTN, m0 = blockIdx.y * kTM;

  if (tid == 0) {
    tc::mbar_init(&bars[0], 1);
    tc::mbar_init(&bars[1], 1);
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)),
                 "r"(kTN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const uint32_t id = tc::idesc<E>(kTM, kTN);
  const int nch = (g.K + per - 1) / per;
  bool ok = true;

  for (int c = 0; c < nch; ++c) {
    const int b = c & 1;
    unsigned char* As = smem + b * 2 * kTileBytes;
    unsigned char* Bs = As + kTileBytes;
    // buffer b is free once the MMAs of chunk c - 2 completed
    if (c >= 2 && !tc::mbar_wait(&bars[b], ((c - 2) >> 1) & 1)) atomicOr(s_err, 1);
    stage<E, AK>(As, g.A, g.lda, g.M, m0, g.K, c * per);
    stage<E, BK>(Bs, g.B, g.ldb, g.N, n0, g.K, c * per);
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    ok = (*s_err == 0);
    if (!ok) break;   // uniform: read after the same barrier by every thread
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
      for (int s = 0; s < kChunk / 32; ++s) {
        const uint64_t da = tc::make_desc(a0 + s * 256, 128, (kChunk / 16) * 128);
        const uint64_t db = tc::make_desc(b0 + s * 256, 128, (kChunk / 16) * 128);
        tc::mma<E>(tmem, da, db, id, (c > 0 || s > 0) ? 1u : 0u);
      }
      tc::mma_commit(&bars[b]);
    }
  }
  if (ok && nch > 0) {
    const int cl = nch - 1;
    if (!tc::mbar_wait(&bars[cl & 1], (cl >> 1) & 1)) atomicOr(s_err, 1);
  }
  __syncthreads();
  ok = (*s_err == 0);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int m = m0 + tid;
    const uint32_t lane = (uint32_t)(32 * warp) << 16;
    for (int c0 = 0; c0 < kTN && n0 + c0 < g.N; c0 += 16) {   // uniform across the CTA
      float v[16];
      tc::tmem_ld16(tmem + lane + c0, v);
      if (m >= g.M) continue;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int n = n0 + c0 + i;
        if (n >= g.N) break;
        float x = v[i];
        if constexpr (EPI == EPI_BIAS) x += g.bias[n];
        if constexpr (EPI == EPI_BIAS_GELU) {
          x += g.bias[n];
          if (g.Zout) g.Zout[(long long)m * g.ldz + n] = x;
          x = gelu(x);
        }
        if constexpr (EPI == EPI_DGELU) x *= gelu_grad(g.Zin[(long long)m * g.ldz + n]);
        g.C[(long long)m * g.ldc + n] = x;
      }
    }
  }
  __syncthreads();
  asm volatile("tcgen05.fence::before_thread_sync;");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTN));
  if (!ok && tid == 0) atomicOr(g.err, 1);
}

// ------------------------------------------------------------------------------------------
// head over the slots (one CTA per RVE; the RVE's 243 coefficients staged in shared memory)
constexpr int kBasis = RF_MLP_BASIS;
constexpr int kOut = RF_MLP_OUT;

__device__ __forceinline__ void unit_dir(const double* mac, float e[3], double* en_out) {
  const double en = sqrt(mac[0] * mac[0] + mac[1] * mac[1] + mac[2] * mac[2] +
                         2.0 * (mac[3] * mac[3] + mac[4] * mac[4] + mac[5] * mac[5]));
  const double inv = en > 0.0 ? 1.0 / en : 0.0;
  e[0] = (float)(mac[0] * inv);
  e[1] = (float)(mac[1] * inv);
  e[2] = (float)(mac[5] * inv);
  if (en_out) *en_out = en;
}

// phi_n(a, b), n = 9 i + j: radial (1, 4 rho, 16 rho^2) x (1, cos 2t, sin 2t, ..., sin 8t) from
// the rational forms of the harmonics; (a, b) != 0
__device__ __forceinline__ void basis27(float a, float b, float* phi) {
  const float r2 = a * a + b * b;
  const float inv = 1.f / r2;
  const float c2 = (a * a - b * b) * inv, s2 = 2.f * a * b * inv;
  const float c4 = c2 * c2 - s2 * s2, s4 = 2.f * s2 * c2;
  const float c6 = c4 * c2 - s4 * s2, s6 = s4 * c2 + c4 * s2;
  const float c8 = c4 * c4 - s4 * s4, s8 = 2.f * s4 * c4;
  const float h[9] = {1.f, c2, s2, c4, s4, c6, s6, c8, s8};
  const float rho = 4.f * sqrtf(r2);
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    phi[j] = h[j];
    phi[9 + j] = h[j] * rho;
    phi[18 + j] = h[j] * rho * rho;
  }
}

// T_cd = sum_n C[cd][n] phi_n (C in shared memory, [9][27])
__device__ __forceinline__ void transfer9(const float* C, const float* phi, float* T) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    float t = 0.f;
#pragma unroll
    for (int n = 0; n < kBasis; ++n) t = fmaf(C[k * kBasis + n], phi[n], t);
    T[k] = t;
  }
}

// per RVE: squared-error and weight partials; per slot dT[cd] = w (Re(conj(res_c) g)) e_d,
// unscaled (the 2 / count factor is applied in k_slot_reduce)
__global__ __launch_bounds__(128) void k_slot_loss(const float* __restrict__ O, long long ldo,
                                                   const float* __restrict__ E,
                                                   const rf_slot* __restrict__ slots,
                                                   const long long* __restrict__ off,
                                                   const float* __restrict__ T, float* dT,
                                                   long long base, double* part) {
  __shared__ float C[kOut];
  __shared__ double red[2][4];
  const int r = blockIdx.x;
  for (int i = threadIdx.x; i < kOut; i += blockDim.x) C[i] = O[(long long)r * ldo + i];
  __syncthreads();
  const float e0 = E[3 * r], e1 = E[3 * r + 1], e2 = E[3 * r + 2];
  const long long s0 = off[r], s1 = off[r + 1];
  double sq = 0.0, wsum = 0.0;
  for (long long s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
    const rf_slot sl = slots[s];
    float* d = dT + (s - base) * 9;
    if (sl.weight == 0.f) {
#pragma unroll
      for (int k = 0; k < 9; ++k) d[k] = 0.f;
      continue;
    }
    float phi[kBasis], Tf[9];
    basis27(sl.a, sl.b, phi);
    transfer9(C, phi, Tf);
    const float* t = T + s * 6;
    float rr[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float m = Tf[c * 3] * e0 + Tf[c * 3 + 1] * e1 + Tf[c * 3 + 2] * e2;
      const float pr = m * sl.g_re - t[2 * c], pi = m * sl.g_im - t[2 * c + 1];
      sq += (double)sl.weight * ((double)pr * pr + (double)pi * pi);
      rr[c] = sl.weight * (pr * sl.g_re + pi * sl.g_im);
    }
    wsum += 6.0 * sl.weight;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      d[c * 3] = rr[c] * e0;
      d[c * 3 + 1] = rr[c] * e1;
      d[c * 3 + 2] = rr[c] * e2;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sq += __shfl_down_sync(0xffffffffu, sq, o);
    wsum += __shfl_down_sync(0xffffffffu, wsum, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sq;
    red[1][threadIdx.x >> 5] = wsum;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    part[2 * r] = red[0][0] + red[0][1] + red[0][2] + red[0][3];
    part[2 * r + 1] = red[1][0] + red[1][1] + red[1][2] + red[1][3];
  }
}

// loss = sum sq / sum w; scal[0] = 2 / sum w (gradient scale), scal[1] = loss
__global__ void k_loss_total(const double* part, int B, double* scal) {
  __shared__ double a[256], b[256];
  double x = 0.0, y = 0.0;
  for (int i = threadIdx.x; i < B; i += blockDim.x) {
    x += part[2 * i];
    y += part[2 * i + 1];
  }
  a[threadIdx.x] = x;
  b[threadIdx.x] = y;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      a[threadIdx.x] += a[threadIdx.x + s];
      b[threadIdx.x] += b[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    scal[0] = b[0] > 0.0 ? 2.0 / b[0] : 0.0;
    scal[1] = b[0] > 0.0 ? a[0] / b[0] : 0.0;
  }
}

// dO[r][cd 27 + n] = (2 / count) sum over the RVE's slots of dT[cd] phi_n (fixed order)
__global__ __launch_bounds__(256) void k_slot_reduce(const rf_slot* __restrict__ slots,
                                                     const long long* __restrict__ off,
                                                     const float* __restrict__ dT,
                                                     long long base, const double* scal,
                                                     float* dO, long long ldo) {
  constexpr int kSlots = 64;
  __shared__ float ph[kSlots][kBasis + 1];
  __shared__ float dt[kSlots][9];
  const int r = blockIdx.x;
  const long long s0 = off[r], s1 = off[r + 1];
  const int k = threadIdx.x / kBasis, n = threadIdx.x % kBasis;   // k < 9 for threads < 243
  float acc = 0.f;
  for (long long c0 = s0; c0 < s1; c0 += kSlots) {
    const int m = (int)min((long long)kSlots, s1 - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const rf_slot sl = slots[c0 + i];
      if (sl.weight != 0.f) {
        basis27(sl.a, sl.b, ph[i]);
      } else {
        for (int q = 0; q < kBasis; ++q) ph[i][q] = 0.f;
      }
    }
    for (int i = threadIdx.x; i < m * 9; i += blockDim.x)
      dt[i / 9][i % 9] = dT[(c0 - base + i / 9) * 9 + i % 9];
    __syncthreads();
    if (threadIdx.x < kOut)
      for (int i = 0; i < m; ++i) acc = fmaf(dt[i][k], ph[i][n], acc);
  }
  if (threadIdx.x < kOut) dO[(long long)r * ldo + threadIdx.x] = (float)(scal[0] * (double)acc);
}

// db[n] = sum_b D[b][n]
__global__ void k_colsum(const float* __restrict__ D, long long ld, int B, int N, float* db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += D[(long long)b * ld + n];
  db[n] = s;
}

// Adam over the flat parameter buffer (bias corrections c1 = 1 / (1 - beta1^t), c2 likewise)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, long long n, float lr, float c1, float c2) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

// targets t[s][2c + part] = coeff[s][c][part] / (N |ebar|); unit directions e[r]
__global__ void k_slot_targets(const double* __restrict__ macro, const rf_slot* __restrict__ slots,
                               const long long* __restrict__ off,
                               const float* __restrict__ coeffs, float* t, float* E) {
  const int r = blockIdx.x;
  float e[3];
  double en;
  unit_dir(macro + 6LL * r, e, &en);
  if (threadIdx.x < 3) E[3 * r + threadIdx.x] = e[threadIdx.x];
  const float inv_en = en > 0.0 ? (float)(1.0 / en) : 0.f;
  for (long long s = off[r] + threadIdx.x; s < off[r + 1]; s += blockDim.x) {
    const float sc = slots[s].weight != 0.f ? slots[s].inv_n * inv_en : 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) t[s * 6 + i] = coeffs[s * 6 + i] * sc;
  }
}

// warm[s][c][part] = N |ebar| p_c at regular slots, 0 elsewhere
__global__ __launch_bounds__(128) void k_slot_predict(const float* __restrict__ O, long long ldo,
                                                      const double* __restrict__ macro,
                                                      const rf_slot* __restrict__ slots,
                                                      const long long* __restrict__ off,
                                                      float* warm) {
  __shared__ float C[kOut];
  const int r = blockIdx.x;
  for (int i = threadIdx.x; i < kOut; i += blockDim.x) C[i] = O[(long long)r * ldo + i];
  __syncthreads();
  float e[3];
  double en;
  unit_dir(macro + 6LL * r, e, &en);
  for (long long s = off[r] + threadIdx.x; s < off[r + 1]; s += blockDim.x) {
    const rf_slot sl = slots[s];
    float* w = warm + s * 6;
    if (sl.weight == 0.f) {
#pragma unroll
      for (int i = 0; i < 6; ++i) w[i] = 0.f;
      continue;
    }
    float phi[kBasis], Tf[9];
    basis27(sl.a, sl.b, phi);
    transfer9(C, phi, Tf);
    const float sc = (float)(en / (double)sl.inv_n);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float m = sc * (Tf[c * 3] * e[0] + Tf[c * 3 + 1] * e[1] + Tf[c * 3 + 2] * e[2]);
      w[2 * c] = m * sl.g_re;
      w[2 * c + 1] = m * sl.g_im;
    }
  }
}

}  // namespace mlp
}  // namespace rfk

// ------------------------------------------------------------------------------------------
// host side
using namespace rfk;
using namespace rfk::mlp;

struct rf_mlp {
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int in = RF_MLP_IN, H = 0, out = RF_MLP_OUT, out_ld = (RF_MLP_OUT + 3) & ~3, maxB = 0;
  long long n_params = 0;
  // padded device layout: offsets (floats) of W1, b1, W2, b2, W3, b3; total size
  long long off[6] = {0, 0, 0, 0, 0, 0};
  long long total = 0;
  float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr;
  float *d_Z1 = nullptr, *d_H1 = nullptr, *d_Z2 = nullptr, *d_H2 = nullptr, *d_O = nullptr;
  float *d_dZ1 = nullptr, *d_dZ2 = nullptr;
  double* d_part = nullptr;   // [maxB][2] loss partials
  double* d_scal = nullptr;   // [0] gradient scale 2 / count, [1] loss
  float* d_dT = nullptr;      // [slots][9] per-slot transfer gradients (grown on demand)
  long long dT_cap = 0;
  int* d_err = nullptr;
  double* h_scal = nullptr;   // pinned
  int* h_err = nullptr;       // pinned
  long long adam_t = 0;
  long long launches = 0;
};

namespace {

int mfail(const char* msg, int code = RF_ERR_INVALID) {
  set_error(msg);
  return code;
}

int launched(rf_mlp* n, const char* what) {
  n->launches += 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RF_OK : cuda_fail(e, what);
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <class E, bool AK, bool BK, int EPI>
int gemm(rf_mlp* n, const GemmArgs& a) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_gemm<E, AK, BK, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)kGemmSmem);
    attr = true;
  }
  if (a.M < 1 || a.N < 1 || a.K < 1) return mfail("mlp gemm: empty operand");
  if ((a.lda & 3) || (a.ldb & 3) || !aligned16(a.A) || !aligned16(a.B))
    return mfail("mlp gemm: operands must be 16-byte aligned with leading dimensions % 4 == 0");
  dim3 grid((a.N + kTN - 1) / kTN, (a.M + kTM - 1) / kTM);
  k_gemm<E, AK, BK, EPI><<<grid, 128, kGemmSmem, n->stream>>>(a);
  return launched(n, "mlp gemm");
}

GemmArgs args(const float* A, long long lda, const float* B, long long ldb, float* C,
              long long ldc, int M, int N, int K, int* err) {
  GemmArgs g{};
  g.A = A;
  g.lda = lda;
  g.B = B;
  g.ldb = ldb;
  g.C = C;
  g.ldc = ldc;
  g.M = M;
  g.N = N;
  g.K = K;
  g.err = err;
  return g;
}

// forward through the three layers into d_O [B][out_ld]; Z1/Z2 kept when `keep` (training)
template <class E>
int forward(rf_mlp* n, int B, const float* x, bool keep) {
  const float* W1 = n->d_p + n->off[0];
  const float* b1 = n->d_p + n->off[1];
  const float* W2 = n->d_p + n->off[2];
  const float* b2 = n->d_p + n->off[3];
  const float* W3 = n->d_p + n->off[4];
  const float* b3 = n->d_p + n->off[5];
  GemmArgs g = args(x, n->in, W1, n->H, n->d_H1, n->H, B, n->H, n->in, n->d_err);
  g.bias = b1;
  g.Zout = keep ? n->d_Z1 : nullptr;
  g.ldz = n->H;
  if (int e = gemm<E, true, false, EPI_BIAS_GELU>(n, g)) return e;
  g = args(n->d_H1, n->H, W2, n->H, n->d_H2, n->H, B, n->H, n->H, n->d_err);
  g.bias = b2;
  g.Zout = keep ? n->d_Z2 : nullptr;
  g.ldz = n->H;
  if (int e = gemm<E, true, false, EPI_BIAS_GELU>(n, g)) return e;
  g = args(n->d_H2, n->H, W3, n->out_ld, n->d_O, n->out_ld, B, n->out, n->H, n->d_err);
  g.bias = b3;
  return gemm<E, true, false, EPI_BIAS>(n, g);
}

int sync_read(rf_mlp* n) {
  cudaError_t e = cudaMemcpyAsync(n->h_scal, n->d_scal, 2 * sizeof(double),
                                  cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(n->h_err, n->d_err, sizeof(int), cudaMemcpyDeviceToHost, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return cuda_fail(e, "mlp readback");
  if (*n->h_err)
    return mfail("a bounded device-side wait ran out in the network GEMM", RF_ERR_TIMEOUT);
  return RF_OK;
}

int slot_args_ok(rf_mlp* n, int B, const void* slots, const int64_t* off, bool train) {
  if (!slots || !off) return mfail("network: null slot table or offsets");
  if (B < 1 || (train && B > n->maxB)) return mfail("network: B must be in [1, max_batch]");
  return RF_OK;
}

}  // namespace

extern "C" {

int rf_mlp_create(rf_mlp** out, int32_t n_hidden, int32_t max_batch, void* stream) {
  set_error("");
  if (!out) return mfail("rf_mlp_create: null output");
  *out = nullptr;
  if (n_hidden < 16 || n_hidden > 4096 || n_hidden % 16 || max_batch < 1 || max_batch > 65536)
    return mfail("rf_mlp_create: n_hidden % 16 == 0 in [16, 4096], max_batch in [1, 65536]");
  rf_mlp* n = new rf_mlp();
  cudaGetDevice(&n->dev);
  n->stream = static_cast<cudaStream_t>(stream);
  if (!n->stream) {
    cudaStreamCreateWithFlags(&n->stream, cudaStreamNonBlocking);
    n->own_stream = true;
  }
  n->H = n_hidden;
  n->maxB = max_batch;
  n->n_params = (long long)n->in * n->H + n->H + (long long)n->H * n->H + n->H +
                (long long)n->H * n->out + n->out;
  const long long sizes[6] = {(long long)n->in * n->H, n->H, (long long)n->H * n->H, n->H,
                              (long long)n->H * n->out_ld, n->out_ld};
  long long o = 0;
  for (int i = 0; i < 6; ++i) {
    n->off[i] = o;
    o += (sizes[i] + 3) & ~3LL;
  }
  n->total = o;
  const long long bh = (long long)max_batch * n->H, bo = (long long)max_batch * n->out_ld;
  bool okm = true;
  auto al = [&](auto** p, long long count) {
    if (!okm) return;
    if (cudaMalloc(p, sizeof(**p) * std::max(count, 1LL)) != cudaSuccess) okm = false;
  };
  al(&n->d_p, n->total);
  al(&n->d_g, n->total);
  al(&n->d_m, n->total);
  al(&n->d_v, n->total);
  al(&n->d_Z1, bh);
  al(&n->d_H1, bh);
  al(&n->d_Z2, bh);
  al(&n->d_H2, bh);
  al(&n->d_dZ1, bh);
  al(&n->d_dZ2, bh);
  al(&n->d_O, bo);
  al(&n->d_part, 2LL * max_batch);
  al(&n->d_scal, 2);
  al(&n->d_err, 1);
  if (okm && cudaMallocHost(&n->h_scal, 2 * sizeof(double)) != cudaSuccess) okm = false;
  if (okm && cudaMallocHost(&n->h_err, sizeof(int)) != cudaSuccess) okm = false;
  if (!okm) {
    rf_mlp_destroy(n);
    return mfail("rf_mlp_create: out of device memory", RF_ERR_OOM);
  }
  *n->h_err = 0;
  cudaMemsetAsync(n->d_p, 0, sizeof(float) * n->total, n->stream);
  cudaMemsetAsync(n->d_g, 0, sizeof(float) * n->total, n->stream);
  cudaMemsetAsync(n->d_m, 0, sizeof(float) * n->total, n->stream);
  cudaMemsetAsync(n->d_v, 0, sizeof(float) * n->total, n->stream);
  cudaMemsetAsync(n->d_O, 0, sizeof(float) * bo, n->stream);
  cudaMemsetAsync(n->d_scal, 0, 2 * sizeof(double), n->stream);
  cudaMemsetAsync(n->d_err, 0, sizeof(int), n->stream);
  if (cudaError_t e = cudaStreamSynchronize(n->stream); e != cudaSuccess) {
    rf_mlp_destroy(n);
    return cuda_fail(e, "rf_mlp_create");
  }
  *out = n;
  return RF_OK;
}

int rf_mlp_get_dims(const rf_mlp* n, rf_mlp_dims* d) {
  if (!n || !d) return mfail("rf_mlp_get_dims: null argument");
  d->n_in = n->in;
  d->n_hidden = n->H;
  d->n_out = n->out;
  d->max_batch = n->maxB;
  d->n_params = n->n_params;
  d->adam_steps = n->adam_t;
  return RF_OK;
}

// compact host layout <-> padded device layout
static void pack(const rf_mlp* n, const float* src, std::vector<float>& dst) {
  dst.assign(n->total, 0.f);
  long long s = 0;
  const long long rows[6] = {n->in, 1, n->H, 1, n->H, 1};
  const long long cols[6] = {n->H, n->H, n->H, n->H, n->out, n->out};
  const long long ld[6] = {n->H, n->H, n->H, n->H, n->out_ld, n->out_ld};
  for (int i = 0; i < 6; ++i)
    for (long long r = 0; r < rows[i]; ++r) {
      std::memcpy(&dst[n->off[i] + r * ld[i]], src + s, sizeof(float) * cols[i]);
      s += cols[i];
    }
}

static void unpack(const rf_mlp* n, const std::vector<float>& src, float* dst) {
  long long s = 0;
  const long long rows[6] = {n->in, 1, n->H, 1, n->H, 1};
  const long long cols[6] = {n->H, n->H, n->H, n->H, n->out, n->out};
  const long long ld[6] = {n->H, n->H, n->H, n->H, n->out_ld, n->out_ld};
  for (int i = 0; i < 6; ++i)
    for (long long r = 0; r < rows[i]; ++r) {
      std::memcpy(dst + s, &src[n->off[i] + r * ld[i]], sizeof(float) * cols[i]);
      s += cols[i];
    }
}

int rf_mlp_set_params(rf_mlp* n, const float* params) {
  if (!n || !params) return mfail("rf_mlp_set_params: null argument");
  std::vector<float> h;
  pack(n, params, h);
  cudaError_t e = cudaMemcpyAsync(n->d_p, h.data(), sizeof(float) * n->total,
                                  cudaMemcpyHostToDevice, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->d_m, 0, sizeof(float) * n->total, n->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->d_v, 0, sizeof(float) * n->total, n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return cuda_fail(e, "rf_mlp_set_params");
  n->adam_t = 0;
  return RF_OK;
}

static int get_flat(const rf_mlp* n, const float* d, float* out, const char* what) {
  if (!n || !out) return mfail("rf_mlp_get: null argument");
  std::vector<float> h(n->total);
  cudaError_t e = cudaMemcpyAsync(h.data(), d, sizeof(float) * n->total, cudaMemcpyDeviceToHost,
                                  n->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->stream);
  if (e != cudaSuccess) return cuda_fail(e, what);
  unpack(n, h, out);
  return RF_OK;
}

int rf_mlp_get_params(const rf_mlp* n, float* params) {
  return get_flat(n, n ? n->d_p : nullptr, params, "rf_mlp_get_params");
}

int rf_mlp_get_grads(const rf_mlp* n, float* grads) {
  return get_flat(n, n ? n->d_g : nullptr, grads, "rf_mlp_get_grads");
}

int rf_mlp_forward(rf_mlp* n, int32_t B, const float* d_x, float* d_out, int32_t precision) {
  if (!n || !d_x || !d_out) return mfail("rf_mlp_forward: null argument");
  if (B < 1 || B > n->maxB) return mfail("rf_mlp_forward: B must be in [1, max_batch]");
  if (!aligned16(d_x)) return mfail("rf_mlp_forward: d_x must be 16-byte aligned");
  int e = precision == RF_MLP_TF32 ? forward<ETf32>(n, B, d_x, false)
          : precision == RF_MLP_BF16 ? forward<EBf16>(n, B, d_x, false)
                                     : mfail("rf_mlp_forward: unknown precision");
  if (e) return e;
  cudaError_t ce = cudaMemcpy2DAsync(d_out, sizeof(float) * n->out, n->d_O,
                                     sizeof(float) * n->out_ld, sizeof(float) * n->out, B,
                                     cudaMemcpyDeviceToDevice, n->stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "rf_mlp_forward");
  return sync_read(n);
}

int rf_mlp_targets(rf_mlp* n, int32_t B, const double* d_macro, const rf_slot* d_slots,
                   const int64_t* d_offsets, const float* d_coeffs, float* d_t, float* d_e) {
  if (!n || !d_macro || !d_coeffs || !d_t || !d_e) return mfail("rf_mlp_targets: null argument");
  if (int e = slot_args_ok(n, B, d_slots, d_offsets, false)) return e;
  k_slot_targets<<<B, 128, 0, n->stream>>>(d_macro, d_slots,
                                            reinterpret_cast<const long long*>(d_offsets),
                                            d_coeffs, d_t, d_e);
  return launched(n, "rf_mlp_targets");
}

int rf_mlp_loss_grad(rf_mlp* n, int32_t B, const float* d_x, const float* d_e,
                     const rf_slot* d_slots, const int64_t* d_offsets, const float* d_t,
                     double* loss) {
  if (!n || !d_x || !d_e || !d_t) return mfail("rf_mlp_loss_grad: null argument");
  if (int e = slot_args_ok(n, B, d_slots, d_offsets, true)) return e;
  if (!aligned16(d_x)) return mfail("rf_mlp_loss_grad: d_x must be 16-byte aligned");
  const long long* off = reinterpret_cast<const long long*>(d_offsets);
  // slots of this minibatch (host read of the two end offsets sizes the scratch)
  long long ends[2] = {0, 0};
  cudaError_t ce = cudaMemcpyAsync(&ends[0], off, sizeof(long long), cudaMemcpyDeviceToHost,
                                   n->stream);
  if (ce == cudaSuccess)
    ce = cudaMemcpyAsync(&ends[1], off + B, sizeof(long long), cudaMemcpyDeviceToHost, n->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(n->stream);
  if (ce != cudaSuccess) return cuda_fail(ce, "rf_mlp_loss_grad offsets");
  const long long nslots = ends[1] - ends[0];
  if (nslots < 0) return mfail("rf_mlp_loss_grad: offsets must not decrease");
  if (nslots > n->dT_cap) {
    if (n->d_dT) cudaFree(n->d_dT);
    n->d_dT = nullptr;
    n->dT_cap = 0;
    const long long cap = std::max(nslots + nslots / 4, 1LL << 16);
    if (cudaMalloc(&n->d_dT, sizeof(float) * 9 * cap) != cudaSuccess)
      return mfail("rf_mlp_loss_grad: out of device memory", RF_ERR_OOM);
    n->dT_cap = cap;
  }
  if (int e = forward<ETf32>(n, B, d_x, true)) return e;
  k_slot_loss<<<B, 128, 0, n->stream>>>(n->d_O, n->out_ld, d_e, d_slots, off, d_t, n->d_dT,
                                         ends[0], n->d_part);
  if (int e = launched(n, "mlp slot loss")) return e;
  k_loss_total<<<1, 256, 0, n->stream>>>(n->d_part, B, n->d_scal);
  if (int e = launched(n, "mlp loss total")) return e;
  k_slot_reduce<<<B, 256, 0, n->stream>>>(d_slots, off, n->d_dT, ends[0], n->d_scal, n->d_O,
                                           n->out_ld);
  if (int e = launched(n, "mlp slot reduce")) return e;
  float* g = n->d_g;
  const float* W2 = n->d_p + n->off[2];
  const float* W3 = n->d_p + n->off[4];
  // dW3 = H2^T dO, db3 = colsum dO
  GemmArgs a = args(n->d_H2, n->H, n->d_O, n->out_ld, g + n->off[4], n->out_ld, n->H, n->out, B,
                    n->d_err);
  if (int e = gemm<ETf32, false, false, EPI_STORE>(n, a)) return e;
  k_colsum<<<(n->out + 255) / 256, 256, 0, n->stream>>>(n->d_O, n->out_ld, B, n->out,
                                                         g + n->off[5]);
  if (int e = launched(n, "mlp colsum")) return e;
  // dZ2 = (dO W3^T) * GELU'(Z2)
  a = args(n->d_O, n->out_ld, W3, n->out_ld, n->d_dZ2, n->H, B, n->H, n->out, n->d_err);
  a.Zin = n->d_Z2;
  a.ldz = n->H;
  if (int e = gemm<ETf32, true, true, EPI_DGELU>(n, a)) return e;
  // dW2 = H1^T dZ2, db2
  a = args(n->d_H1, n->H, n->d_dZ2, n->H, g + n->off[2], n->H, n->H, n->H, B, n->d_err);
  if (int e = gemm<ETf32, false, false, EPI_STORE>(n, a)) return e;
  k_colsum<<<(n->H + 255) / 256, 256, 0, n->stream>>>(n->d_dZ2, n->H, B, n->H, g + n->off[3]);
  if (int e = launched(n, "mlp colsum")) return e;
  // dZ1 = (dZ2 W2^T) * GELU'(Z1)
  a = args(n->d_dZ2, n->H, W2, n->H, n->d_dZ1, n->H, B, n->H, n->H, n->d_err);
  a.Zin = n->d_Z1;
  a.ldz = n->H;
  if (int e = gemm<ETf32, true, true, EPI_DGELU>(n, a)) return e;
  // dW1 = X^T dZ1, db1
  a = args(d_x, n->in, n->d_dZ1, n->H, g + n->off[0], n->H, n->in, n->H, B, n->d_err);
  if (int e = gemm<ETf32, false, false, EPI_STORE>(n, a)) return e;
  k_colsum<<<(n->H + 255) / 256, 256, 0, n->stream>>>(n->d_dZ1, n->H, B, n->H, g + n->off[1]);
  if (int e = launched(n, "mlp colsum")) return e;
  if (loss) {
    if (int e = sync_read(n)) return e;
    *loss = n->h_scal[1];
  }
  return RF_OK;
}

int rf_mlp_adam(rf_mlp* n, float lr) {
  if (!n || !(lr > 0.f)) return mfail("rf_mlp_adam: lr must be > 0");
  n->adam_t += 1;
  const double t = (double)n->adam_t;
  const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, t)));
  const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, t)));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, n->dev);
  k_adam<<<sms * 4, 256, 0, n->stream>>>(n->d_p, n->d_g, n->d_m, n->d_v, n->total, lr, c1, c2);
  return launched(n, "rf_mlp_adam");
}

int rf_mlp_train_step(rf_mlp* n, int32_t B, const float* d_x, const float* d_e,
                      const rf_slot* d_slots, const int64_t* d_offsets, const float* d_t,
                      float lr, double* loss) {
  if (int e = rf_mlp_loss_grad(n, B, d_x, d_e, d_slots, d_offsets, d_t, loss)) return e;
  return rf_mlp_adam(n, lr);
}

int rf_mlp_predict_warm(rf_mlp* n, int32_t B, const float* d_x, const double* d_macro,
                        const rf_slot* d_slots, const int64_t* d_offsets, float* d_warm) {
  if (!n || !d_x || !d_macro || !d_warm) return mfail("rf_mlp_predict_warm: null argument");
  if (int e = slot_args_ok(n, B, d_slots, d_offsets, false)) return e;
  if (!aligned16(d_x)) return mfail("rf_mlp_predict_warm: d_x must be 16-byte aligned");
  const long long* off = reinterpret_cast<const long long*>(d_offsets);
  for (int b0 = 0; b0 < B; b0 += n->maxB) {
    const int nb = std::min(n->maxB, B - b0);
    if (int e = forward<EBf16>(n, nb, d_x + (long long)b0 * n->in, false)) return e;
    k_slot_predict<<<nb, 128, 0, n->stream>>>(n->d_O, n->out_ld, d_macro + 6LL * b0, d_slots,
                                               off + b0, d_warm);
    if (int e = launched(n, "rf_mlp_predict_warm")) return e;
  }
  return RF_OK;
}

int rf_mlp_launches(const rf_mlp* n, int64_t* launches) {
  if (!n || !launches) return mfail("rf_mlp_launches: null argument");
  *launches = n->launches;
  return RF_OK;
}

int rf_mlp_destroy(rf_mlp* n) {
  if (!n) return RF_OK;
  if (n->stream) cudaStreamSynchronize(n->stream);
  cudaFree(n->d_p);
  cudaFree(n->d_g);
  cudaFree(n->d_m);
  cudaFree(n->d_v);
  cudaFree(n->d_Z1);
  cudaFree(n->d_H1);
  cudaFree(n->d_Z2);
  cudaFree(n->d_H2);
  cudaFree(n->d_dZ1);
  cudaFree(n->d_dZ2);
  cudaFree(n->d_O);
  cudaFree(n->d_part);
  cudaFree(n->d_scal);
  cudaFree(n->d_dT);
  cudaFree(n->d_err);
  if (n->h_scal) cudaFreeHost(n->h_scal);
  if (n->h_err) cudaFreeHost(n->h_err);
  if (n->own_stream) cudaStreamDestroy(n->stream);
  delete n;
  return RF_OK;
}

}  // extern "C"
