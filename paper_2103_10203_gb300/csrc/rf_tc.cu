// Tensor-core (tcgen05) transforms along x for the split-precision modes.
//
// The row kernel of one update (Sec. 4, steps d, a, b along x) as two GEMMs around the law:
//   inverse   eps[x][q]  = sum_j' Phi[x][j'] * Tq[q][j']          (M = 128 x, N = Qp, K = 2 Kx)
//   law       tau[q][x]  = sigma(eps) - C0 : eps                    (per voxel, FP32)
//   forward   T'[j'][q]  = sum_x  Phi[x][j'] * tau[q][x]           (M = 128 j' per tile, K = 128 x)
// with q = (row, component), j' = 2 j + (0: real, 1: imaginary part) over the pattern's kx >= 0
// columns, Phi[x][2j] = cos(2 pi kx_j x / Nx), Phi[x][2j+1] = -sin(...), and Tq holding the
// line coefficients scaled by w_j / N. One CTA owns a 128-wide slice of x for R rows; the
// forward sums over its slice only, and the transform along y adds the slices' partial sums.
//
// Operands are split into hi + lo parts of the tensor-core type (BF16 or TF32) and multiplied
// as hi*hi + hi*lo + lo*hi with FP32 accumulation in tensor memory. All operand tiles use the
// canonical no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix). The
// twiddle tiles are precomputed per pattern in that exact layout and staged into shared memory
// with bulk asynchronous copies; every mbarrier wait is bounded and reports a timeout.
//
// The transforms along y and z (Sec. 4 steps b and d on the reduced rectangle) run on the tensor
// cores as well, as one real GEMM per axis and direction: complex out[m][n] = sum_k W[m][k]
// in[k][n] with W = exp(sign 2 pi i mv kv / L), written with real and imaginary parts
// interleaved, D[2m + 0] = sum_k (Wr, -Wi) . (Xr, Xi) and D[2m + 1] = sum_k (Wi, Wr) . (Xr, Xi),
// so that A = W is 2M x 2K, B = X is 2K x N and D is 2M x N (64 complex outputs per 128-lane
// tile). A is precomputed per pattern; X is split into hi + lo while it is staged.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "rf_internal.cuh"
#include "rf_law.cuh"
#include "rf_tcgen05.cuh"

namespace rfk {
namespace tc {

constexpr int kTile = 128;           // x slice width and j' tile height
constexpr int kChunkBytes = 128;     // K bytes per staged chunk row
constexpr int kTileBytes = kTile * kChunkBytes;   // 16 KB: one 128-row chunk of one part
constexpr int kMaxQ = 48;            // Qp: rows * components per CTA (padded to 16)

// ------------------------------------------------------------------------------------------
// twiddle tiles: PhiI[xs][jc][part] (rows x, K = j' chunk), PhiF[jt][xs][xc][part] (rows j',
// K = x chunk); each tile 128 rows x 128 bytes in the core-matrix layout
template <class E>
__global__ void k_phi_tiles(const int* kx, int Kx, int Nx, const float2* tab, int nXS, int nJC,
                            int nJT, int nXC, unsigned char* phiI, unsigned char* phiF) {
  constexpr int per = kChunkBytes / E::kBytes;   // elements per chunk row
  const long long total = (long long)nXS * kTile * nJC * per;   // (x, j') elements
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int jp = (int)(i % ((long long)nJC * per));
    const int x = (int)(i / ((long long)nJC * per));
    float v = 0.f;
    if (x < Nx && jp < 2 * Kx) {
      const int j = jp >> 1;
      const int m = (int)(((long long)kx[j] * x) % Nx);
      const float2 w = tab[m];                 // (cos, sin)(2 pi m / Nx)
      v = (jp & 1) ? -w.y : w.x;
    }
    const int xs = x / kTile, xr = x % kTile;
    // inverse tile
    {
      const int jc = jp / per, k = jp % per;
      unsigned char* base = phiI + ((long long)(xs * nJC + jc) * 2) * kTileBytes;
      put_split<E>(base, base + kTileBytes, cm_off(xr, k * E::kBytes, kChunkBytes), v);
    }
    // forward tile (only j' inside the nJT tiles)
    if (jp < nJT * kTile) {
      const int jt = jp / kTile, jr = jp % kTile;
      const int xc = xr / per, k = xr % per;
      unsigned char* base =
          phiF + ((long long)((jt * nXS + xs) * nXC + xc) * 2) * kTileBytes;
      put_split<E>(base, base + kTileBytes, cm_off(jr, k * E::kBytes, kChunkBytes), v);
    }
  }
}

// hi + lo split of one 16-byte core-matrix row segment (8 BF16 or 4 TF32 values)
template <class E>
__device__ __forceinline__ void split_seg(const float* x, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
  if constexpr (E::kBytes == 2) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * i]), h1 = __float2bfloat16_rn(x[2 * i + 1]);
      const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * i] - __bfloat162float(h0));
      const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * i + 1] - __bfloat162float(h1));
      h[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
      l[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h[i]) : "f"(x[i]));
      const float r = x[i] - __uint_as_float(h[i]);
      asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l[i]) : "f"(r));
    }
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// ------------------------------------------------------------------------------------------
struct TcRowArgs {
  const float2* T;        // [rows][NC][Kx]
  float* Tout;            // [nXS][rows][NC][2 Kx]
  const uint8_t* phase;
  float* state;
  const float* fac;
  const unsigned char* phiI;
  const unsigned char* phiF;
  int Nx, Kx, rows, R, Qp, nJC, nJT, nXC, nXS;
  uint32_t tmem_cols;
  long long N;
  LawParams law;
  const int* done;
  int* err;
  long wait_limit;   // polls per bounded wait
  int stall;         // test hook: first wait on a barrier that nothing completes
};

}  // namespace tc

namespace tc {

template <class E, int NC, bool PLASTIC>
__global__ __launch_bounds__(128) void k_tc_row(TcRowArgs a) {
  if (a.done && *a.done) return;
  constexpr int per = kChunkBytes / E::kBytes;         // K elements per chunk
  constexpr int tau_rb = kTile * E::kBytes;            // tau row bytes (K = 128 x)
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* bufA = smem;                                  // 2 x (hi, lo) 16 KB tiles
  unsigned char* bufT = smem + 4 * kTileBytes;                 // 2 x (hi, lo) Qp x 128 B
  const int tq_bytes = a.Qp * kChunkBytes;
  unsigned char* tau = bufT + 4 * tq_bytes;                    // (hi, lo) Qp x tau_rb
  const int tau_bytes = a.Qp * tau_rb;
  // lbar[2], mbar[2], and a barrier that nothing completes (the stall test)
  uint64_t* bars = reinterpret_cast<uint64_t*>(tau + 2 * tau_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 5);
  int* s_err = reinterpret_cast<int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5;
  const int xs = blockIdx.x;
  const int x = xs * kTile + tid;
  const int row0 = blockIdx.y * a.R;
  const int Q = a.R * NC;

  if (tid == 0) {
    for (int i = 0; i < 5; ++i) mbar_init(&bars[i], 1);
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = (uint32_t)(32 * warp) << 16;

  const int n_stages = a.nJC + a.nJT * a.nXC;
  const uint32_t id_mma = idesc<E>(kTile, a.Qp);
  // Failures (a bounded wait that ran out) are combined in s_err at CTA barriers, so that every
  // thread takes the same path through barriers and warp-collective tensor-memory loads.
  if (a.stall) {
    if (tid == 0 && !mbar_wait(&bars[4], 0, a.wait_limit)) atomicOr(s_err, 1);
    __syncthreads();
  }
  bool ok = (*s_err == 0);
  // phases issued by thread 0 on the copy barriers (nl) and the product barriers (nm); each
  // barrier has at most one issued phase that no successful wait has seen
  int nl[2] = {0, 0}, nm[2] = {0, 0};

  for (int g = 0; ok && g < n_stages; ++g) {
    const int b = g & 1;
    unsigned char* A = bufA + b * 2 * kTileBytes;
    unsigned char* Tb = bufT + b * 2 * tq_bytes;
    // buffer b is free once the MMAs of stage g - 2 completed
    if (g >= 2 && !mbar_wait(&bars[2 + b], ((g - 2) >> 1) & 1, a.wait_limit)) {
      ok = false;
      atomicOr(s_err, 1);
    }
    if (tid == 0 && ok) {
      ++nl[b];
      const unsigned char* src;
      if (g < a.nJC) {
        src = a.phiI + ((long long)(xs * a.nJC + g) * 2) * kTileBytes;
      } else {
        const int f = g - a.nJC, jt = f / a.nXC, xc = f % a.nXC;
        src = a.phiF + ((long long)((jt * a.nXS + xs) * a.nXC + xc) * 2) * kTileBytes;
      }
      bulk_load(A, src, 2 * kTileBytes, &bars[b]);
    }
    if (g < a.nJC && ok) {
      // Tq chunk: rows q, K = j' in [g * per, (g + 1) * per). Item i = (row q, 16-byte segment
      // sg) with the row's low three bits fastest, so that a warp's 16-byte stores fill whole
      // core matrices; each batch issues all its loads before the splits.
      constexpr int cps = 8 / E::kBytes;   // complex values per segment
      const int items = a.Qp * (kChunkBytes / 16);
      for (int i0 = tid; i0 < items; i0 += 4 * blockDim.x) {
        float v[4][2 * cps];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * blockDim.x;
          const int q = ((i >> 6) << 3) | (i & 7), sg = (i >> 3) & 7;
          const int r = q / NC, c = q - r * NC, row = row0 + r;
          const bool live = i < items && q < Q && row < a.rows;
          const float2* tp = a.T + ((long long)row * NC + c) * a.Kx;
#pragma unroll
          for (int qq = 0; qq < cps; ++qq) {
            const int j = g * (per / 2) + sg * cps + qq;
            float2 t = make_float2(0.f, 0.f);
            float f = 0.f;
            if (live && j < a.Kx) {
              t = tp[j];
              f = a.fac[j];
            }
            v[u][2 * qq] = f * t.x;
            v[u][2 * qq + 1] = f * t.y;
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = i0 + u * blockDim.x;
          if (i >= items) continue;
          const int q = ((i >> 6) << 3) | (i & 7), sg = (i >> 3) & 7;
          uint4 hi, lo;
          split_seg<E>(v[u], hi, lo);
          const uint32_t off = cm_off(q, sg * 16, kChunkBytes);
          *reinterpret_cast<uint4*>(Tb + off) = hi;
          *reinterpret_cast<uint4*>(Tb + tq_bytes + off) = lo;
        }
      }
    }
    if (g == a.nJC) {
      // law: D1 complete (stage nJC - 1 committed); eps for x = this thread's lane
      if (!mbar_wait(&bars[2 + ((a.nJC - 1) & 1)], ((a.nJC - 1) >> 1) & 1, a.wait_limit))
        atomicOr(s_err, 1);
      __syncthreads();
      ok = (*s_err == 0);
    }
    if (g == a.nJC && ok) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      float ev[kMaxQ];
#pragma unroll
      for (int c0 = 0; c0 < kMaxQ; c0 += 16)
        if (c0 < a.Qp) tmem_ld16(tmem + lane_base + c0, ev + c0);
      unsigned char* th = tau;
      unsigned char* tl = tau + tau_bytes;
#pragma unroll
      for (int r = 0; r < kMaxQ / NC; ++r) {
        if (r >= a.R) break;
        const int row = row0 + r;
        float tv[6] = {0, 0, 0, 0, 0, 0};
        if (row < a.rows && x < a.Nx) {
          const long long gi = (long long)row * a.Nx + x;
          float e6[6];
          if (NC == 3) {
            e6[0] = ev[r * NC + 0];
            e6[1] = ev[r * NC + 1];
            e6[2] = 0.f;
            e6[3] = 0.f;
            e6[4] = 0.f;
            e6[5] = ev[r * NC + 2];
          } else {
#pragma unroll
            for (int i = 0; i < 6; ++i) e6[i] = ev[r * NC + i];
          }
          const DevPhase ph = a.law.ph[a.phase[gi]];
          float ep[6] = {0, 0, 0, 0, 0, 0};
          float alpha = 0.f;
          if (PLASTIC) {
            if (NC == 3) {
              ep[0] = a.state[gi];
              ep[1] = a.state[a.N + gi];
              ep[5] = a.state[2 * a.N + gi];
              ep[2] = -(ep[0] + ep[1]);
              alpha = a.state[3 * a.N + gi];
            } else {
#pragma unroll
              for (int i = 0; i < 6; ++i) ep[i] = a.state[i * a.N + gi];
              alpha = a.state[6 * a.N + gi];
            }
          }
          LawOut o;
          stress6<PLASTIC>(e6, ph, ep, alpha, o);
          const float tr = e6[0] + e6[1] + e6[2];
#pragma unroll
          for (int i = 0; i < 3; ++i) tv[i] = o.s[i] - (a.law.lam0 * tr + 2.f * a.law.mu0 * e6[i]);
#pragma unroll
          for (int i = 3; i < 6; ++i) tv[i] = o.s[i] - 2.f * a.law.mu0 * e6[i];
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int c6 = NC == 3 ? (c == 2 ? 5 : c) : c;
          put_split<E>(th, tl, cm_off(r * NC + c, tid * E::kBytes, tau_rb), tv[c6]);
        }
      }
      // padding rows of tau are zero
      for (int q = Q; q < a.Qp; ++q) put_split<E>(th, tl, cm_off(q, tid * E::kBytes, tau_rb), 0.f);
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0 && *s_err == 0) {
      if (!mbar_wait(&bars[b], (g >> 1) & 1, a.wait_limit)) {
        atomicOr(s_err, 1);
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a_hi = smem_u32(A), a_lo = a_hi + kTileBytes;
        if (g < a.nJC) {
          const uint32_t b_hi = smem_u32(Tb), b_lo = b_hi + tq_bytes;
          const uint32_t d = tmem;   // D1 at columns [0, Qp)
          for (int s = 0; s < kChunkBytes / 32; ++s) {
            const uint32_t o = s * 256;
            const uint32_t sbo_a = (kChunkBytes / 16) * 128, sbo_b = sbo_a;
            const uint64_t ah = make_desc(a_hi + o, 128, sbo_a), al = make_desc(a_lo + o, 128, sbo_a);
            const uint64_t bh = make_desc(b_hi + o, 128, sbo_b), bl = make_desc(b_lo + o, 128, sbo_b);
            const uint32_t first = (g == 0 && s == 0) ? 0u : 1u;
            mma<E>(d, ah, bh, id_mma, first);
            mma<E>(d, ah, bl, id_mma, 1u);
            mma<E>(d, al, bh, id_mma, 1u);
          }
        } else {
          const int f = g - a.nJC, jt = f / a.nXC, xc = f % a.nXC;
          const uint32_t d = tmem + (uint32_t)(a.Qp * (1 + jt));
          const uint32_t t_hi = smem_u32(tau), t_lo = t_hi + tau_bytes;
          const uint32_t sbo_t = (tau_rb / 16) * 128;
          for (int s = 0; s < kChunkBytes / 32; ++s) {
            const uint32_t oa = s * 256;
            const uint32_t ob = (xc * (kChunkBytes / 16) + 2 * s) * 128;
            const uint32_t sbo_a = (kChunkBytes / 16) * 128;
            const uint64_t ah = make_desc(a_hi + oa, 128, sbo_a), al = make_desc(a_lo + oa, 128, sbo_a);
            const uint64_t bh = make_desc(t_hi + ob, 128, sbo_t), bl = make_desc(t_lo + ob, 128, sbo_t);
            const uint32_t first = (xc == 0 && s == 0) ? 0u : 1u;
            mma<E>(d, ah, bh, id_mma, first);
            mma<E>(d, ah, bl, id_mma, 1u);
            mma<E>(d, al, bh, id_mma, 1u);
          }
        }
        mma_commit(&bars[2 + b]);
        ++nm[b];
      }
    }
    __syncthreads();
    ok = (*s_err == 0);
    if (!ok) break;     // uniform: every thread read s_err after the same barrier
  }
  // all MMAs done: wait for the last stage's commit
  if (ok) {
    const int gl = n_stages - 1;
    if (!mbar_wait(&bars[2 + (gl & 1)], (gl >> 1) & 1, a.wait_limit)) atomicOr(s_err, 1);
  }
  __syncthreads();
  ok = (*s_err == 0);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok) {
    const int jp_base = 0;
    for (int jt = 0; jt < a.nJT; ++jt) {
      const int jp = jt * kTile + tid + jp_base;
      float ov[kMaxQ];
#pragma unroll
      for (int c0 = 0; c0 < kMaxQ; c0 += 16)
        if (c0 < a.Qp) tmem_ld16(tmem + lane_base + (uint32_t)(a.Qp * (1 + jt)) + c0, ov + c0);
      if (jp < 2 * a.Kx) {
#pragma unroll
        for (int q = 0; q < kMaxQ; ++q) {
          if (q >= Q) break;
          const int r = q / NC, c = q % NC, row = row0 + r;
          if (row < a.rows)
            a.Tout[(((long long)xs * a.rows + row) * NC + c) * (2LL * a.Kx) + jp] = ov[q];
        }
      }
    }
  } else if (tid == 0) {
    // a wait gave up: report it, then let the copies and products in flight finish (each
    // barrier's last issued phase, with the default limit) before tensor memory is released
    atomicExch(a.err, 1);
    for (int b = 0; b < 2; ++b) {
      if (nl[b] > 0) mbar_wait(&bars[b], (nl[b] - 1) & 1);
      if (nm[b] > 0) mbar_wait(&bars[2 + b], (nm[b] - 1) & 1);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols));
}

}  // namespace tc

namespace tc {

// A tiles of one axis transform: tile (mt, g) covers complex rows [64 mt, 64 mt + 64) and
// elements [g per, (g + 1) per) of 2K; hi and lo parts back to back (2 x 16 KB per tile)
template <class E>
__global__ void k_axis_tiles(int M, int K, const int* mvals, const int* kvals, const float2* tab,
                             int L, int sign, int nMT, int nKC, unsigned char* A) {
  constexpr int per = kChunkBytes / E::kBytes;
  const long long total = (long long)nMT * nKC * kTile * per;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(i % per);
    const int r = (int)((i / per) % kTile);
    const long long t = i / ((long long)per * kTile);
    const int g = (int)(t % nKC), mt = (int)(t / nKC);
    const int m = mt * 64 + (r >> 1);
    const int kp = g * per + e, k = kp >> 1;
    float v = 0.f;
    if (m < M && k < K) {
      const long long mv = mvals ? mvals[m] : m, kv = kvals ? kvals[k] : k;
      float2 w = tab[(int)((mv * kv) % L)];   // (cos, sin)(2 pi mv kv / L)
      if (sign < 0) w.y = -w.y;
      const bool im_row = r & 1, im_col = kp & 1;
      v = im_row ? (im_col ? w.x : w.y) : (im_col ? -w.y : w.x);
    }
    unsigned char* base = A + ((long long)(mt * nKC + g) * 2) * kTileBytes;
    put_split<E>(base, base + kTileBytes, cm_off(r, e * E::kBytes, kChunkBytes), v);
  }
}

struct TcAxisArgs {
  const float2* in;       // [in_splits][batch][K][N] (the splits are summed)
  int in_splits;
  long long in_split_stride, in_bstride;
  float2* out;            // [batch][M][N]
  long long out_bstride;
  const unsigned char* A;
  int M, N, K, nKC, NT, lNT;   // lNT = log2(NT)
  uint32_t tmem_cols;
  const int* done;
  int* err;
  long wait_limit;   // polls per bounded wait
  int stall;         // test hook: first wait on a barrier that nothing completes
};

// one CTA: 64 complex output rows (blockIdx.y) x NT columns (blockIdx.x) of one batch entry
// (blockIdx.z); 256 threads stage the operands, warps 0-3 (one thread per accumulator lane)
// read the result
template <class E>
__global__ __launch_bounds__(256) void k_tc_axis(TcAxisArgs a) {
  if (a.done && *a.done) return;
  constexpr int per = kChunkBytes / E::kBytes;   // K elements per chunk
  constexpr int kc = per / 2;                    // complex k per chunk
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* As = smem;                          // hi, lo: 2 x 16 KB
  unsigned char* Bs = smem + 2 * kTileBytes;         // hi, lo: 2 x NT x 128 B
  const int bbytes = a.NT * kChunkBytes;
  // [0] A copy, [1] MMAs, [2] a barrier that nothing completes (the stall test)
  uint64_t* bars = reinterpret_cast<uint64_t*>(Bs + 2 * bbytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 3);
  int* s_err = reinterpret_cast<int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int n0 = blockIdx.x * a.NT, mt = blockIdx.y;
  const long long b = blockIdx.z;
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    *s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  const uint32_t id_mma = idesc<E>(kTile, a.NT);
  const float2* inb = a.in + b * a.in_bstride;
  if (a.stall && tid == 0 && !mbar_wait(&bars[2], 0, a.wait_limit)) atomicOr(s_err, 1);
  bool ok = true;
  int nl = 0, nm = 0;   // phases thread 0 issued on the copy and the product barrier
  for (int g = 0; g < a.nKC; ++g) {
    // the buffers are free once the previous chunk's MMAs completed
    if (g > 0 && !mbar_wait(&bars[1], (g - 1) & 1, a.wait_limit)) atomicOr(s_err, 1);
    __syncthreads();
    ok = (*s_err == 0);
    if (!ok) break;   // uniform: every thread read s_err after the same barrier
    if (tid == 0) {
      bulk_load(As, a.A + ((long long)(mt * a.nKC + g) * 2) * kTileBytes, 2 * kTileBytes,
                &bars[0]);
      ++nl;
    }
    // B chunk: item i = (row nn, 16-byte segment sg) holds cps complex k of column n0 + nn;
    // consecutive threads take consecutive columns (coalesced loads), each batch issues all its
    // loads before the splits, and every segment goes to shared memory as one 16-byte store
    constexpr int cps = 8 / E::kBytes;   // complex values per 16-byte segment
    const int items = a.NT * (kChunkBytes / 16);
    for (int i0 = tid; i0 < items; i0 += 4 * blockDim.x) {
      float2 v[4][cps];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        const int nn = i & (a.NT - 1), sg = i >> a.lNT, n = n0 + nn;
#pragma unroll
        for (int q = 0; q < cps; ++q) {
          const int k = g * kc + sg * cps + q;
          v[u][q] = make_float2(0.f, 0.f);
          if (i < items && k < a.K && n < a.N) {
            const float2* p = inb + (long long)k * a.N + n;
            v[u][q] = p[0];
            for (int t = 1; t < a.in_splits; ++t) {
              const float2 w = p[t * a.in_split_stride];
              v[u][q].x += w.x;
              v[u][q].y += w.y;
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int i = i0 + u * blockDim.x;
        if (i >= items) continue;
        const int nn = i & (a.NT - 1), sg = i >> a.lNT;
        uint4 hi, lo;
        split_seg<E>(reinterpret_cast<const float*>(v[u]), hi, lo);
        const uint32_t off = cm_off(nn, sg * 16, kChunkBytes);
        *reinterpret_cast<uint4*>(Bs + off) = hi;
        *reinterpret_cast<uint4*>(Bs + bbytes + off) = lo;
      }
    }
    asm volatile("fence.proxy.async.shared::cta;");
    __syncthreads();
    if (tid == 0) {
      if (!mbar_wait(&bars[0], g & 1, a.wait_limit)) {
        atomicOr(s_err, 1);
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a_hi = smem_u32(As), a_lo = a_hi + kTileBytes;
        const uint32_t b_hi = smem_u32(Bs), b_lo = b_hi + bbytes;
        const uint32_t sbo = (kChunkBytes / 16) * 128;
        for (int st = 0; st < kChunkBytes / 32; ++st) {
          const uint32_t o = st * 256;
          const uint64_t ah = make_desc(a_hi + o, 128, sbo), al = make_desc(a_lo + o, 128, sbo);
          const uint64_t bh = make_desc(b_hi + o, 128, sbo), bl = make_desc(b_lo + o, 128, sbo);
          const uint32_t first = (g == 0 && st == 0) ? 0u : 1u;
          mma<E>(tmem, ah, bh, id_mma, first);
          mma<E>(tmem, ah, bl, id_mma, 1u);
          mma<E>(tmem, al, bh, id_mma, 1u);
        }
        mma_commit(&bars[1]);
        ++nm;
      }
    }
  }
  if (ok && !mbar_wait(&bars[1], (a.nKC - 1) & 1, a.wait_limit)) atomicOr(s_err, 1);
  __syncthreads();
  ok = (*s_err == 0);
  asm volatile("tcgen05.fence::after_thread_sync;");
  if (ok && tid < 128) {
    // lane tid holds D row tid: the real (even) or imaginary (odd) part of output m
    const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
    const int m = mt * 64 + (tid >> 1);
    float2* ob = a.out + b * a.out_bstride + (long long)m * a.N;
    for (int c0 = 0; c0 < a.NT; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + lane_base + (uint32_t)c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float w = __shfl_xor_sync(0xffffffffu, v[i], 1);
        const int n = n0 + c0 + i;
        if (!(tid & 1) && m < a.M && n < a.N) ob[n] = make_float2(v[i], w);
      }
    }
  } else if (tid == 0) {
    // a wait gave up: report it, then let the copy and the products in flight finish (the
    // last issued phase of each barrier, with the default limit) before tensor memory is
    // released
    atomicExch(a.err, 1);
    if (nl > 0) mbar_wait(&bars[0], (nl - 1) & 1);
    if (nm > 0) mbar_wait(&bars[1], (nm - 1) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols));
}

}  // namespace tc

// ------------------------------------------------------------------------------------------
// host side
int tc_setup(rf_ctx* c) {
  using namespace tc;
  const bool bf = c->opt.precision == RF_PREC_SPLIT_BF16;
  const int bytes = bf ? 2 : 4;
  const int per = kChunkBytes / bytes;
  c->tc_nXS = (c->nx + kTile - 1) / kTile;
  const int jp = 2 * c->Kx;
  c->tc_nJT = (jp + kTile - 1) / kTile;
  c->tc_nJC = (c->tc_nJT * kTile) / per;     // inverse K covers the same padded range
  c->tc_nXC = kTile / per;
  // rows per CTA: Qp * (1 + nJT) tensor-memory columns must fit in 512
  int R = (c->nc == 3) ? 16 : 8;
  auto qp_of = [&](int r) { return ((r * c->nc + 15) / 16) * 16; };
  while (R > 1 && qp_of(R) * (1 + c->tc_nJT) > 512) --R;
  const int Qp = qp_of(R);
  if (Qp * (1 + c->tc_nJT) > 512) {
    set_error("split precision: pattern too wide for tensor memory (2 Kx > 1152)");
    return RF_ERR_INVALID;
  }
  c->tc_R = R;
  c->tc_Qp = Qp;
  uint32_t cols = 32;
  while (cols < (uint32_t)(Qp * (1 + c->tc_nJT))) cols <<= 1;
  c->tc_cols = cols;
  const size_t tile_pairs_I = (size_t)c->tc_nXS * c->tc_nJC;
  const size_t tile_pairs_F = (size_t)c->tc_nJT * c->tc_nXS * c->tc_nXC;
  if (int er = palloc(c, &c->d_phiI, tile_pairs_I * 2 * kTileBytes, "split precision buffers"))
    return er;
  if (int er = palloc(c, &c->d_phiF, tile_pairs_F * 2 * kTileBytes, "split precision buffers"))
    return er;
  if (int er = palloc(c, &c->d_Tout, (size_t)c->tc_nXS * c->rows * c->nc * 2 * c->Kx,
                      "split precision buffers"))
    return er;
  if (int er = palloc(c, &c->d_tc_err, 1, "split precision buffers")) return er;
  cudaError_t e = cudaMemsetAsync(c->d_tc_err, 0, sizeof(int), c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "split precision buffers");
  if (bf)
    k_phi_tiles<EBf16><<<608, 256, 0, c->stream>>>(c->d_kx, c->Kx, c->nx, c->d_twx, c->tc_nXS,
                                                    c->tc_nJC, c->tc_nJT, c->tc_nXC, c->d_phiI,
                                                    c->d_phiF);
  else
    k_phi_tiles<ETf32><<<608, 256, 0, c->stream>>>(c->d_kx, c->Kx, c->nx, c->d_twx, c->tc_nXS,
                                                    c->tc_nJC, c->tc_nJT, c->tc_nXC, c->d_phiI,
                                                    c->d_phiF);
  c->launches += 1;
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "phi tiles");
  // A tiles of the transforms along y (and z): forward (rows = pattern values, K = positions)
  // and inverse (rows = positions, K = pattern values)
  struct AxisSpec {
    TcAxis* dst;
    int M, K;
    const int* mvals;
    const int* kvals;
    const float2* tab;
    int L, sign;
  };
  AxisSpec specs[4] = {{&c->tc_yf, c->Ky, c->ny, c->d_kym, nullptr, c->d_twy, c->ny, -1},
                       {&c->tc_yi, c->ny, c->Ky, nullptr, c->d_kym, c->d_twy, c->ny, +1},
                       {&c->tc_zf, c->Kz, c->nz, c->d_kzm, nullptr, c->d_twz, c->nz, -1},
                       {&c->tc_zi, c->nz, c->Kz, nullptr, c->d_kzm, c->d_twz, c->nz, +1}};
  for (int i = 0; i < (c->dim == 3 ? 4 : 2); ++i) {
    const AxisSpec& sp = specs[i];
    TcAxis& ax = *sp.dst;
    ax.M = sp.M;
    ax.K = sp.K;
    ax.nMT = (sp.M + 63) / 64;
    ax.nKC = (2 * sp.K + per - 1) / per;
    if (int er = palloc(c, &ax.A, (size_t)ax.nMT * ax.nKC * 2 * kTileBytes, "axis tiles"))
      return er;
    if (bf)
      k_axis_tiles<EBf16><<<304, 256, 0, c->stream>>>(sp.M, sp.K, sp.mvals, sp.kvals, sp.tab,
                                                      sp.L, sp.sign, ax.nMT, ax.nKC, ax.A);
    else
      k_axis_tiles<ETf32><<<304, 256, 0, c->stream>>>(sp.M, sp.K, sp.mvals, sp.kvals, sp.tab,
                                                      sp.L, sp.sign, ax.nMT, ax.nKC, ax.A);
    c->launches += 1;
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "axis tiles");
  }
  const int tau_rb = kTile * bytes;
  // force one CTA per SM when it needs all 512 tensor-memory columns
  size_t smem = 4 * kTileBytes + 4 * (size_t)Qp * kChunkBytes + 2 * (size_t)Qp * tau_rb + 64;
  if (cols > 256 && smem < 120 * 1024) smem = 120 * 1024;
  c->tc_smem = smem;
  return RF_OK;
}

// One transform along y or z on the tensor cores (see the top of this file); the column tile
// NT is the largest of 256, 128, 64, 32 that still gives about two CTAs per SM.
int launch_tc_axis(rf_ctx* c, const TcAxis& ax, const float2* in, int in_splits,
                   long long in_split_stride, long long in_bstride, float2* out,
                   long long out_bstride, int N, int batch, const int* done) {
  using namespace tc;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
  int NT = 256;
  while (NT > 32 && (long long)((N + NT - 1) / NT) * ax.nMT * batch < 2LL * sms) NT >>= 1;
  TcAxisArgs a{};
  a.in = in;
  a.in_splits = in_splits;
  a.in_split_stride = in_split_stride;
  a.in_bstride = in_bstride;
  a.out = out;
  a.out_bstride = out_bstride;
  a.A = ax.A;
  a.M = ax.M;
  a.N = N;
  a.K = ax.K;
  a.nKC = ax.nKC;
  a.NT = NT;
  a.lNT = 0;
  while ((1 << a.lNT) < NT) ++a.lNT;
  a.tmem_cols = (uint32_t)std::max(32, NT);
  a.done = done;
  a.err = &c->d_status->timeout;
  a.wait_limit = c->opt.wait_limit > 0 ? (long)c->opt.wait_limit : kWaitLimit;
  a.stall = c->opt.stall_test;
  const size_t smem = 2 * kTileBytes + 2 * (size_t)NT * kChunkBytes + 64;
  dim3 grid((N + NT - 1) / NT, ax.nMT, batch);
  if (c->opt.precision == RF_PREC_SPLIT_BF16)
    k_tc_axis<EBf16><<<grid, 256, smem, c->stream>>>(a);
  else
    k_tc_axis<ETf32><<<grid, 256, smem, c->stream>>>(a);
  c->launches += 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RF_OK : cuda_fail(e, "tc axis");
}

void init_attributes_tc() {
  using namespace tc;
  const int s = 200 * 1024;
  cudaFuncSetAttribute(k_tc_axis<EBf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_tc_axis<ETf32>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_tc_row<EBf16, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_tc_row<EBf16, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_tc_row<EBf16, 6, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_tc_row<EBf16, 6, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_tc_row<ETf32, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_tc_row<ETf32, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_tc_row<ETf32, 6, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_tc_row<ETf32, 6, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
}

template <class E, int NC, bool PL>
static int tc_row_launch(rf_ctx* c, const tc::TcRowArgs& a) {
  dim3 grid(c->tc_nXS, (c->rows + c->tc_R - 1) / c->tc_R);
  tc::k_tc_row<E, NC, PL><<<grid, 128, c->tc_smem, c->stream>>>(a);
  c->launches += 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RF_OK : cuda_fail(e, "tc row");
}

int launch_tc_row(rf_ctx* c, const int* done) {
  tc::TcRowArgs a{};
  a.T = c->d_T1;
  a.Tout = c->d_Tout;
  a.phase = c->d_phase;
  a.state = c->d_state;
  a.fac = c->d_fac;
  a.phiI = c->d_phiI;
  a.phiF = c->d_phiF;
  a.Nx = c->nx;
  a.Kx = c->Kx;
  a.rows = c->rows;
  a.R = c->tc_R;
  a.Qp = c->tc_Qp;
  a.nJC = c->tc_nJC;
  a.nJT = c->tc_nJT;
  a.nXC = c->tc_nXC;
  a.nXS = c->tc_nXS;
  a.tmem_cols = c->tc_cols;
  a.N = c->N;
  a.law = c->law;
  a.done = done;
  a.err = &c->d_status->timeout;
  a.wait_limit = c->opt.wait_limit > 0 ? (long)c->opt.wait_limit : tc::kWaitLimit;
  a.stall = c->opt.stall_test;
  const bool bf = c->opt.precision == RF_PREC_SPLIT_BF16;
  const bool pl = c->has_plastic;
  if (c->nc == 3) {
    if (bf) return pl ? tc_row_launch<tc::EBf16, 3, true>(c, a) : tc_row_launch<tc::EBf16, 3, false>(c, a);
    return pl ? tc_row_launch<tc::ETf32, 3, true>(c, a) : tc_row_launch<tc::ETf32, 3, false>(c, a);
  }
  if (bf) return pl ? tc_row_launch<tc::EBf16, 6, true>(c, a) : tc_row_launch<tc::EBf16, 6, false>(c, a);
  return pl ? tc_row_launch<tc::ETf32, 6, true>(c, a) : tc_row_launch<tc::ETf32, 6, false>(c, a);
}

}  // namespace rfk
