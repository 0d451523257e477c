// Row kernel of the FFT transform mode with warp-resident FFTs, for grid rows of 1024 voxels
// (2D): steps d (along x), a and b (along x) of Sec. 4 for one grid row per warp at a time.
//
// A row's three strain lines (11, 22, 12) travel as two complex sequences, A = line 11 + i line
// 22 and B = line 12. Each 1024-point FFT is a four-step 32 x 32 transform: lane k1 holds the
// 32 inputs k1 + 32 k2 in registers, a 32-point DFT in registers (two 16-point DFTs and a
// radix-2 step), a twiddle exp(sign 2 pi i k1 n2 / 1024), a transpose through a padded
// warp-private shared-memory region (pitch 33), and a second 32-point DFT. After the inverse
// transforms, lane n2 holds the voxels x = 32 n1 + n2 of the row: the law runs on them in
// registers, and the forward transforms run the same steps in the opposite order. Only the warp
// synchronises (__syncwarp); the block meets once, after its prologue. The spectra are built
// from and reduced to the pattern's kx columns (Hermitian completion and separation) in the same
// shared-memory region. The final pass keeps the shared-memory row kernel.
#include <algorithm>

#include "rf_fftcore.cuh"
#include "rf_internal.cuh"
#include "rf_law.cuh"

namespace rfk {
namespace wfft {

constexpr int kN = 1024;             // row length handled here
constexpr int kPad = 33;             // transpose pitch (entries): conflict-free rows and columns
constexpr int kRegion = 32 * kPad;   // entries of one warp region (>= kN)
constexpr int kPairRegion = 2 * kRegion;   // SA and SB of one warp pair

// exp(sign i pi q / 16) for q in [0, 16): the 32-point kernel's twiddles (cos and sin of
// multiples of pi / 16)
__device__ __forceinline__ float2 w32(int q, int sign) {
  const float c[9] = {1.f,
                      0.98078528040323044912f,
                      0.92387953251128675613f,
                      0.83146961230254523708f,
                      0.70710678118654752440f,
                      0.55557023301960222474f,
                      0.38268343236508977173f,
                      0.19509032201612826785f,
                      0.f};
  const float cs = q <= 8 ? c[q] : -c[16 - q];
  const float sn = q <= 8 ? c[8 - q] : c[q - 8];
  return make_float2(cs, sign < 0 ? -sn : sn);
}

// 32-point DFT of v in registers (natural order in and out): even and odd samples through two
// 16-point DFTs, then X[q] = E[q] + W^q O[q], X[q + 16] = E[q] - W^q O[q], W = exp(sign 2 pi i / 32)
__device__ __forceinline__ void dft32(float2* v, int sign) {
  float2 e[16], o[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    e[m] = v[2 * m];
    o[m] = v[2 * m + 1];
  }
  fftc::dft16(e, sign);
  fftc::dft16(o, sign);
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int i = 4 * (q & 3) + (q >> 2);   // where the 16-point kernel leaves its output q
    const float2 E = e[i];
    const float2 O = fftc::cmul(o[i], w32(q, sign));
    v[q] = make_float2(E.x + O.x, E.y + O.y);
    v[q + 16] = make_float2(E.x - O.x, E.y - O.y);
  }
}

// Forward transform (exp(-2 pi i k n / 1024)) of the sequence whose entries 32 n1 + n2 lane n2
// holds in v[n1]; afterwards lane k1 holds the outputs k1 + 32 k2 in v[k2]. tab[t] =
// exp(+2 pi i t / 1024). With k = k1 + 32 k2 and n = 32 n1 + n2: a 32-point DFT over n1 per
// lane, the twiddle exp(-2 pi i k1 n2 / 1024), a transpose through T and a 32-point DFT over n2.
// The inverse transform is the conjugate of the forward transform of the conjugate, with the
// roles of the two index orders exchanged; the row kernel calls this one body for all four of
// its transforms (the kernel's code stays small enough for the instruction cache).
__device__ __forceinline__ void fwd1024(float2* v, float2* T, const float2* __restrict__ tab,
                                        int lane) {
#pragma unroll 1
  for (int h = 0; h < 2; ++h) {
    dft32(v, -1);
    if (h == 1) break;
    // twiddle exp(-2 pi i k1 n2 / 1024) with n2 = lane and k1 = 4 a + b as the product of the
    // table's exp(2 pi i 4 a n2 / 1024) and exp(2 pi i b n2 / 1024), conjugated: ten loads
    // instead of 31 (fewer registers in flight), one extra rounding per twiddle
    float2 lo[4], hi[8];
    lo[0] = hi[0] = make_float2(1.f, 0.f);
#pragma unroll
    for (int b = 1; b < 4; ++b) lo[b] = __ldg(tab + b * lane);
#pragma unroll
    for (int q = 1; q < 8; ++q) hi[q] = __ldg(tab + 4 * q * lane);
#pragma unroll
    for (int k1 = 1; k1 < 32; ++k1) {
      float2 w = (k1 & 3) == 0 ? hi[k1 >> 2]
                 : (k1 >> 2) == 0 ? lo[k1 & 3] : fftc::cmul(hi[k1 >> 2], lo[k1 & 3]);
      w.y = -w.y;
      v[k1] = fftc::cmul(v[k1], w);
    }
    __syncwarp();
#pragma unroll
    for (int k1 = 0; k1 < 32; ++k1) T[k1 * kPad + lane] = v[k1];
    __syncwarp();
#pragma unroll
    for (int n2 = 0; n2 < 32; ++n2) v[n2] = T[lane * kPad + n2];
    __syncwarp();
  }
}

struct RowWArgs {
  const float2* T;      // [rows][NC][Kx] strain line coefficients
  float2* Tout;         // [rows][NC][Kx] polarization line coefficients
  const uint8_t* phase;
  const float* state;   // [4][N] or null
  const int* kx;        // [Kx]
  const float2* table;  // exp(+2 pi i t / 1024), t < 1024
  int Kx, rows;
  long long N;
  float invN;
  LawParams law;
  const int* done;
};

// Barrier of the two warps of pair p (named barrier 1 + p; 0 is the block's). Both warps of a
// pair reach each of these once per row.
__device__ __forceinline__ void pair_sync(int p) {
  if (p == 0) asm volatile("bar.sync 1, 64;" ::: "memory");
  else asm volatile("bar.sync 2, 64;" ::: "memory");
}

// A warp pair per grid row: warp 0 of the pair carries A = line 11 + i line 22, warp 1 carries
// B = line 12. Each builds its sequence's spectrum (Hermitian completion of the kx >= 0
// coefficients) and transforms it to space (an inverse transform); the pair meets, each warp runs
// the law on half of the row's voxels, the pair meets again, and each warp transforms its part of
// the polarization back and writes the pattern's kx columns. Shared memory per pair: SA and SB,
// each holding its sequence's spectrum, its transposes and, between the transforms, the
// sequence in space.
template <bool PLASTIC, int R>
__global__ __maxnreg__(128) void k_fft_row_w(RowWArgs a) {
  constexpr int NC = 3, L = kN;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ DevPhase phs[kMaxPhases];
  const int lane = threadIdx.x & 31, pair = threadIdx.x >> 6, role = (threadIdx.x >> 5) & 1;
  const int Kx = a.Kx;
  int* kxs = reinterpret_cast<int*>(smem);
  float2* SA = reinterpret_cast<float2*>(smem + (((size_t)Kx * sizeof(int) + 15) & ~(size_t)15)) +
               (size_t)pair * kPairRegion;
  float2* SB = SA + kRegion;
  float2* S = role ? SB : SA;   // this warp's region
  for (int i = threadIdx.x; i < Kx; i += blockDim.x) kxs[i] = a.kx[i];
  for (int i = threadIdx.x; i < kMaxPhases; i += blockDim.x) phs[i] = a.law.ph[i];
  __syncthreads();
  grid_dep_wait();
  if (a.done && *a.done) return;   // the same flag value for every thread of the grid
  const float lam0 = a.law.lam0, mu0 = a.law.mu0;
  for (int row = blockIdx.x * R + pair; row < a.rows; row += gridDim.x * R) {
    const float2* Tr = a.T + (long long)row * NC * Kx;
    float2* To = a.Tout + (long long)row * NC * Kx;
    // ---- spectrum: A from lines 11 and 22, B from line 12; loads eight per lane in flight
#pragma unroll
    for (int i = 0; i < 32; ++i) S[lane + 32 * i] = make_float2(0.f, 0.f);
    __syncwarp();
    const float2* l0 = Tr + (role ? 2 * Kx : 0);
#pragma unroll 1
    for (int j0 = 0; j0 < Kx; j0 += 256) {
      float2 c0[8], c1[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + lane + 32 * u;
        c0[u] = c1[u] = make_float2(0.f, 0.f);
        if (j < Kx) {
          c0[u] = l0[j];
          if (!role) c1[u] = Tr[Kx + j];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int j = j0 + lane + 32 * u;
        if (j >= Kx) continue;
        const int k = kxs[j];
        float2 t0 = c0[u], t1 = c1[u];
        const bool self = (k == 0) || (2 * k == L);
        if (self) {
          t0.y = 0.f;
          t1.y = 0.f;
        }
        // t0 + i t1 at k, conj(t0) + i conj(t1) at L - k (t1 = 0 for B)
        S[k] = make_float2(t0.x - t1.y, t0.y + t1.x);
        if (!self) S[L - k] = make_float2(t0.x + t1.y, t1.x - t0.y);
      }
    }
    __syncwarp();
    // the law's first phase ids and internal variables (voxels x = 32 n1 + lane for n1 in this
    // warp's half of the row, kU per step) go out before the transform to space; each law step
    // then loads the next step's while it computes
    constexpr int kU = 2;
    const int nb = 16 * role;
    const long long g0 = (long long)row * L + lane;
    uint8_t pid[kU], pidn[kU];
    float stv[kU][4], stn[kU][4];
    auto load = [&](int n1b, uint8_t* pd, float (*st)[4]) {
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const long long g = g0 + 32 * (n1b + u);
        pd[u] = a.phase[g];
        if (PLASTIC) {
#pragma unroll
          for (int i = 0; i < 4; ++i) st[u][i] = a.state[i * a.N + g];
        }
      }
    };
    load(nb, pid, stv);
    // ---- to space: the conjugate of the forward transform of the conjugate spectrum
    float2 v[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      v[i] = S[lane + 32 * i];
      v[i].y = -v[i].y;
    }
    __syncwarp();
    fwd1024(v, S, a.table, lane);
    // this warp's sequence in space, voxel x at S[x]
#pragma unroll
    for (int i = 0; i < 32; ++i) S[lane + 32 * i] = make_float2(v[i].x, -v[i].y);
    pair_sync(pair);
    // ---- the law
    {
#pragma unroll 1
      for (int n1b = nb; n1b < nb + 16; n1b += kU) {
        if (n1b + kU < nb + 16) load(n1b + kU, pidn, stn);
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int x = 32 * (n1b + u) + lane;
          const float2 qa = SA[x];
          float e6[6] = {qa.x * a.invN, qa.y * a.invN, 0.f, 0.f, 0.f, SB[x].x * a.invN};
          float ep[6] = {0, 0, 0, 0, 0, 0};
          float alpha = 0.f;
          if (PLASTIC) {
            ep[0] = stv[u][0];
            ep[1] = stv[u][1];
            ep[5] = stv[u][2];
            ep[2] = -(ep[0] + ep[1]);
            alpha = stv[u][3];
          }
          LawOut o;
          stress6<PLASTIC>(e6, phs[pid[u]], ep, alpha, o);
          const float tr = e6[0] + e6[1] + e6[2];
          SA[x] = make_float2(o.s[0] - (lam0 * tr + 2.f * mu0 * e6[0]),
                             o.s[1] - (lam0 * tr + 2.f * mu0 * e6[1]));
          SB[x] = make_float2(o.s[5] - 2.f * mu0 * e6[5], 0.f);
        }
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          pid[u] = pidn[u];
#pragma unroll
          for (int i = 0; i < 4; ++i) stv[u][i] = stn[u][i];
        }
      }
    }
    pair_sync(pair);
    // ---- the polarization's coefficients: forward transform, then the pattern's kx columns,
    // B (role 1) directly, A (role 0) separated into lines 11 and 22
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = S[lane + 32 * i];
    __syncwarp();
    fwd1024(v, S, a.table, lane);
#pragma unroll
    for (int i = 0; i < 32; ++i) S[lane + 32 * i] = v[i];
    __syncwarp();
#pragma unroll 4
    for (int j = lane; j < Kx; j += 32) {
      const int k = kxs[j];
      const float2 zk = S[k];
      if (role) {
        float2 z = zk;
        if (k == 0 || 2 * k == L) z.y = 0.f;   // a real line's self-conjugate coefficients
        To[2 * Kx + j] = z;
      } else {
        const float2 zm = S[k == 0 ? 0 : L - k];
        To[j] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        To[Kx + j] = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
      }
    }
    __syncwarp();
  }
}

}  // namespace wfft

size_t row_warp_smem(int Kx, int warps) {
  return (((size_t)Kx * sizeof(int) + 15) & ~(size_t)15) +
         (size_t)(warps / 2) * wfft::kPairRegion * sizeof(float2);
}

bool row_warp_ok(const rf_ctx* c) { return c->dim == 2 && c->nx == wfft::kN && c->nc == 3; }

void init_attributes_fftwarp() {
  const int s = 64 * 1024;
  cudaFuncSetAttribute(wfft::k_fft_row_w<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(wfft::k_fft_row_w<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(wfft::k_fft_row_w<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(wfft::k_fft_row_w<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  // many small blocks per SM: the largest shared-memory carveout
  const int pc = cudaSharedmemCarveoutMaxShared;
  cudaFuncSetAttribute(wfft::k_fft_row_w<true, 1>, cudaFuncAttributePreferredSharedMemoryCarveout, pc);
  cudaFuncSetAttribute(wfft::k_fft_row_w<false, 1>, cudaFuncAttributePreferredSharedMemoryCarveout, pc);
  cudaFuncSetAttribute(wfft::k_fft_row_w<true, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, pc);
  cudaFuncSetAttribute(wfft::k_fft_row_w<false, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, pc);
  cudaGetLastError();
}

// One row pass (not the final one) with c->fft_row_warps (2 or 4) warps per block: one or two
// grid rows per block, a warp pair per row.
int launch_fft_row_warp(rf_ctx* c, const int* done) {
  wfft::RowWArgs a{};
  a.T = c->d_T1;
  a.Tout = c->d_T1p;
  a.phase = c->d_phase;
  a.state = c->d_state;
  a.kx = c->d_kx;
  a.table = c->d_twx;
  a.Kx = c->Kx;
  a.rows = c->rows;
  a.N = c->N;
  a.invN = (float)(1.0 / (double)c->N);
  a.law = c->law;
  a.done = done;
  const int R = c->fft_row_warps / 2;
  const dim3 grid((unsigned)((c->rows + R - 1) / R)), block(64 * R);
  const size_t smem = row_warp_smem(c->Kx, 2 * R);
  const bool pl = c->has_plastic;
  cudaError_t e;
  if (R == 1)
    e = pl ? launch_pdl(wfft::k_fft_row_w<true, 1>, grid, block, smem, c->stream, a)
           : launch_pdl(wfft::k_fft_row_w<false, 1>, grid, block, smem, c->stream, a);
  else
    e = pl ? launch_pdl(wfft::k_fft_row_w<true, 2>, grid, block, smem, c->stream, a)
           : launch_pdl(wfft::k_fft_row_w<false, 2>, grid, block, smem, c->stream, a);
  c->launches += 1;
  if (e != cudaSuccess) return cuda_fail(e, "fft row (warp FFTs)");
  e = cudaGetLastError();
  return e == cudaSuccess ? RF_OK : cuda_fail(e, "fft row (warp FFTs)");
}

}  // namespace rfk
