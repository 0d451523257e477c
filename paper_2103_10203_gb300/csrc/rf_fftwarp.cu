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

// Line-coefficient layouts between the row pass and the column phase: row-major [rows][NC][Kx]
// (every other column mode), or row-group slabs [rows / 4][Kx][4][NC] (the warp-FFT column
// phase): the coefficients of four consecutive rows at one kx are 96 contiguous bytes, so the
// row pass (a block per group of four rows) reads and writes its group as one contiguous block
// and the column phase (a block per kx) reads and writes whole 32-byte sectors.
constexpr int kGroup = 4;
__device__ __forceinline__ long long slab_at(int j, int y, int c, int Kx) {
  return ((((long long)(y >> 2) * Kx + j) << 2) + (y & 3)) * 3 + c;
}

struct RowWArgs {
  const float2* T;      // strain line coefficients (row-major or kx slabs)
  float2* Tout;         // polarization line coefficients (same layout)
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

// Barrier of the two warps of pair p < 4 (named barrier 1 + p; 0 is the block's). Both warps of
// a pair reach each of these once per row.
__device__ __forceinline__ void pair_sync(int p) {
  switch (p) {
    case 0: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
    case 1: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
    case 2: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
    default: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
  }
}

// A warp pair per grid row: warp 0 of the pair carries A = line 11 + i line 22, warp 1 carries
// B = line 12. Each builds its sequence's spectrum (Hermitian completion of the kx >= 0
// coefficients) and transforms it to space (an inverse transform); the pair meets, each warp runs
// the law on half of the row's voxels, the pair meets again, and each warp transforms its part of
// the polarization back and writes the pattern's kx columns. Shared memory per pair: SA and SB,
// each holding its sequence's spectrum, its transposes and, between the transforms, the
// sequence in space. SLAB (R = 4, a block per row group): the group's line coefficients are
// staged in shared memory, loaded and stored by the whole block as one contiguous block.
// One grid row of the row pass for the warp pair of this thread (pair = threadIdx.x / 64 within
// the block; both warps of the pair call it with the same row). SLAB: the whole block calls it
// for the four rows of one group (it stages the group through G with block barriers).
template <bool PLASTIC, bool SLAB>
__device__ __forceinline__ void row_pass(const RowWArgs& a, int row, const int* kxs,
                                         const DevPhase* phs, float2* G, float2* SA, float2* SB) {
  constexpr int NC = 3, L = kN;
  const int lane = threadIdx.x & 31, pair = threadIdx.x >> 6, role = (threadIdx.x >> 5) & 1;
  const int Kx = a.Kx;
  float2* S = role ? SB : SA;   // this warp's region
  const float lam0 = a.law.lam0, mu0 = a.law.mu0;
  const float2* Tr = a.T + (long long)row * NC * Kx;
  float2* To = a.Tout + (long long)row * NC * Kx;
  const int r4 = row & (kGroup - 1);
  if (SLAB) {
    // the group's coefficients: Kx * 96 contiguous bytes, 16-byte loads
    const float4* src = reinterpret_cast<const float4*>(a.T + slab_at(0, row - r4, 0, Kx));
    const int n4 = Kx * kGroup * NC / 2;
    for (int q0 = threadIdx.x; q0 < n4; q0 += 4 * blockDim.x) {
      float4 t[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (q0 + u * (int)blockDim.x < n4) t[u] = __ldcg(src + q0 + u * blockDim.x);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * blockDim.x;
        if (q >= n4) continue;
        // entries 2q, 2q + 1 of [Kx][4][NC]
        const int e = 2 * q, j = e / 12, m = e - 12 * j;
        G[m * Kx + j] = make_float2(t[u].x, t[u].y);
        G[(m + 1) * Kx + j] = make_float2(t[u].z, t[u].w);   // m even: m + 1 < 12
      }
    }
    __syncthreads();
  }
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
        if (SLAB) {
          const float2* p = G + (r4 * NC + (role ? 2 : 0)) * Kx + j;
          c0[u] = p[0];
          if (!role) c1[u] = p[Kx];
        } else {
          c0[u] = l0[j];
          if (!role) c1[u] = Tr[Kx + j];
        }
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
  if (SLAB) __syncthreads();   // the staged group is read; it takes the outputs next
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
      if (SLAB) G[(r4 * NC + 2) * Kx + j] = z;
      else To[2 * Kx + j] = z;
    } else {
      const float2 zm = S[k == 0 ? 0 : L - k];
      const float2 t0 = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      const float2 t1 = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
      if (SLAB) {
        float2* p = G + r4 * NC * Kx + j;
        p[0] = t0;
        p[Kx] = t1;
      } else {
        To[j] = t0;
        To[Kx + j] = t1;
      }
    }
  }
  __syncwarp();
  if (SLAB) {
    // the group's polarization coefficients out with 16-byte stores
    __syncthreads();
    float4* dst = reinterpret_cast<float4*>(a.Tout + slab_at(0, row - r4, 0, Kx));
    const int n4 = Kx * kGroup * NC / 2;
    for (int q = threadIdx.x; q < n4; q += blockDim.x) {
      const int e = 2 * q, j = e / 12, m = e - 12 * j;
      const float2 z0 = G[m * Kx + j], z1 = G[(m + 1) * Kx + j];
      dst[q] = make_float4(z0.x, z0.y, z1.x, z1.y);
    }
    __syncthreads();   // before the next group overwrites the staging
  }
}

template <bool PLASTIC, int R, bool SLAB>
__global__ __maxnreg__(128) void k_fft_row_w(RowWArgs a) {
  constexpr int NC = 3;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ DevPhase phs[kMaxPhases];
  const int pair = threadIdx.x >> 6;
  const int Kx = a.Kx;
  int* kxs = reinterpret_cast<int*>(smem);
  // row-group slabs: the block's group staged in shared memory as [4][NC][Kx] (lanes on
  // consecutive kx read and write it without bank conflicts)
  float2* G = reinterpret_cast<float2*>(smem + (((size_t)Kx * sizeof(int) + 15) & ~(size_t)15));
  float2* SA = G + (SLAB ? (size_t)Kx * kGroup * NC : 0) + (size_t)pair * kPairRegion;
  float2* SB = SA + kRegion;
  for (int i = threadIdx.x; i < Kx; i += blockDim.x) kxs[i] = a.kx[i];
  for (int i = threadIdx.x; i < kMaxPhases; i += blockDim.x) phs[i] = a.law.ph[i];
  __syncthreads();
  grid_dep_wait();
  if (a.done && *a.done) return;   // the same flag value for every thread of the grid
  for (int row = blockIdx.x * R + pair; row < a.rows; row += gridDim.x * R)
    row_pass<PLASTIC, SLAB>(a, row, kxs, phs, G, SA, SB);
}

struct ColWArgs {
  const float2* T1p;      // [Kx][1024][NC] polarization line coefficients (row pass output)
  float2* T1;             // [Kx][1024][NC] strain line coefficients (next row pass input)
  float2* ER;             // [Ky][NC][Kx] strain coefficients on the (ky, kx) rectangle
  const int* jptr;        // [Kx + 1] offsets of each kx's entries in the grouped order
  const int2* jent;       // grouped order: (rectangle row iy, frequency kind)
  const float4* jn;       // grouped order: unit wave vector and multiplicity
  const int* kym;         // position (ky mod Ny) of each rectangle row
  const float2* table;    // exp(+2 pi i t / 1024), t < 1024
  int Kx;
  float inv2mu0, cgam;
  Status* st;
  unsigned* counter;      // blocks finished (reset to 0 by the last block)
  double* part;           // [gridDim.x]
  const int* done;
  cudaGraphConditionalHandle cond;
  int use_cond;
};

constexpr int kColRegion = kRegion + kN;   // a column warp's region: R (1056) and D (1024)

// Column phase of a 2D update on 1024 x 1024 grids (steps b, c, d of Sec. 4 along y, fused), on
// line coefficients in row-group slabs: a block takes M kx values, a warp each of their NC
// component columns. The block loads its kx's 96-byte pieces of every row group (16-byte loads,
// whole sectors) into the warps' regions R; each
// warp transforms its column forward in registers and leaves the spectrum in R; the block applies
// the Green operator at its kx's pattern entries (all NC components of an entry come from the
// regions of the same kx), writes the new coefficients to ER and into the zeroed spectra D, and
// sums the convergence measure; each warp transforms D back to space along y (R as the transpose
// buffer), the block stores its pieces for the next row pass and then writes its FP64 partial of
// the measure (the last block takes the decision). INIT: only the inverse of the coefficients
// held in ER (the start of a solve), no decision.
// The column phase of the kx values j0 .. j0 + M - 1 (those below Kx) for the whole block: warps
// 0 .. 3M - 1 carry the component columns (warp w: kx j0 + w / 3, component w % 3, region
// R0 + w kColRegion); further warps of the block take part in the block-wide loops only. WAIT:
// the pattern's entry data are fetched before the dependency wait and the pass returns false at
// once if the solve is done (else they are fetched just before the Green step). Each thread's
// share of the convergence measure is added to diff. The whole block calls it.
template <int M, bool INIT, bool WAIT, int kB = 4, int kL = 16>
__device__ __forceinline__ bool col_pass(const ColWArgs& a, int j0, float2* R0, double Nd,
                                         double& diff) {
  // kB entries and kL 16-byte slab loads per thread in flight
  constexpr int NC = 3;
  constexpr int kSlab4 = kN * NC / 2;   // float4 of one kx: 256 row groups of 6
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const bool active = w < 3 * M;   // a warp with a component column
  const int nj = min(M, a.Kx - j0);   // kx values of this block
  float2* R = R0 + w * kColRegion;
  float2* D = R + kRegion;
  const int e0 = a.jptr[j0], e1 = a.jptr[j0 + nj];
  const int eM = M == 2 ? a.jptr[j0 + 1] : e1;   // first entry of the second kx
  if (active) {
#pragma unroll
    for (int i = 0; i < 32; ++i) D[lane + 32 * i] = make_float2(0.f, 0.f);
  }
  // the pattern's entry data (fixed with the pattern): the first kB entries of this thread are
  // fetched before the dependency wait
  int2 en[kB];
  float4 nv[kB];
  int pos[kB];
  auto fetch = [&](int eb) {
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int e = eb + u * blockDim.x;
      if (e < e1) {
        en[u] = a.jent[e];
        if (!INIT) nv[u] = a.jn[e];
      }
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int e = eb + u * blockDim.x;
      if (e < e1) pos[u] = a.kym[en[u].x];
    }
  };
  if constexpr (WAIT) {
    fetch(e0 + threadIdx.x);
    grid_dep_wait();
    if (!INIT && a.done && __ldcg(a.done)) return false;   // the same value for every thread
    // the zeroed spectra D before any thread scatters into them (the update's path meets the
    // barrier after its slab loads, the start's has none of its own)
    if (INIT) __syncthreads();
  } else {
    __syncthreads();   // the zeroed spectra D before any thread scatters into them
  }
  float2 v[32];
  if (!INIT) {
    // the block's kx in every row group: 96 contiguous bytes (six float4) per group; float4 k
    // of group g holds the entries 2k, 2k + 1 of [4][NC], i.e. (y - 4 g, c) = divmod(., NC)
    const float4* src = reinterpret_cast<const float4*>(a.T1p);
    for (int q0 = threadIdx.x; q0 < nj * kSlab4; q0 += kL * blockDim.x) {
      float4 t[kL];
#pragma unroll
      for (int u = 0; u < kL; ++u) {
        const int q = q0 + u * blockDim.x;
        if (q < nj * kSlab4) {
          const int jj = q >= kSlab4 ? 1 : 0, r = q - jj * kSlab4, g = r / 6;
          t[u] = __ldcg(src + ((long long)g * a.Kx + j0 + jj) * 6 + (r - 6 * g));
        }
      }
#pragma unroll
      for (int u = 0; u < kL; ++u) {
        const int q = q0 + u * blockDim.x;
        if (q >= nj * kSlab4) continue;
        const int jj = q >= kSlab4 ? 1 : 0, r = q - jj * kSlab4, g = r / 6, e = 2 * (r - 6 * g);
        const int y0 = 4 * g + e / NC, c0 = e % NC;
        const int y1 = 4 * g + (e + 1) / NC, c1 = (e + 1) % NC;
        R0[(jj * NC + c0) * kColRegion + y0] = make_float2(t[u].x, t[u].y);
        R0[(jj * NC + c1) * kColRegion + y1] = make_float2(t[u].z, t[u].w);
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = R[lane + 32 * i];
      __syncwarp();
      fwd1024(v, R, a.table, lane);
#pragma unroll
      for (int i = 0; i < 32; ++i) R[lane + 32 * i] = v[i];
    }
    __syncthreads();
  }
  // Green operator at the block's pattern entries (INIT: the held coefficients), kB per thread
  // with their loads issued together (tau^ read only where it is used: regular frequencies, and
  // the zero frequency under mixed control)
  for (int eb = e0 + threadIdx.x; eb < e1; eb += kB * blockDim.x) {
    float2 old[kB][NC];
    if (!WAIT || eb != e0 + (int)threadIdx.x) fetch(eb);
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int e = eb + u * blockDim.x;
      if (e < e1) {
        const int je = (M == 2 && e >= eM) ? 1 : 0;
        const long long base = ((long long)en[u].x * NC) * a.Kx + j0 + je;
#pragma unroll
        for (int cc = 0; cc < NC; ++cc) old[u][cc] = __ldcg(a.ER + base + (long long)cc * a.Kx);
      }
    }
#pragma unroll
    for (int u = 0; u < kB; ++u) {
      const int e = eb + u * blockDim.x;
      if (e >= e1) continue;
      const int je = (M == 2 && e >= eM) ? 1 : 0;
      if (INIT) {
#pragma unroll
        for (int cc = 0; cc < NC; ++cc)
          R0[(je * NC + cc) * kColRegion + kRegion + pos[u]] = old[u][cc];
        continue;
      }
      const int kind = en[u].y;
      const long long base = ((long long)en[u].x * NC) * a.Kx + j0 + je;
      const bool mixed0 = kind == 1 && a.st->mixed;
      float2 tv[NC];
#pragma unroll
      for (int cc = 0; cc < NC; ++cc)
        tv[cc] = (kind == 0 || mixed0) ? R0[(je * NC + cc) * kColRegion + pos[u]]
                                       : make_float2(0.f, 0.f);
      float er[NC], ei[NC];
      const double* ebar = a.st->ebar;
      double em[6];
      if (mixed0) {
        mixed_macro<NC>(tv, Nd, a.st, em);
        for (int i = 0; i < 6; ++i) a.st->ebar[i] = em[i];
        ebar = em;
      }
      green_update<NC>(kind, nv[u], tv, ebar, Nd, a.inv2mu0, a.cgam, er, ei);
      float d = 0.f;   // one frequency's squared increment (at most six non-negative terms)
#pragma unroll
      for (int cc = 0; cc < NC; ++cc) {
        const float dr = er[cc] - old[u][cc].x, di = ei[cc] - old[u][cc].y;
        const float wc = (comp6<NC>(cc) >= 3) ? 2.f : 1.f;   // Frobenius: shear counted twice
        d = fmaf(nv[u].w * wc, dr * dr + di * di, d);
        const float2 z = make_float2(er[cc], ei[cc]);
        a.ER[base + (long long)cc * a.Kx] = z;
        R0[(je * NC + cc) * kColRegion + kRegion + pos[u]] = z;   // D of warp (je, cc)
      }
      diff += (double)d;
    }
  }
  __syncthreads();   // every spectrum D is complete
  // inverse along y as the conjugate of the forward transform of the conjugate; the column back
  // to R, then the block's pieces out with 16-byte stores; the convergence decision after them
  // (it only gates the next update), so the last block's decision is all that trails the stores
  if (active) {
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      v[i] = D[lane + 32 * i];
      v[i].y = -v[i].y;
    }
    fwd1024(v, R, a.table, lane);
#pragma unroll
    for (int i = 0; i < 32; ++i) R[lane + 32 * i] = make_float2(v[i].x, -v[i].y);
  }
  __syncthreads();
  float4* dst = reinterpret_cast<float4*>(a.T1);
  for (int q = threadIdx.x; q < nj * kSlab4; q += blockDim.x) {
    const int jj = q >= kSlab4 ? 1 : 0, r = q - jj * kSlab4, g = r / 6, e = 2 * (r - 6 * g);
    const int y0 = 4 * g + e / NC, c0 = e % NC;
    const int y1 = 4 * g + (e + 1) / NC, c1 = (e + 1) % NC;
    const float2 z0 = R0[(jj * NC + c0) * kColRegion + y0];
    const float2 z1 = R0[(jj * NC + c1) * kColRegion + y1];
    dst[((long long)g * a.Kx + j0 + jj) * 6 + (r - 6 * g)] = make_float4(z0.x, z0.y, z1.x, z1.y);
  }
  return true;
}

template <int M, bool INIT>
__global__ __launch_bounds__(96 * M) void k_fft_colphase_w(ColWArgs a, double Nd) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[3 * M];
  __shared__ double sh[32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double diff = 0.0;
  if (!col_pass<M, INIT, true>(a, blockIdx.x * M, reinterpret_cast<float2*>(smem), Nd, diff))
    return;
  if constexpr (!INIT) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) diff += __shfl_down_sync(0xffffffffu, diff, o);
    if (lane == 0) red[w] = diff;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int i = 0; i < 3 * M; ++i) t += red[i];
      a.part[blockIdx.x] = t;
      __threadfence();
      last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      decide(a.part, gridDim.x, a.st, sh);
      if (threadIdx.x == 0) {
        *a.counter = 0u;
        // the only call site of the loop condition in this mode: one thread of one block
        if (a.use_cond && a.st->done) cudaGraphSetConditional(a.cond, 0u);
      }
    }
  }
}

// ---- persistent solve on the warp-FFT kernels (one cooperative launch per solve)

struct PersistWArgs {
  RowWArgs row;          // T = T1, Tout = T1p (row-group slabs), no done flag
  ColWArgs col;          // T1p -> T1, status and partials, no done flag
  unsigned* bar;         // [2] arrival count, generation
  long bar_limit;        // polls per barrier wait
  double Nd;
  int n_groups;          // row groups of four rows
  int n_col;             // column items of two kx
  unsigned long long* trace;   // nullable: [trace_cap][3] global-timer stamps per update
  int trace_cap;
};

__device__ __forceinline__ unsigned pw_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long pw_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier over the whole co-resident grid (arrival count and generation word); false if the
// wait ran out after `limit` polls.
__device__ bool pw_grid_sync(unsigned* bar, long limit, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = pw_ld_acquire(bar + 1);
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long it = 0;
      while (pw_ld_acquire(bar + 1) == gen) {
        if (++it > limit) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    *s_flag = ok;
  }
  __syncthreads();
  return *s_flag != 0;
}

// Every update of a 2D 1024^2 solve in one cooperative launch of 256-thread blocks: the start's
// inverse along y of the held coefficients, then per update the row pass over the row groups,
// a grid barrier, the column pass over pairs of kx (writing one FP64 partial each), a grid
// barrier, and the decision, which every block takes identically from the partials in a fixed
// order (block 0 writes the status). The passes are the ones of the launch-per-phase kernels.
template <bool PLASTIC>
__global__ __launch_bounds__(256, 2) void k_persist_w(const __grid_constant__ PersistWArgs a) {
  constexpr int NC = 3;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ DevPhase phs[kMaxPhases];
  __shared__ double red[8];
  __shared__ int s_flag, s_done, s_iters;
  __shared__ double s_rmin;
  __shared__ unsigned long long s_tupd, s_trow;
  const int Kx = a.row.Kx, tid = threadIdx.x, pair = tid >> 6;
  int* kxs = reinterpret_cast<int*>(smem);
  float2* base = reinterpret_cast<float2*>(smem + (((size_t)Kx * sizeof(int) + 15) & ~(size_t)15));
  float2* G = base;                                   // row pass: staged group
  float2* SA = base + (size_t)Kx * kGroup * NC + (size_t)pair * kPairRegion;
  float2* SB = SA + kRegion;
  for (int i = tid; i < Kx; i += blockDim.x) kxs[i] = a.row.kx[i];
  for (int i = tid; i < kMaxPhases; i += blockDim.x) phs[i] = a.row.law.ph[i];
  if (tid == 0) {
    s_iters = a.col.st->iters;
    s_rmin = a.col.st->rmin;
  }
  __syncthreads();
  double d0 = 0.0;
  for (int p = blockIdx.x; p < a.n_col; p += gridDim.x) {
    col_pass<2, true, false, 1, 4>(a.col, 2 * p, base, a.Nd, d0);
    __syncthreads();
  }
  if (!pw_grid_sync(a.bar, a.bar_limit, &s_flag)) {
    if (tid == 0) atomicExch(&a.col.st->timeout, 1);
    return;
  }
  if (a.trace && blockIdx.x == 0 && tid == 0) s_tupd = pw_now();
  for (int u = 0;; ++u) {
    for (int g = blockIdx.x; g < a.n_groups; g += gridDim.x)
      row_pass<PLASTIC, true>(a.row, kGroup * g + pair, kxs, phs, G, SA, SB);
    if (!pw_grid_sync(a.bar, a.bar_limit, &s_flag)) {
      if (tid == 0) atomicExch(&a.col.st->timeout, 1);
      return;
    }
    if (a.trace && blockIdx.x == 0 && tid == 0) s_trow = pw_now();
    for (int p = blockIdx.x; p < a.n_col; p += gridDim.x) {
      double diff = 0.0;
      col_pass<2, false, false, 1, 4>(a.col, 2 * p, base, a.Nd, diff);
      const double t = block_sum_d(diff, red);
      if (tid == 0) a.col.part[p] = t;
    }
    if (!pw_grid_sync(a.bar, a.bar_limit, &s_flag)) {
      if (tid == 0) atomicExch(&a.col.st->timeout, 1);
      return;
    }
    // decision from the partials in a fixed order, the same in every block
    double s = 0.0;
    for (int i = tid; i < a.n_col; i += blockDim.x) s += __ldcg(a.col.part + i);
    s = block_sum_d(s, red);
    if (tid == 0) {
      // tol, enorm, inv_n2 and max_iter are set by the host before the launch
      Status* st = a.col.st;
      double r = sqrt(s * st->inv_n2);
      if (st->enorm > 0.0) r /= st->enorm;
      const int iters = s_iters + 1;
      const double rmin = fmin(s_rmin, r);
      s_iters = iters;
      s_rmin = rmin;
      int done = 0, nonfinite = 0, diverged = 0;
      if (!isfinite(r)) {
        nonfinite = done = 1;
      } else if (r > kDivergeRatio * rmin && r > kDivergeFloor) {
        diverged = done = 1;
      } else if (r < st->tol || iters >= st->max_iter) {
        done = 1;
      }
      if (blockIdx.x == 0) {
        st->iters = iters;
        st->last_r = r;
        st->rmin = rmin;
        st->nonfinite = nonfinite;
        st->diverged = diverged;
        st->done = done;
        if (a.trace && u < a.trace_cap) {
          const unsigned long long t_col = pw_now();
          a.trace[3 * u] = s_tupd;
          a.trace[3 * u + 1] = s_trow;
          a.trace[3 * u + 2] = t_col;
          s_tupd = t_col;
        }
      }
      s_done = done;
    }
    __syncthreads();
    if (s_done) break;
  }
}

}  // namespace wfft

// largest dynamic shared memory of the row kernel (two rows per block) and of the column
// phase (two kx columns per block), set as the kernels' limits
constexpr int kRowWSmemMax = 128 * 1024, kColWSmemMax = 112 * 1024, kPersistWSmemMax = 200 * 1024;

size_t row_warp_smem(int Kx, int warps) {
  // warps = 8: the row-group slab kernel, with its group staged
  return (((size_t)Kx * sizeof(int) + 15) & ~(size_t)15) +
         (warps == 8 ? (size_t)Kx * wfft::kGroup * 3 * sizeof(float2) : 0) +
         (size_t)(warps / 2) * wfft::kPairRegion * sizeof(float2);
}

bool row_warp_ok(const rf_ctx* c) { return c->dim == 2 && c->nx == wfft::kN && c->nc == 3; }

bool col_warp_ok(const rf_ctx* c) {
  return c->dim == 2 && c->nx == wfft::kN && c->ny == wfft::kN && c->nc == 3 &&
         c->d_jptr != nullptr && c->d_jent != nullptr;
}

static size_t col_warp_smem(int M) { return (size_t)3 * M * wfft::kColRegion * sizeof(float2); }

template <int M, bool INIT>
static void set_colw_attributes() {
  cudaFuncSetAttribute(wfft::k_fft_colphase_w<M, INIT>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, kColWSmemMax);
  cudaFuncSetAttribute(wfft::k_fft_colphase_w<M, INIT>,
                       cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
}

template <bool PL, int R, bool SLAB>
static void set_roww_attributes() {
  cudaFuncSetAttribute(wfft::k_fft_row_w<PL, R, SLAB>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, kRowWSmemMax);
  // many small blocks per SM: the largest shared-memory carveout
  cudaFuncSetAttribute(wfft::k_fft_row_w<PL, R, SLAB>,
                       cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
}

// Shared memory of a persistent warp-FFT block: kx values, then the larger of the row pass's
// (staged group and four pair regions) and the column pass's (six column regions)
static size_t persist_w_smem(int Kx) {
  const size_t row = (size_t)Kx * wfft::kGroup * 3 + 4 * (size_t)wfft::kPairRegion;
  const size_t col = 6 * (size_t)wfft::kColRegion;
  return (((size_t)Kx * sizeof(int) + 15) & ~(size_t)15) + std::max(row, col) * sizeof(float2);
}

static const void* persist_w_kernel(bool pl) {
  return pl ? (const void*)wfft::k_persist_w<true> : (const void*)wfft::k_persist_w<false>;
}

void init_attributes_fftwarp() {
  set_roww_attributes<true, 1, false>();
  set_roww_attributes<false, 1, false>();
  set_roww_attributes<true, 2, false>();
  set_roww_attributes<false, 2, false>();
  set_roww_attributes<true, 4, true>();
  set_roww_attributes<false, 4, true>();
  set_colw_attributes<1, false>();
  set_colw_attributes<2, false>();
  set_colw_attributes<1, true>();
  set_colw_attributes<2, true>();
  for (bool pl : {true, false}) {
    cudaFuncSetAttribute(persist_w_kernel(pl), cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kPersistWSmemMax);
    cudaFuncSetAttribute(persist_w_kernel(pl), cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
  }
  cudaGetLastError();
}

// The warp-FFT column phase with c->fft_colw_M (1 or 2) kx columns per block on kx slabs
// (T1p -> Green operator and decision -> T1); init: the inverse along y of the coefficients held
// in ER into T1 (the start of a solve in this mode).
static int colw_launch(rf_ctx* c, const int* done, bool init) {
  wfft::ColWArgs a{};
  a.T1p = c->d_T1p;
  a.T1 = c->d_T1;
  a.ER = c->d_ER;
  a.jptr = c->d_jptr;
  a.jent = c->d_jent;
  a.jn = c->d_jn;
  a.kym = c->d_kym;
  a.table = c->d_twy;
  a.Kx = c->Kx;
  a.inv2mu0 = (float)(0.5 / c->mu0);
  a.cgam = (float)((c->lam0 + c->mu0) / (c->mu0 * (c->lam0 + 2.0 * c->mu0)));
  a.st = c->d_status;
  a.counter = c->d_counter;
  a.part = c->d_part;
  a.done = done;
  a.cond = c->while_cond;
  a.use_cond = (!init && c->capturing_while) ? 1 : 0;
  const int M = c->fft_colw_M;
  if ((M != 1 && M != 2) || col_warp_smem(M) > (size_t)kColWSmemMax) {
    set_error("fft column phase (warp FFTs): kx columns per block must be 1 or 2");
    return RF_ERR_INVALID;
  }
  if (!init) trace_stage(c, 6);
  const dim3 grid((unsigned)((c->Kx + M - 1) / M)), block(96 * M);
  const size_t sm = col_warp_smem(M);
  const double Nd = (double)c->N;
  cudaError_t e;
  if (init)
    e = M == 1 ? launch_pdl(wfft::k_fft_colphase_w<1, true>, grid, block, sm, c->stream, a, Nd)
               : launch_pdl(wfft::k_fft_colphase_w<2, true>, grid, block, sm, c->stream, a, Nd);
  else
    e = M == 1 ? launch_pdl(wfft::k_fft_colphase_w<1, false>, grid, block, sm, c->stream, a, Nd)
               : launch_pdl(wfft::k_fft_colphase_w<2, false>, grid, block, sm, c->stream, a, Nd);
  c->launches += 1;
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fft column phase (warp FFTs)");
  if (!init) trace_end(c);
  return RF_OK;
}

bool persist_warp_ok(const rf_ctx* c) {
  if (!col_warp_ok(c) || !c->d_bar || c->rows % wfft::kGroup != 0) return false;
  const size_t sm = persist_w_smem(c->Kx);
  if (sm > (size_t)kPersistWSmemMax) return false;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persist_w_kernel(c->has_plastic), 256,
                                                    sm) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return occ >= 1;
}

// One cooperative launch: the start's inverse along y, then updates until the decision ends the
// solve (the status on the device holds tol, max_iter and the normalisation).
int launch_persist_warp(rf_ctx* c, unsigned long long* trace, int trace_cap) {
  const size_t sm = persist_w_smem(c->Kx);
  int sms = 152, occ = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
  const void* k = persist_w_kernel(c->has_plastic);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 256, sm) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    set_error("persistent warp-FFT solve: no co-resident grid for this pattern");
    return RF_ERR_INVALID;
  }
  wfft::PersistWArgs a{};
  wfft::RowWArgs& r = a.row;
  r.T = c->d_T1;
  r.Tout = c->d_T1p;
  r.phase = c->d_phase;
  r.state = c->d_state;
  r.kx = c->d_kx;
  r.table = c->d_twx;
  r.Kx = c->Kx;
  r.rows = c->rows;
  r.N = c->N;
  r.invN = (float)(1.0 / (double)c->N);
  r.law = c->law;
  r.done = nullptr;
  wfft::ColWArgs& q = a.col;
  q.T1p = c->d_T1p;
  q.T1 = c->d_T1;
  q.ER = c->d_ER;
  q.jptr = c->d_jptr;
  q.jent = c->d_jent;
  q.jn = c->d_jn;
  q.kym = c->d_kym;
  q.table = c->d_twy;
  q.Kx = c->Kx;
  q.inv2mu0 = (float)(0.5 / c->mu0);
  q.cgam = (float)((c->lam0 + c->mu0) / (c->mu0 * (c->lam0 + 2.0 * c->mu0)));
  q.st = c->d_status;
  q.counter = c->d_counter;
  q.part = c->d_part;
  q.done = nullptr;
  q.use_cond = 0;
  a.bar = c->d_bar;
  a.bar_limit = 1L << 26;
  a.Nd = (double)c->N;
  a.n_groups = c->rows / wfft::kGroup;
  a.n_col = (c->Kx + 1) / 2;
  a.trace = trace;
  a.trace_cap = trace_cap;
  cudaError_t e = cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned), c->stream);
  if (e == cudaSuccess) {
    void* args[] = {&a};
    e = cudaLaunchCooperativeKernel(k, dim3((unsigned)(std::min(occ, 2) * sms)), dim3(256), args,
                                    sm, c->stream);
  }
  c->launches += 1;
  return e == cudaSuccess ? RF_OK : cuda_fail(e, "persistent warp-FFT solve");
}

int launch_fft_colphase_warp(rf_ctx* c, const int* done) { return colw_launch(c, done, false); }

int launch_fft_coly_init_warp(rf_ctx* c) { return colw_launch(c, nullptr, true); }

// One row pass (not the final one) with c->fft_row_warps warps per block, a warp pair per row:
// 2 or 4 (one or two rows per block) on row-major line coefficients, 8 (a row group of four
// rows per block) on row-group slabs when the column phase is the warp-FFT one.
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
  const bool slab = c->fft_colmode == kColWarp;
  const int R = c->fft_row_warps / 2;
  const dim3 grid((unsigned)((c->rows + R - 1) / R)), block(64 * R);
  const size_t smem = row_warp_smem(c->Kx, 2 * R);
  if ((slab ? (R != 4 || c->rows % 4 != 0) : (R != 1 && R != 2)) ||
      smem > (size_t)kRowWSmemMax) {
    set_error("fft row (warp FFTs): one or two rows per block, four on row-group slabs");
    return RF_ERR_INVALID;
  }
  const bool pl = c->has_plastic;
  cudaError_t e;
#define RF_ROWW(P, RR, S) launch_pdl(wfft::k_fft_row_w<P, RR, S>, grid, block, smem, c->stream, a)
  if (slab) e = pl ? RF_ROWW(true, 4, true) : RF_ROWW(false, 4, true);
  else if (R == 1) e = pl ? RF_ROWW(true, 1, false) : RF_ROWW(false, 1, false);
  else e = pl ? RF_ROWW(true, 2, false) : RF_ROWW(false, 2, false);
#undef RF_ROWW
  c->launches += 1;
  if (e != cudaSuccess) return cuda_fail(e, "fft row (warp FFTs)");
  e = cudaGetLastError();
  return e == cudaSuccess ? RF_OK : cuda_fail(e, "fft row (warp FFTs)");
}

}  // namespace rfk
