// FFT transform mode: steps b and d of Sec. 4 as full FFTs along each axis restricted to the
// reduced set (the paper's own choice of transform), for grid sizes 2^b or 3 * 2^b, FP32.
//
// Along x (row kernel, fused with the law): two real lines are packed into one complex
// sequence z = a + i b; the inverse builds z's spectrum from the lines' kx >= 0 coefficients
// (Hermitian completion), transforms back, applies the law per voxel, packs tau the same way,
// transforms forward and separates the two lines' spectra at the pattern's kx columns.
// Along y and z (column kernel): sparse spectra (the pattern's distinct ky or kz values) are
// scattered into full-length sequences for the inverse; the forward keeps only those values.
// The transforms are out-of-place Stockham stages in shared memory (rf_fftcore.cuh), with an
// FP32 twiddle table computed in FP64.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "rf_fftcore.cuh"
#include "rf_internal.cuh"
#include "rf_law.cuh"

namespace rfk {

using fftc::cmul;
using fftc::fft_block;
using fftc::copy_twiddles;
using fftc::sw;

struct FftRowArgs {
  const float2* T;      // [rows][NC][Kx]
  float2* Tout;         // [rows][NC][Kx]
  const uint8_t* phase;
  float* state;
  const int* kx;
  const float2* table;  // twiddle buffer of length Nx (rf_fftcore.cuh)
  int Nx, Kx, rows;
  int rbase, rextra;    // block b holds rows [b rbase + min(b, rextra), ...): rbase rows, one
                        // more for b < rextra
  FastDiv dL, dKx;      // division by Nx and Kx
  long long N;
  float invN;
  LawParams law;
  float* eps_out;
  float* sig_out;
  float* alpha_out;
  double* sbar_part;
  double* viol_part;
  int commit;
  const int* done;
};

template <int NC, bool PLASTIC, bool FINAL>
__global__ __launch_bounds__(512) void k_fft_row(FftRowArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int L = a.Nx;
  const int row0 = blockIdx.x * a.rbase + min((int)blockIdx.x, a.rextra);
  const int R = a.rbase + ((int)blockIdx.x < a.rextra ? 1 : 0);   // rows of this block
  const int S = R * NC;                // real lines in this block
  const int P = (S + 1) / 2;           // packed complex sequences
  float2* tw = reinterpret_cast<float2*>(smem);    // stage twiddles
  float2* b0 = tw + fftc::stage_len(L);
  const int span = fftc::span_of(P * L);
  float2* b1 = b0 + span;
  int* kxs = reinterpret_cast<int*>(b1 + span);   // past b1's rounded span
  __shared__ double red[32];   // one entry per warp
  __shared__ DevPhase phs[kMaxPhases];
  const int tid = threadIdx.x;
  copy_twiddles(a.table, L, tw);
  for (int i = tid; i < a.Kx; i += blockDim.x) kxs[i] = a.kx[i];
  for (int i = tid; i < kMaxPhases; i += blockDim.x) phs[i] = a.law.ph[i];
  for (int i = tid; i < span; i += blockDim.x) b0[i] = make_float2(0.f, 0.f);
  grid_dep_wait();
  const int dn = (!FINAL && a.done) ? *a.done : 0;   // the same flag value for every thread
  // spectra: line s = r * NC + c is the real (s even) or imaginary (s odd) carrier of p = s / 2
  // coefficients are loaded in register batches (both carriers), then scattered: the real
  // carriers write, and after a barrier the imaginary carriers add. The batch loop's trip count
  // is the same for every thread (it contains barriers).
  constexpr int kBatch = 8;
  const int nsc = P * a.Kx;
  float2 tl[2][kBatch];
  auto load_batch = [&](int base) {
#pragma unroll
    for (int pass = 0; pass < 2; ++pass)
#pragma unroll
      for (int m = 0; m < kBatch; ++m) {
        tl[pass][m] = make_float2(0.f, 0.f);
        const int u = base + tid + m * blockDim.x;
        if (u < nsc) {
          const int p = fdiv(u, a.dKx), j = u - p * a.Kx;
          const int s = 2 * p + pass;
          const int r = s / NC, c = s - r * NC, row = row0 + r;
          if (s < S && row < a.rows) tl[pass][m] = a.T[((long long)row * NC + c) * a.Kx + j];
        }
      }
  };
  // the first batch goes out together with the flag (discarded if it is set)
  load_batch(0);
  if (dn) return;
  __syncthreads();   // the zeroed buffer
  for (int base = 0; base < nsc; base += kBatch * blockDim.x) {
    if (base > 0) load_batch(base);
#pragma unroll
    for (int m = 0; m < kBatch; ++m) {
      const int u = base + tid + m * blockDim.x;
      if (u >= nsc) continue;
      const int p = fdiv(u, a.dKx), j = u - p * a.Kx;
      float2 t = tl[0][m];
      const int k = kxs[j];
      const bool self = (k == 0) || (2 * k == L);
      if (self) t.y = 0.f;
      const int zb0 = p * L;
      b0[sw(zb0 + k)] = t;
      if (!self) b0[sw(zb0 + L - k)] = make_float2(t.x, -t.y);
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kBatch; ++m) {
      const int u = base + tid + m * blockDim.x;
      if (u >= nsc) continue;
      const int p = fdiv(u, a.dKx), j = u - p * a.Kx;
      if (2 * p + 1 >= S) continue;
      float2 t = tl[1][m];
      const int k = kxs[j];
      const bool self = (k == 0) || (2 * k == L);
      if (self) t.y = 0.f;
      const int zb0 = p * L;
      float2& zk = b0[sw(zb0 + k)];
      zk.x -= t.y;        // add i * t at k and i * conj(t) at L - k
      zk.y += t.x;
      if (!self) {
        float2& zm = b0[sw(zb0 + L - k)];
        zm.x += t.y;
        zm.y += t.x;
      }
    }
    __syncthreads();
  }
  float2* zb = fft_block(b0, b1, tw, L, P, +1);
  float2* other = (zb == b0) ? b1 : b0;
  double sb[6] = {0, 0, 0, 0, 0, 0};
  double vmax = 0.0;
  const float lam0 = a.law.lam0, mu0 = a.law.mu0;
  constexpr int kVox = 4;
  constexpr int NS = NC == 3 ? 4 : 7;
  for (int vb = 0; vb < R * L; vb += kVox * blockDim.x) {
    int pid[kVox];
    float stv[kVox][NS];
#pragma unroll
    for (int u = 0; u < kVox; ++u) {
      const int v = vb + tid + u * blockDim.x;
      const int r = fdiv(v, a.dL), x = v - r * L, row = row0 + r;
      pid[u] = 0;
      if (v < R * L && row < a.rows) {
        const long long g = (long long)row * L + x;
        pid[u] = a.phase[g];
        if (PLASTIC) {
#pragma unroll
          for (int i = 0; i < NS; ++i) stv[u][i] = a.state[i * a.N + g];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kVox; ++u) {
      const int v = vb + tid + u * blockDim.x;
      if (v >= R * L) continue;
      const int r = fdiv(v, a.dL), x = v - r * L, row = row0 + r;
      float e[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int s = r * NC + c;
        const float2 z = zb[sw((s >> 1) * L + x)];
        e[c] = ((s & 1) ? z.y : z.x) * a.invN;
      }
      float tau6[6] = {0, 0, 0, 0, 0, 0};
      if (row < a.rows) {
        const long long g = (long long)row * L + x;
        float e6[6];
        comp_to6<NC>(e, e6);
        const DevPhase ph = phs[pid[u]];
        float ep[6] = {0, 0, 0, 0, 0, 0};
        float alpha = 0.f;
        if (PLASTIC) {
          if (NC == 3) {
            ep[0] = stv[u][0];
            ep[1] = stv[u][1];
            ep[5] = stv[u][2];
            ep[2] = -(ep[0] + ep[1]);
            alpha = stv[u][3];
          } else {
#pragma unroll
            for (int i = 0; i < 6; ++i) ep[i] = stv[u][i];
            alpha = stv[u][NS - 1];
          }
        }
        LawOut o;
        stress6<PLASTIC>(e6, ph, ep, alpha, o);
        if (!FINAL) {
          const float tr = e6[0] + e6[1] + e6[2];
#pragma unroll
          for (int i = 0; i < 3; ++i) tau6[i] = o.s[i] - (lam0 * tr + 2.f * mu0 * e6[i]);
#pragma unroll
          for (int i = 3; i < 6; ++i) tau6[i] = o.s[i] - 2.f * mu0 * e6[i];
        } else {
#pragma unroll
          for (int i = 0; i < 6; ++i) sb[i] += (double)o.s[i];
          if (a.eps_out) {
#pragma unroll
            for (int i = 0; i < 6; ++i) a.eps_out[i * a.N + g] = e6[i];
          }
          if (a.sig_out) {
#pragma unroll
            for (int i = 0; i < 6; ++i) a.sig_out[i * a.N + g] = o.s[i];
          }
          if (PLASTIC) {
            if (a.commit) store_state<NC>(a.state, a.N, g, o.ep, o.alpha);
            if (a.alpha_out) a.alpha_out[g] = o.alpha;
            if (o.yielded) {
              double s0 = o.s[0], s1 = o.s[1], s2 = o.s[2];
              double pmd = (s0 + s1 + s2) / 3.0;
              double d0 = s0 - pmd, d1 = s1 - pmd, d2 = s2 - pmd;
              double qq = d0 * d0 + d1 * d1 + d2 * d2 +
                          2.0 * ((double)o.s[3] * o.s[3] + (double)o.s[4] * o.s[4] +
                                 (double)o.s[5] * o.s[5]);
              double yl = (double)ph.sy + (double)ph.H * (double)o.alpha;
              vmax = fmax(vmax, fabs(sqrt(1.5 * qq) - yl) / (double)ph.sy);
            }
          } else if (a.alpha_out) {
            a.alpha_out[g] = 0.f;
          }
        }
      }
      if (!FINAL) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int s = r * NC + c;
          float* dst = reinterpret_cast<float*>(other + sw((s >> 1) * L + x));
          dst[s & 1] = tau6[comp6<NC>(c)];
        }
      }
    }
  }
  if (FINAL) {
    for (int i = 0; i < 6; ++i) {
      double t = block_sum_d(sb[i], red);
      if (tid == 0) a.sbar_part[blockIdx.x * 6 + i] = t;
    }
    double vm = block_max_d(vmax, red);
    if (tid == 0) a.viol_part[blockIdx.x] = vm;
    return;
  }
  // an odd line count leaves the last sequence's imaginary carrier unused: zero it
  if (S & 1)
    for (int x = tid; x < L; x += blockDim.x) other[sw((P - 1) * L + x)].y = 0.f;
  __syncthreads();
  float2* zf = fft_block(other, zb, tw, L, P, -1);
  for (int u = tid; u < S * a.Kx; u += blockDim.x) {
    const int s = fdiv(u, a.dKx), j = u - s * a.Kx;
    const int r = s / NC, c = s - r * NC, row = row0 + r;
    if (row >= a.rows) continue;
    const int k = kxs[j];
    const int zb0 = (s >> 1) * L;
    const float2 zk = zf[sw(zb0 + k)], zm = zf[sw(zb0 + (k == 0 ? 0 : L - k))];
    float2 out;
    if ((s & 1) == 0) out = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    else out = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    a.Tout[((long long)row * NC + c) * a.Kx + j] = out;
  }
}

struct FftColArgs {
  const float2* in;
  long long in_bstride;
  int in_rows;            // rows of `in` (sparse count if in_list)
  const int* in_list;     // nullable: row i holds position in_list[i] (reduced mod L)
  float2* out;
  long long out_bstride;
  int out_rows;
  const int* out_list;    // nullable: output row i = position out_list[i]
  int ncols, L, C, sign;
  FastDiv dC;
  const float2* table;
  const int* done;
};

// columns [col0, col0 + C) of a row-major [rows][ncols] array, batched over blockIdx.y
__global__ __launch_bounds__(256) void k_fft_cols(FftColArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int L = a.L, C = a.C;
  float2* tw = reinterpret_cast<float2*>(smem);
  float2* b0 = tw + fftc::stage_len(L);
  const int span = fftc::span_of(C * L);
  float2* b1 = b0 + span;
  const int col0 = blockIdx.x * C;
  const long long b = blockIdx.y;
  const float2* in = a.in + b * a.in_bstride;
  float2* out = a.out + b * a.out_bstride;
  copy_twiddles(a.table, L, tw);
  if (a.in_list)
    for (int i = threadIdx.x; i < span; i += blockDim.x) b0[i] = make_float2(0.f, 0.f);
  grid_dep_wait();
  // loads are issued in batches of 8 per thread before they are stored, so their latencies
  // overlap; the first batch goes out together with the flag (discarded if it is set)
  const int dn = a.done ? *a.done : 0;   // the same flag value for every thread of the block
  const int total = a.in_rows * C;
  float2 v[8];
  int dst[8];
  auto load_batch = [&](int i0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * blockDim.x;
      v[u] = make_float2(0.f, 0.f);
      dst[u] = -1;
      if (i < total) {
        const int r = fdiv(i, a.dC), cc = i - r * C, col = col0 + cc;
        if (col < a.ncols) v[u] = in[(long long)r * a.ncols + col];
        dst[u] = cc * L + (a.in_list ? a.in_list[r] : r);
      }
    }
  };
  load_batch(threadIdx.x);
  if (dn) return;
  __syncthreads();   // the zeroed buffer
  for (int i0 = threadIdx.x;;) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (dst[u] >= 0) b0[sw(dst[u])] = v[u];
    i0 += 8 * blockDim.x;
    if (i0 >= total) break;
    load_batch(i0);
  }
  __syncthreads();
  const float2* z = fft_block(b0, b1, tw, L, C, a.sign);
  for (int i = threadIdx.x; i < a.out_rows * C; i += blockDim.x) {
    const int r = fdiv(i, a.dC), cc = i - r * C, col = col0 + cc;
    if (col >= a.ncols) continue;
    const int pos = a.out_list ? a.out_list[r] : r;
    out[(long long)r * a.ncols + col] = z[sw(cc * L + pos)];
  }
}

// Fused column phase (2D): steps b to d of Sec. 4 between two row passes for a group of M
// consecutive kx columns with all NC components. The forward transforms along y of the
// polarization lines give tau^ at every ky; the Green operator of the reference medium
// (Sec. 3) turns tau^ into the new strain coefficients at the group's pattern entries
// (eps^ = -Gamma0 : tau^, N ebar at the zero frequency, 0 at null frequencies), which are
// stored, summed into the convergence measure (FP64 block partials; the last block takes the
// decision) and scattered into zeroed columns for the inverse transforms along y. Frequencies
// of different kx never meet in these steps, so each group is independent of the others.
struct ColPhaseArgs {
  const float2* T1p;      // [ny][NC][Kx] polarization line coefficients (row pass output)
  float2* T1;             // [ny][NC][Kx] strain line coefficients (next row pass input)
  float2* ER;             // [Ky][NC][Kx] strain coefficients on the (ky, kx) rectangle
  const int* jptr;        // [Kx + 1]
  const int* jlist;       // half-pattern entries grouped by kx index
  const HIdx* hidx;
  const float4* hn;       // unit wave vector and multiplicity
  const int* kym;         // position (ky mod Ny) of each rectangle row
  const float2* table;    // twiddle buffer of length Ny
  int Kx, L, M;
  FastDiv dC;             // division by NC * M
  float inv2mu0, cgam;
  Status* st;
  unsigned* counter;      // blocks finished (reset to 0 by the last block)
  double* part;           // [gridDim.x]
  const int* done;
  cudaGraphConditionalHandle cond;
  int use_cond;
};

template <int NC>
__global__ __launch_bounds__(256) void k_fft_colphase(ColPhaseArgs a, double Nd) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[8];
  __shared__ double sh[32];
  __shared__ bool last;
  const int L = a.L, M = a.M, C = NC * M;   // sequence q = jj NC + c
  const int j0 = blockIdx.x * M;
  float2* tw = reinterpret_cast<float2*>(smem);
  float2* b0 = tw + fftc::stage_len(L);
  const int span = fftc::span_of(C * L);
  float2* b1 = b0 + span;
  copy_twiddles(a.table, L, tw);
  const int e0 = a.jptr[j0], e1 = a.jptr[min(j0 + M, a.Kx)];
  grid_dep_wait();
  if (a.done && __ldcg(a.done)) return;   // the same flag value for every thread of the grid
  // polarization lines of the group, loads in batches of 8 (kx past the last column read 0)
  const int tot = L * C;
  for (int i0 = threadIdx.x; i0 < tot; i0 += 8 * blockDim.x) {
    float2 v[8];
    int dst[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * blockDim.x;
      v[u] = make_float2(0.f, 0.f);
      dst[u] = -1;
      if (i < tot) {
        const int y = fdiv(i, a.dC), q = i - y * C;
        const int jj = q / NC, c = q - jj * NC;
        if (j0 + jj < a.Kx) v[u] = a.T1p[((long long)y * NC + c) * a.Kx + j0 + jj];
        dst[u] = q * L + y;
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (dst[u] >= 0) b0[sw(dst[u])] = v[u];
  }
  __syncthreads();
  const float2* z = fft_block(b0, b1, tw, L, C, -1);
  float2* w = (z == b0) ? b1 : b0;   // free after the last stage's barrier
  for (int i = threadIdx.x; i < span; i += blockDim.x) w[i] = make_float2(0.f, 0.f);
  __syncthreads();
  double diff = 0.0;
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    const int h = a.jlist[e];
    const HIdx hi = a.hidx[h];
    const float4 n = a.hn[h];
    const int jj = hi.j - j0, pos = a.kym[hi.iy];
    const long long base = ((long long)hi.iy * NC) * a.Kx + hi.j;
    // tau^ is read only where it is used: regular frequencies, and the zero frequency under
    // mixed control
    const bool mixed0 = hi.kind == 1 && a.st->mixed;
    float2 tv[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c)
      tv[c] = (hi.kind == 0 || mixed0) ? z[sw((jj * NC + c) * L + pos)] : make_float2(0.f, 0.f);
    float er[NC], ei[NC];
    const double* eb = a.st->ebar;
    double em[6];
    if (mixed0) {
      mixed_macro<NC>(tv, Nd, a.st, em);
      for (int i = 0; i < 6; ++i) a.st->ebar[i] = em[i];
      eb = em;
    }
    green_update<NC>(hi.kind, n, tv, eb, Nd, a.inv2mu0, a.cgam, er, ei);
    float d = 0.f;   // one frequency's squared increment (at most six non-negative terms)
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float2 old = a.ER[base + (long long)c * a.Kx];
      const float dr = er[c] - old.x, di = ei[c] - old.y;
      const float wc = (comp6<NC>(c) >= 3) ? 2.f : 1.f;   // Frobenius: shear counted twice
      d = fmaf(n.w * wc, dr * dr + di * di, d);
      const float2 nv = make_float2(er[c], ei[c]);
      a.ER[base + (long long)c * a.Kx] = nv;
      w[sw((jj * NC + c) * L + pos)] = nv;
    }
    diff += (double)d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) diff += __shfl_down_sync(0xffffffffu, diff, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = diff;
  __syncthreads();   // also orders the scattered coefficients before the inverse transforms
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
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
  const float2* zi = fft_block(w, const_cast<float2*>(z), tw, L, C, +1);
  for (int i = threadIdx.x; i < tot; i += blockDim.x) {
    const int y = fdiv(i, a.dC), q = i - y * C;
    const int jj = q / NC, c = q - jj * NC;
    if (j0 + jj < a.Kx) a.T1[((long long)y * NC + c) * a.Kx + j0 + jj] = zi[sw(q * L + y)];
  }
}

// Green operator inside the inverse transform along y (2D): a block takes C line columns
// (column col = c Kx + kx) and, for every pattern entry of each column's kx, reads tau^ of all
// NC components from the forward transform's rectangle, applies eps^ = -Gamma0 : tau^ (Sec. 3,
// Sec. 4 step c; N ebar at the zero frequency, 0 at null frequencies) and keeps its own
// component c: stored to ER, summed into the convergence measure (FP64 block partials; the
// last block takes the decision) and scattered into the zeroed column for the inverse FFT
// (Sec. 4 step d). Each frequency's operator is evaluated once per component; nothing else is
// shared between blocks.
struct GreenInvArgs {
  const float2* OUT;      // [Ky][NC][Kx] tau^ on the (ky, kx) rectangle
  float2* ER;             // [Ky][NC][Kx]
  float2* T1;             // [ny][NC][Kx]
  const int* jptr;        // [Kx + 1]
  const int2* jent;       // kx-grouped entries: rectangle row iy, frequency kind
  const float4* jn;       // kx-grouped entries: unit wave vector, multiplicity
  const int* kym;
  const float2* table;    // twiddle buffer of length Ny
  int Kx, L, C, ncols;
  FastDiv dC, dKx;
  float inv2mu0, cgam;
  Status* st;
  unsigned* counter;
  double* part;
  const int* done;
  cudaGraphConditionalHandle cond;
  int use_cond;
};

template <int NC>
__global__ __launch_bounds__(256) void k_fft_green_inv(GreenInvArgs a, double Nd) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[8];
  __shared__ double sh[32];
  __shared__ bool last;
  __shared__ int cbeg[65], ckx[64], cc_[64];   // flattened entry ranges of the block's columns
  const int L = a.L, C = a.C;
  float2* tw = reinterpret_cast<float2*>(smem);
  float2* b0 = tw + fftc::stage_len(L);
  const int span = fftc::span_of(C * L);
  float2* b1 = b0 + span;
  const int col0 = blockIdx.x * C;
  const int ncc = min(C, a.ncols - col0);
  if (threadIdx.x == 0) {
    int t = 0;
    for (int cc = 0; cc < ncc; ++cc) {
      const int col = col0 + cc, c = fdiv(col, a.dKx), kx = col - c * a.Kx;
      cbeg[cc] = t;
      ckx[cc] = kx;
      cc_[cc] = c;
      t += a.jptr[kx + 1] - a.jptr[kx];
    }
    cbeg[ncc] = t;
  }
  copy_twiddles(a.table, L, tw);
  for (int i = threadIdx.x; i < span; i += blockDim.x) b0[i] = make_float2(0.f, 0.f);
  __syncthreads();
  // the entries' data does not depend on the previous kernel: load it before waiting
  constexpr int kE = 4;
  const int tot = cbeg[ncc];
  int ecc[kE], epos[kE], eiy[kE], ekind[kE];
  float4 en[kE];
#pragma unroll
  for (int u = 0; u < kE; ++u) {
    const int t = threadIdx.x + u * blockDim.x;
    ecc[u] = -1;
    if (t < tot) {
      int cc = 0;
      while (t >= cbeg[cc + 1]) ++cc;
      const int e = a.jptr[ckx[cc]] + (t - cbeg[cc]);
      const int2 en2 = a.jent[e];
      ecc[u] = cc;
      eiy[u] = en2.x;
      ekind[u] = en2.y;
      en[u] = a.jn[e];
      epos[u] = a.kym[en2.x];
    }
  }
  grid_dep_wait();
  if (a.done && __ldcg(a.done)) return;   // the same flag value for every thread of the grid
  double diff = 0.0;
  // tau^ (all components) and the old coefficient of every entry, loads issued together
  float2 tv[kE][NC], old[kE];
#pragma unroll
  for (int u = 0; u < kE; ++u) {
    if (ecc[u] < 0) continue;
    const long long base = ((long long)eiy[u] * NC) * a.Kx + ckx[ecc[u]];
#pragma unroll
    for (int q = 0; q < NC; ++q) tv[u][q] = a.OUT[base + (long long)q * a.Kx];
    old[u] = a.ER[base + (long long)cc_[ecc[u]] * a.Kx];
  }
#pragma unroll
  for (int u = 0; u < kE; ++u) {
    if (ecc[u] < 0) continue;
    const int c = cc_[ecc[u]];
    float erc[NC], eic[NC], er = 0.f, ei = 0.f;
    const double* eb = a.st->ebar;
    double em[6];
    if (ekind[u] == 1 && a.st->mixed) {   // one of NC blocks (component c) meets it; c 0 writes
      mixed_macro<NC>(tv[u], Nd, a.st, em);
      if (c == 0)
        for (int i = 0; i < 6; ++i) a.st->ebar[i] = em[i];
      eb = em;
    }
    green_update<NC>(ekind[u], en[u], tv[u], eb, Nd, a.inv2mu0, a.cgam, erc, eic);
#pragma unroll
    for (int q = 0; q < NC; ++q)   // keep this block's component (no dynamic register index)
      if (q == c) {
        er = erc[q];
        ei = eic[q];
      }
    const float dr = er - old[u].x, di = ei - old[u].y;
    const int c6 = NC == 3 ? (c == 2 ? 5 : c) : c;
    const float wc = c6 >= 3 ? 2.f : 1.f;   // Frobenius: shear counted twice
    diff += (double)(en[u].w * wc * (dr * dr + di * di));
    const float2 nv = make_float2(er, ei);
    a.ER[((long long)eiy[u] * NC + c) * a.Kx + ckx[ecc[u]]] = nv;
    b0[sw(ecc[u] * L + epos[u])] = nv;
  }
  // entries beyond kE per thread (columns denser than kE x blockDim entries together)
  for (int t = threadIdx.x + kE * blockDim.x; t < tot; t += blockDim.x) {
    int cc = 0;
    while (t >= cbeg[cc + 1]) ++cc;
    const int e = a.jptr[ckx[cc]] + (t - cbeg[cc]);
    const int2 en2 = a.jent[e];
    const float4 n = a.jn[e];
    const int c = cc_[cc], kx = ckx[cc];
    const long long base = ((long long)en2.x * NC) * a.Kx + kx;
    const bool mixed0 = en2.y == 1 && a.st->mixed;
    float2 tq[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q)
      tq[q] = (en2.y == 0 || mixed0) ? a.OUT[base + (long long)q * a.Kx] : make_float2(0.f, 0.f);
    float erc[NC], eic[NC], er = 0.f, ei = 0.f;
    const double* eb = a.st->ebar;
    double em[6];
    if (mixed0) {
      mixed_macro<NC>(tq, Nd, a.st, em);
      if (c == 0)
        for (int i = 0; i < 6; ++i) a.st->ebar[i] = em[i];
      eb = em;
    }
    green_update<NC>(en2.y, n, tq, eb, Nd, a.inv2mu0, a.cgam, erc, eic);
#pragma unroll
    for (int q = 0; q < NC; ++q)
      if (q == c) {
        er = erc[q];
        ei = eic[q];
      }
    float2* erp = a.ER + base + (long long)c * a.Kx;
    const float2 o = *erp;
    const float dr = er - o.x, di = ei - o.y;
    const int c6 = NC == 3 ? (c == 2 ? 5 : c) : c;
    const float wc = c6 >= 3 ? 2.f : 1.f;
    diff += (double)(n.w * wc * (dr * dr + di * di));
    const float2 nv = make_float2(er, ei);
    *erp = nv;
    b0[sw(cc * L + a.kym[en2.x])] = nv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) diff += __shfl_down_sync(0xffffffffu, diff, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = diff;
  __syncthreads();   // also orders the scattered coefficients before the transforms
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
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
  const float2* z = fft_block(b0, b1, tw, L, C, +1);
  for (int i = threadIdx.x; i < L * C; i += blockDim.x) {
    const int y = fdiv(i, a.dC), cc = i - y * C, col = col0 + cc;
    if (col < a.ncols) a.T1[(long long)y * a.ncols + col] = z[sw(cc * L + y)];
  }
}

// ------------------------------------------------------------------------------------------
// host side
static int fft_check(rf_ctx* c, const char* what) {
  c->launches += 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RF_OK : cuda_fail(e, what);
}

static size_t cols_smem(int L, int C) {
  return ((size_t)fftc::stage_len(L) + 2 * (size_t)fftc::span_of(C * L)) * sizeof(float2);
}

static size_t row_smem(int L, int nc, int Kx, int R) {
  const int P = (R * nc + 1) / 2;
  return ((size_t)fftc::stage_len(L) + 2 * (size_t)fftc::span_of(P * L)) * sizeof(float2) +
         (size_t)Kx * sizeof(int) +
         16;
}

constexpr size_t kFftSmemMax = 200 * 1024;

static size_t colphase_smem(int L, int nc, int M) {
  return ((size_t)fftc::stage_len(L) + 2 * (size_t)fftc::span_of(nc * M * L)) * sizeof(float2);
}

static int fft_cols(rf_ctx* c, const float2* in, long long in_bs, int in_rows, const int* in_list,
                    float2* out, long long out_bs, int out_rows, const int* out_list, int ncols,
                    int L, int batch, int sign, const float2* tab, const int* done) {
  FftColArgs a;
  a.in = in;
  a.in_bstride = in_bs;
  a.in_rows = in_rows;
  a.in_list = in_list;
  a.out = out;
  a.out_bstride = out_bs;
  a.out_rows = out_rows;
  a.out_list = out_list;
  a.ncols = ncols;
  a.L = L;
  a.C = std::max(1, std::min(c->fft_C, a.ncols));
  a.dC = make_fastdiv((unsigned)a.C);
  a.sign = sign;
  a.table = tab;
  a.done = done;
  const size_t smem = cols_smem(L, a.C);
  dim3 grid((ncols + a.C - 1) / a.C, batch);
  cudaError_t e = launch_pdl(k_fft_cols, grid, dim3(c->fft_col_threads), smem, c->stream, a);
  if (e != cudaSuccess) return cuda_fail(e, "fft cols");
  return fft_check(c, "fft cols");
}

// rows per row-kernel block (default: about 6144 complex points per ping-pong buffer) and
// columns per column-kernel block (default: 4096 / L points); the autotuner may replace both
static void set_rows(rf_ctx* c, int R) {
  R = std::max(1, std::min(R, c->rows));
  c->fft_R = R;
  c->fft_rbase = R;
  c->fft_rextra = 0;
  c->fft_blocks = (c->rows + R - 1) / R;
  c->fft_smem = row_smem(c->nx, c->nc, c->Kx, R);
}

// nb blocks holding floor(rows / nb) or one more rows each, the larger blocks first: when the
// first wave places one block per SM and nb is a multiple of the SM count, every SM ends up
// with a balanced share of rows
static void set_rows_balanced(rf_ctx* c, int nb) {
  nb = std::max(1, std::min(nb, c->rows));
  c->fft_rbase = c->rows / nb;
  c->fft_rextra = c->rows % nb;
  c->fft_R = c->fft_rbase + (c->fft_rextra > 0 ? 1 : 0);
  c->fft_blocks = nb;
  c->fft_smem = row_smem(c->nx, c->nc, c->Kx, c->fft_R);
}

int fft_geometry(rf_ctx* c) {
  const int L = c->nx;
  if (c->opt.fft_row_blocks > 0) set_rows_balanced(c, c->opt.fft_row_blocks);
  else set_rows(c, c->opt.fft_rows > 0 ? c->opt.fft_rows : (2 * 6144) / (c->nc * L));
  if (c->fft_smem > kFftSmemMax) {
    set_error("FFT mode: rows too long for the row kernel's shared memory");
    return RF_ERR_INVALID;
  }
  int C = c->opt.fft_cols > 0 ? c->opt.fft_cols : std::max(1, std::min(32, 4096 / c->ny));
  const int Lc = std::max(c->ny, c->dim == 3 ? c->nz : 1);
  while (C > 1 && cols_smem(Lc, C) > kFftSmemMax) --C;
  if (cols_smem(Lc, C) > kFftSmemMax) {
    set_error("FFT mode: columns too long for the column kernel's shared memory");
    return RF_ERR_INVALID;
  }
  c->fft_C = C;
  c->fft_row_warps = (c->opt.fft_row_warps > 0 && row_warp_ok(c)) ? c->opt.fft_row_warps : 0;
  // fused column phase (2D): kx columns per block within shared memory
  c->fft_colmode = kColSeparate;
  c->fft_M = std::max(1, std::min(c->opt.fft_fuse_kx > 0 ? c->opt.fft_fuse_kx : 1, c->Kx));
  c->fft_M_threads = 256;
  if (c->dim == 2 && c->opt.fft_fuse >= 0) {
    while (c->fft_M > 1 && colphase_smem(c->ny, c->nc, c->fft_M) > kFftSmemMax) --c->fft_M;
    const bool fits = colphase_smem(c->ny, c->nc, c->fft_M) <= kFftSmemMax;
    if (c->opt.fft_fuse == 3) c->fft_colmode = kColPersistent;   // geometry set with the pattern
    if (c->opt.fft_fuse == 1) {
      if (!fits) {
        set_error("FFT mode: columns too long for the fused column kernel's shared memory");
        return RF_ERR_INVALID;
      }
      c->fft_colmode = kColFused;
    } else if (c->opt.fft_fuse == 2) {
      c->fft_colmode = kColGreenInv;
    } else if (c->opt.fft_fuse == 4) {
      if (c->nx != 1024 || c->ny != 1024 || c->nc != 3 ||
          (c->opt.fft_row_warps != 0 && c->opt.fft_row_warps != 8)) {
        set_error("FFT mode: the warp-FFT column phase needs a 1024 x 1024 grid in 2D and the "
                  "warp-FFT row kernel");
        return RF_ERR_INVALID;
      }
      c->fft_colmode = kColWarp;
      c->fft_colw_M = c->opt.fft_fuse_kx > 0 ? c->opt.fft_fuse_kx : 1;
      c->fft_row_warps = 8;   // the row-group slab row kernel
    } else if (c->opt.fft_fuse == 5) {
      if (c->nx != 1024 || c->ny != 1024 || c->nc != 3) {
        set_error("FFT mode: the persistent warp-FFT solve needs a 1024 x 1024 grid in 2D");
        return RF_ERR_INVALID;
      }
      c->fft_colmode = kColPersistW;
      c->fft_colw_M = 2;
      c->fft_row_warps = 8;
    }
  }
  return RF_OK;
}

static FftRowArgs fft_row_args(rf_ctx* c, const int* done) {
  FftRowArgs a{};
  a.T = c->d_T1;
  a.Tout = c->d_T1p;
  a.phase = c->d_phase;
  a.state = c->d_state;
  a.kx = c->d_kx;
  a.table = c->d_twx;
  a.Nx = c->nx;
  a.Kx = c->Kx;
  a.dL = make_fastdiv((unsigned)c->nx);
  a.dKx = make_fastdiv((unsigned)std::max(1, c->Kx));
  a.rows = c->rows;
  a.rbase = c->fft_rbase;
  a.rextra = c->fft_rextra;
  a.N = c->N;
  a.invN = (float)(1.0 / (double)c->N);
  a.law = c->law;
  a.done = done;
  return a;
}

void init_attributes_fft() {
  const int s = 200 * 1024;
  cudaFuncSetAttribute(k_fft_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_fft_colphase<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_fft_green_inv<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_fft_row<3, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_fft_row<3, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_fft_row<3, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_fft_row<3, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_fft_row<6, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_fft_row<6, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_fft_row<6, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_fft_row<6, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
}

template <int NC, bool PL, bool FIN>
static int fft_row_launch(rf_ctx* c, const FftRowArgs& a) {
  if (FIN) {
    k_fft_row<NC, PL, FIN><<<c->fft_blocks, c->fft_row_threads, c->fft_smem, c->stream>>>(a);
  } else {
    cudaError_t e = launch_pdl(k_fft_row<NC, PL, FIN>, dim3(c->fft_blocks), dim3(c->fft_row_threads),
                               c->fft_smem, c->stream, a);
    if (e != cudaSuccess) return cuda_fail(e, "fft row");
  }
  return fft_check(c, "fft row");
}

int launch_fft_row(rf_ctx* c, const int* done, bool final_pass, int commit) {
  if (!final_pass && c->fft_row_warps > 0) return launch_fft_row_warp(c, done);
  FftRowArgs a = fft_row_args(c, done);
  if (final_pass) {
    a.eps_out = c->d_eps;
    a.sig_out = c->d_sig;
    a.alpha_out = c->d_alpha;
    a.sbar_part = c->d_sbar_part;
    a.viol_part = c->d_viol_part;
    a.commit = commit;
  }
  const bool pl = c->has_plastic;
  if (c->nc == 3) {
    if (final_pass)
      return pl ? fft_row_launch<3, true, true>(c, a) : fft_row_launch<3, false, true>(c, a);
    return pl ? fft_row_launch<3, true, false>(c, a) : fft_row_launch<3, false, false>(c, a);
  }
  if (final_pass)
    return pl ? fft_row_launch<6, true, true>(c, a) : fft_row_launch<6, false, true>(c, a);
  return pl ? fft_row_launch<6, true, false>(c, a) : fft_row_launch<6, false, false>(c, a);
}

// inverse transforms along z and y: ER -> T1
int fft_inverse_stages(rf_ctx* c, const int* done) {
  const int NCK = c->nc * c->Kx;
  if (c->dim == 3) {
    trace_stage(c, 0);
    if (int e = fft_cols(c, c->d_ER, 0, c->Kz, c->d_kzm, c->d_T2, 0, c->nz, nullptr,
                         c->Ky * NCK, c->nz, 1, +1, c->d_twz, done))
      return e;
    trace_stage(c, 1);
    return fft_cols(c, c->d_T2, (long long)c->Ky * NCK, c->Ky, c->d_kym, c->d_T1,
                    (long long)c->ny * NCK, c->ny, nullptr, NCK, c->ny, c->nz, +1, c->d_twy, done);
  }
  trace_stage(c, 1);
  return fft_cols(c, c->d_ER, 0, c->Ky, c->d_kym, c->d_T1, 0, c->ny, nullptr, NCK, c->ny, 1, +1,
                  c->d_twy, done);
}

// forward transforms along y and z: T1p -> OUT (one split)
int fft_forward_stages(rf_ctx* c, const int* done) {
  const int NCK = c->nc * c->Kx;
  if (c->dim == 3) {
    trace_stage(c, 3);
    if (int e = fft_cols(c, c->d_T1p, (long long)c->ny * NCK, c->ny, nullptr, c->d_T2f,
                         (long long)c->Ky * NCK, c->Ky, c->d_kym, NCK, c->ny, c->nz, -1,
                         c->d_twy, done))
      return e;
    trace_stage(c, 4);
    return fft_cols(c, c->d_T2f, 0, c->nz, nullptr, c->d_OUT, 0, c->Kz, c->d_kzm, c->Ky * NCK,
                    c->nz, 1, -1, c->d_twz, done);
  }
  trace_stage(c, 3);
  return fft_cols(c, c->d_T1p, 0, c->ny, nullptr, c->d_OUT, 0, c->Ky, c->d_kym, NCK, c->ny, 1,
                  -1, c->d_twy, done);
}

int launch_fft_colphase(rf_ctx* c, const int* done) {
  ColPhaseArgs a{};
  a.T1p = c->d_T1p;
  a.T1 = c->d_T1;
  a.ER = c->d_ER;
  a.jptr = c->d_jptr;
  a.jlist = c->d_jlist;
  a.hidx = c->d_hidx;
  a.hn = c->d_hn;
  a.kym = c->d_kym;
  a.table = c->d_twy;
  a.Kx = c->Kx;
  a.L = c->ny;
  a.M = c->fft_M;
  a.dC = make_fastdiv((unsigned)(c->nc * c->fft_M));
  a.inv2mu0 = (float)(0.5 / c->mu0);
  a.cgam = (float)((c->lam0 + c->mu0) / (c->mu0 * (c->lam0 + 2.0 * c->mu0)));
  a.st = c->d_status;
  a.counter = c->d_counter;
  a.part = c->d_part;
  a.done = done;
  a.cond = c->while_cond;
  a.use_cond = c->capturing_while ? 1 : 0;
  trace_stage(c, 6);
  const dim3 grid((unsigned)((c->Kx + c->fft_M - 1) / c->fft_M));
  cudaError_t e = launch_pdl(k_fft_colphase<3>, grid, dim3(c->fft_M_threads),
                             colphase_smem(c->ny, c->nc, c->fft_M), c->stream, a, (double)c->N);
  if (e != cudaSuccess) return cuda_fail(e, "fft column phase");
  const int r = fft_check(c, "fft column phase");
  trace_end(c);
  return r;
}

int launch_fft_green_inv(rf_ctx* c, const int* done) {
  GreenInvArgs a{};
  a.OUT = c->d_OUT;
  a.ER = c->d_ER;
  a.T1 = c->d_T1;
  a.jptr = c->d_jptr;
  a.jent = c->d_jent;
  a.jn = c->d_jn;
  a.kym = c->d_kym;
  a.table = c->d_twy;
  a.Kx = c->Kx;
  a.L = c->ny;
  a.ncols = c->nc * c->Kx;
  a.C = std::max(1, std::min(c->fft_C, a.ncols));
  a.dC = make_fastdiv((unsigned)a.C);
  a.dKx = make_fastdiv((unsigned)std::max(1, c->Kx));
  a.inv2mu0 = (float)(0.5 / c->mu0);
  a.cgam = (float)((c->lam0 + c->mu0) / (c->mu0 * (c->lam0 + 2.0 * c->mu0)));
  a.st = c->d_status;
  a.counter = c->d_counter;
  a.part = c->d_part;
  a.done = done;
  a.cond = c->while_cond;
  a.use_cond = c->capturing_while ? 1 : 0;
  trace_stage(c, 5);
  const dim3 grid((unsigned)((a.ncols + a.C - 1) / a.C));
  cudaError_t e = launch_pdl(k_fft_green_inv<3>, grid, dim3(c->fft_col_threads),
                             cols_smem(c->ny, a.C), c->stream, a, (double)c->N);
  if (e != cudaSuccess) return cuda_fail(e, "fft green + inverse");
  const int r = fft_check(c, "fft green + inverse");
  trace_end(c);
  return r;
}

static int tck(cudaError_t e, const char* what) { return e == cudaSuccess ? RF_OK : cuda_fail(e, what); }

// Autotuner for the FFT tiles: each candidate runs one untimed launch and then three timed groups
// of three launches of the stage it governs (CUDA events on the context's stream) on the
// context's own buffers; the candidate with the fastest group stays. Candidates that exceed
// shared memory are skipped.
int fft_autotune(rf_ctx* c) {
  // fused column phase: compared with the three separate kernels (fft_fuse = 0), or only its
  // block shape chosen (fft_fuse = 1 without fft_fuse_kx)
  const bool fuse_auto = c->dim == 2 && c->opt.fft_fuse == 0 && c->d_jptr &&
                         colphase_smem(c->ny, c->nc, 1) <= kFftSmemMax;
  const bool fuse_shape = c->fft_colmode == kColFused && c->opt.fft_fuse_kx == 0;
  // the warp-FFT column phase: compared with the other modes (fft_fuse 0) or only its kx columns
  // per block chosen (fft_fuse 4 without fft_fuse_kx)
  const bool colw_auto = fuse_auto && col_warp_ok(c) && c->opt.fft_row_warps == 0 &&
                         c->opt.fft_rows <= 0 && c->opt.fft_row_blocks <= 0;
  const bool colw_shape = c->fft_colmode == kColWarp && c->opt.fft_fuse_kx == 0;
  const bool rows_pinned = c->opt.fft_rows > 0 || c->opt.fft_row_blocks > 0;
  // the warp-FFT row kernel: compared with the shared-memory row kernel's best tile (the
  // warp-FFT column phase fixes it to its row-group slab form)
  const bool warp_need = c->fft_colmode == kColWarp || c->fft_colmode == kColPersistW;
  const bool warp_auto = !rows_pinned && c->opt.fft_row_warps == 0 && row_warp_ok(c) && !warp_need;
  // the persistent solve: compared with the other modes (fft_fuse 0, unless the row kernel's
  // tiles are pinned) or only its geometry chosen (fft_fuse 3); needs the barrier words set up
  // with the pattern
  const bool persist_auto = c->dim == 2 && c->d_jptr && c->d_bar &&
                            ((c->opt.fft_fuse == 0 && !rows_pinned) || c->opt.fft_fuse == 3);
  if (rows_pinned && c->opt.fft_cols > 0 && !fuse_auto && !fuse_shape && !persist_auto &&
      !colw_shape)
    return RF_OK;
  rf_ctx::Tuned& tu = c->tuned;
  if (tu.valid && tu.Kx == c->Kx && tu.Ky == c->Ky && tu.Kz == c->Kz) {
    // same transform shapes as the last tuning on this context: same choice
    if (!rows_pinned) {
      if (tu.row_blocks_balanced) set_rows_balanced(c, tu.row_blocks_balanced);
      else set_rows(c, tu.R);
      c->fft_row_threads = tu.row_threads;
      if (warp_auto) c->fft_row_warps = tu.row_warps;
    }
    if (c->opt.fft_cols <= 0) {
      c->fft_C = tu.C;
      c->fft_col_threads = tu.col_threads;
    }
    if (fuse_auto || fuse_shape) {
      c->fft_M = tu.M;
      c->fft_M_threads = tu.M_threads;
      if (fuse_auto) {
        c->fft_colmode = tu.colmode == kColPersistent ? kColSeparate : tu.colmode;
        c->fft_colw_M = tu.colw_M;
      }
    }
    if (colw_shape) c->fft_colw_M = tu.colw_M;
    if (persist_auto && tu.persist_per_sm > 0 &&
        persist_geometry(c, tu.persist_threads, tu.persist_per_sm)) {
      if (c->opt.fft_fuse == 0 && tu.colmode == kColPersistent) c->fft_colmode = kColPersistent;
    }
    return RF_OK;
  }
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "tuner");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(cudaGetLastError(), "tuner");
  }
  int err = RF_OK;
  const int NCK = c->nc * c->Kx;
  err = tck(cudaMemsetAsync(c->d_T1, 0, sizeof(float2) * (size_t)c->rows * NCK, c->stream), "tuner");
  if (!err) err = tck(cudaMemsetAsync(c->d_ER, 0, sizeof(float2) * c->rect, c->stream), "tuner");
  if (!err)
    err = tck(cudaMemsetAsync(c->d_T1p, 0, sizeof(float2) * (size_t)c->rows * NCK, c->stream),
              "tuner");
  // the fastest of three timed groups of three launches (one untimed launch first): the
  // minimum is robust to a stray slow launch, so repeated tunings of one pattern agree
  auto time_it = [&](auto&& run, float* ms) -> int {
    if (int e = run()) return e;
    *ms = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, c->stream);
      for (int i = 0; i < 3; ++i)
        if (int e = run()) return e;
      cudaEventRecord(e1, c->stream);
      if (int e = tck(cudaEventSynchronize(e1), "tuner")) return e;
      float t = 0.f;
      if (int e = tck(cudaEventElapsedTime(&t, e0, e1), "tuner")) return e;
      *ms = std::min(*ms, t);
    }
    return RF_OK;
  };
  // one whole update (row pass and column phase) in the given column mode
  auto run_update = [&](int mode) -> int {
    if (mode == kColFused) {
      if (int e = launch_fft_row(c, nullptr, false, 0)) return e;
      return launch_fft_colphase(c, nullptr);
    }
    if (mode == kColWarp) {
      if (int e = launch_fft_row(c, nullptr, false, 0)) return e;
      return launch_fft_colphase_warp(c, nullptr);
    }
    if (mode == kColGreenInv) {
      if (int e = launch_fft_row(c, nullptr, false, 0)) return e;
      if (int e = fft_forward_stages(c, nullptr)) return e;
      return launch_fft_green_inv(c, nullptr);
    }
    if (int e = fft_inverse_stages(c, nullptr)) return e;
    if (int e = launch_fft_row(c, nullptr, false, 0)) return e;
    if (int e = fft_forward_stages(c, nullptr)) return e;
    return launch_gamma_finalize(c, 1, nullptr);
  };
  if (!err && !rows_pinned) {
    // uniform tiles of R rows, and balanced partitions over k blocks per SM
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
    struct Cand {
      int R, nb;   // nb > 0: balanced over nb blocks
    };
    std::vector<Cand> cands;
    for (int R : {1, 2, 4, 8, 16})
      if (R <= c->rows && row_smem(c->nx, c->nc, c->Kx, R) <= kFftSmemMax) cands.push_back({R, 0});
    for (int k = 1; sms > 0 && k <= 8; ++k) {
      const int nb = k * sms;
      if (nb >= c->rows || c->rows % nb == 0) continue;   // uniform tiles cover these
      const int Rmax = c->rows / nb + 1;
      if (row_smem(c->nx, c->nc, c->Kx, Rmax) <= kFftSmemMax) cands.push_back({Rmax, nb});
    }
    c->fft_row_warps = 0;   // the shared-memory row kernel's tiles first (it runs the final pass)
    float best = 1e30f;
    Cand bestC{c->fft_R, 0};
    int bestT = c->fft_row_threads;
    for (const Cand& cd : cands) {
      for (int T : {128, 256, 512}) {
        if (cd.nb) set_rows_balanced(c, cd.nb);
        else set_rows(c, cd.R);
        c->fft_row_threads = T;
        float ms = 0.f;
        err = time_it([&] { return launch_fft_row(c, nullptr, false, 0); }, &ms);
        if (err) break;
        if (ms < best) {
          best = ms;
          bestC = cd;
          bestT = T;
        }
      }
      if (err) break;
    }
    if (bestC.nb) set_rows_balanced(c, bestC.nb);
    else set_rows(c, bestC.R);
    c->fft_row_threads = bestT;
    c->fft_row_warps = warp_need ? 8
                       : (c->opt.fft_row_warps > 0 && row_warp_ok(c)) ? c->opt.fft_row_warps : 0;
    if (!err && warp_auto) {
      int bestW = 0;
      for (int W : {2, 4}) {
        c->fft_row_warps = W;
        float ms = 0.f;
        err = time_it([&] { return launch_fft_row(c, nullptr, false, 0); }, &ms);
        if (err) break;
        if (ms < best) {
          best = ms;
          bestW = W;
        }
      }
      c->fft_row_warps = bestW;
    }
  }
  if (!err && c->opt.fft_cols <= 0) {
    const int Lc = std::max(c->ny, c->dim == 3 ? c->nz : 1);
    float best = 1e30f;
    int bestC = c->fft_C, bestT = c->fft_col_threads;
    for (int C : {1, 2, 4, 8, 16, 32}) {
      if (cols_smem(Lc, C) > kFftSmemMax) continue;
      for (int T : {64, 128, 256}) {
        c->fft_C = C;
        c->fft_col_threads = T;
        float ms = 0.f;
        err = time_it([&] {
          if (int e = fft_inverse_stages(c, nullptr)) return e;
          return fft_forward_stages(c, nullptr);
        }, &ms);
        if (err) break;
        if (ms < best) {
          best = ms;
          bestC = C;
          bestT = T;
        }
      }
      if (err) break;
    }
    c->fft_C = bestC;
    c->fft_col_threads = bestT;
  }
  if (!err && (fuse_auto || fuse_shape)) {
    const std::vector<int> Ms = c->opt.fft_fuse_kx > 0 ? std::vector<int>{c->opt.fft_fuse_kx}
                                                       : std::vector<int>{1, 2, 4};
    float best = 1e30f;
    int bestM = c->fft_M, bestT = c->fft_M_threads;
    for (int M : Ms) {
      if (M > std::max(1, c->Kx) || colphase_smem(c->ny, c->nc, M) > kFftSmemMax) continue;
      for (int T : {128, 256}) {
        c->fft_M = M;
        c->fft_M_threads = T;
        float ms = 0.f;
        err = time_it([&] { return launch_fft_colphase(c, nullptr); }, &ms);
        if (err) break;
        if (ms < best) {
          best = ms;
          bestM = M;
          bestT = T;
        }
      }
      if (err) break;
    }
    c->fft_M = bestM;
    c->fft_M_threads = bestT;
    if (!err && fuse_auto) {
      // the three modes of the column phase, each timed over one update's column work
      float sep = 1e30f, gi = 1e30f;
      err = time_it([&] {
        if (int e = fft_forward_stages(c, nullptr)) return e;
        if (int e = launch_gamma_finalize(c, 1, nullptr)) return e;
        return fft_inverse_stages(c, nullptr);
      }, &sep);
      if (!err)
        err = time_it([&] {
          if (int e = fft_forward_stages(c, nullptr)) return e;
          return launch_fft_green_inv(c, nullptr);
        }, &gi);
      c->fft_colmode = kColSeparate;
      if (!err && gi < sep && gi <= best) c->fft_colmode = kColGreenInv;
      else if (!err && best < sep) c->fft_colmode = kColFused;
      if (!err && colw_auto) {
        // whole updates: the mode chosen so far against the warp-FFT column phase with the
        // warp-FFT row kernel on kx slabs
        const int keep_mode = c->fft_colmode, keep_w = c->fft_row_warps;
        float t_keep = 1e30f;
        err = time_it([&] { return run_update(keep_mode); }, &t_keep);
        c->fft_colmode = kColWarp;
        c->fft_row_warps = 8;
        float bw = 1e30f;
        int bestMw = 1;
        for (int Mw : {1, 2}) {
          if (err) break;
          c->fft_colw_M = Mw;
          float ms = 0.f;
          err = time_it([&] { return run_update(kColWarp); }, &ms);
          if (!err && ms < bw) {
            bw = ms;
            bestMw = Mw;
          }
        }
        c->fft_colw_M = bestMw;
        if (err || !(bw < t_keep)) {
          c->fft_colmode = keep_mode;
          c->fft_row_warps = keep_w;
        }
      }
    }
  }
  if (!err && colw_shape) {
    float bw = 1e30f;
    int bestMw = 1;
    for (int Mw : {1, 2}) {
      c->fft_colw_M = Mw;
      float ms = 0.f;
      err = time_it([&] { return launch_fft_colphase_warp(c, nullptr); }, &ms);
      if (err) break;
      if (ms < bw) {
        bw = ms;
        bestMw = Mw;
      }
    }
    c->fft_colw_M = bestMw;
  }
  if (!err && persist_auto) {
    // per-update time of the best separate-kernel mode against the persistent solve (one launch
    // of 8 updates with tol = 0; its start adds one inverse pass, which counts against it)
    float t_np = 1e30f;
    const int mode_np = c->fft_colmode == kColPersistent ? kColSeparate : c->fft_colmode;
    if (c->opt.fft_fuse == 0) {
      const int keep = c->fft_colmode;
      c->fft_colmode = mode_np;
      err = time_it([&] { return run_update(mode_np); }, &t_np);
      t_np /= 3.f;
      c->fft_colmode = keep;
    }
    constexpr int kUpd = 8;
    Status& hs = *c->h_status;
    std::memset(&hs, 0, sizeof(Status));
    hs.max_iter = kUpd;
    hs.tol = 0.0;
    hs.enorm = 1.0;
    hs.inv_n2 = 1.0 / ((double)c->N * (double)c->N);
    hs.rmin = HUGE_VAL;
    hs.lam0 = c->lam0;
    hs.mu0 = c->mu0;
    float best = 1e30f;
    int bestT = 0, bestK = 0;
    const int cand[4][2] = {{512, 2}, {256, 2}, {512, 1}, {256, 1}};
    for (const auto& cd : cand) {
      if (err || !persist_geometry(c, cd[0], cd[1])) continue;
      float ms = 1e30f;
      const int e = time_it([&] {
        if (int e2 = tck(cudaMemcpyAsync(c->d_status, c->h_status, sizeof(Status),
                                         cudaMemcpyHostToDevice, c->stream), "tuner"))
          return e2;
        return launch_persist_solve(c, nullptr, 0);
      }, &ms);
      if (e) {   // a launch the device refuses (co-residency) is not a candidate
        cudaGetLastError();
        set_error("");
        continue;
      }
      ms /= 3.f * kUpd;
      if (ms < best) {
        best = ms;
        bestT = cd[0];
        bestK = cd[1];
      }
    }
    if (bestT > 0) {
      persist_geometry(c, bestT, bestK);
      if (c->opt.fft_fuse == 3 || best < t_np) c->fft_colmode = kColPersistent;
      else c->fft_colmode = mode_np;
    } else if (c->opt.fft_fuse == 3) {
      set_error("persistent solve: no cooperative launch of this pattern succeeded");
      err = RF_ERR_CUDA;
    } else {
      c->fft_colmode = mode_np;
    }
  }
  if (!err && colw_auto && persist_warp_ok(c)) {
    // the persistent solve on the warp-FFT passes against the mode chosen so far, per update
    auto time_persist = [&](int mode, float* per_update) -> int {
      constexpr int kUpd = 8;
      Status& hs = *c->h_status;
      std::memset(&hs, 0, sizeof(Status));
      hs.max_iter = kUpd;
      hs.tol = 0.0;
      hs.enorm = 1.0;
      hs.inv_n2 = 1.0 / ((double)c->N * (double)c->N);
      hs.rmin = HUGE_VAL;
      hs.lam0 = c->lam0;
      hs.mu0 = c->mu0;
      float ms = 1e30f;
      const int e = time_it([&] {
        if (int e2 = tck(cudaMemcpyAsync(c->d_status, c->h_status, sizeof(Status),
                                         cudaMemcpyHostToDevice, c->stream), "tuner"))
          return e2;
        return mode == kColPersistW ? launch_persist_warp(c, nullptr, 0)
                                    : launch_persist_solve(c, nullptr, 0);
      }, &ms);
      *per_update = ms / (3.f * kUpd);
      return e;
    };
    const int keep_mode = c->fft_colmode, keep_w = c->fft_row_warps, keep_M = c->fft_colw_M;
    float t_cur = 1e30f;
    if (keep_mode == kColPersistent) {
      err = time_persist(kColPersistent, &t_cur);
    } else {
      err = time_it([&] { return run_update(keep_mode); }, &t_cur);
      t_cur /= 3.f;
    }
    float t_pw = 1e30f;
    if (!err) {
      c->fft_colmode = kColPersistW;
      c->fft_row_warps = 8;
      c->fft_colw_M = 2;
      const int e = time_persist(kColPersistW, &t_pw);
      if (e) {   // a launch the device refuses (co-residency) is not a candidate
        cudaGetLastError();
        set_error("");
        t_pw = 1e30f;
      }
    }
    if (err || !(t_pw < t_cur)) {
      c->fft_colmode = keep_mode;
      c->fft_row_warps = keep_w;
      c->fft_colw_M = keep_M;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!err) {
    tu.valid = true;
    tu.Kx = c->Kx;
    tu.Ky = c->Ky;
    tu.Kz = c->Kz;
    tu.R = c->fft_R;
    tu.row_blocks_balanced = c->fft_rextra > 0 ? c->fft_blocks : 0;
    tu.row_threads = c->fft_row_threads;
    tu.C = c->fft_C;
    tu.col_threads = c->fft_col_threads;
    tu.M = c->fft_M;
    tu.M_threads = c->fft_M_threads;
    tu.colmode = c->fft_colmode;
    tu.persist_per_sm = c->persist_per_sm;
    tu.persist_threads = c->persist_threads;
    tu.row_warps = c->fft_row_warps;
    tu.colw_M = c->fft_colw_M;
  }
  return err;
}

}  // namespace rfk
