// Batched solver: many independent 2D RVEs of uneven size (FE-FFT Gauss points), each with its
// own phase map, adapted pattern and macroscopic strain, solved together.
//
// Two forms, the faster chosen by timing at creation (options.batch_resident). RVE-resident
// (kb_resident, square RVEs with sides 64, 96, 128, 192, 256): one launch per solve, a block
// holds one RVE for all of its updates and its final pass, RVEs taken largest first from a
// queue. Sweeps: one update of every unconverged RVE is five persistent kernels, each walking
// a work list of (RVE, tile) items in a fixed order (largest RVEs first) with a stride of the
// grid size:
//   inverse y transform tiles, row tiles (x transforms + law), forward y transform tiles,
//   Green-operator chunks (with squared-increment partials), per-RVE convergence decisions.
// Items of converged RVEs return at once. A solve is one CUDA graph launch: a conditional while
// node whose body is a few updates; the decision kernel's last block clears the loop condition
// once every RVE is done (converged, capped, non-finite or diverged). Elastic phases, plane
// strain (NC = 3), FP32 transforms: FFT items along x and y for sides 2^b and 3 2^b with
// options.transform = RF_TRANSFORM_FFT, pruned-DFT items otherwise; convergence measure and
// homogenised stress in FP64. Rows per row item (per size class) and the persistent grid size
// are chosen per batch by a timing autotuner.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "../../include/rf_mlp.h"
#include "rf_fftcore.cuh"
#include "rf_internal.cuh"
#include "rf_law.cuh"

namespace rfk {

namespace {

constexpr int NC = 3;

struct BDesc {
  int nx, ny, Kx, Ky;
  int Kh, rows, R, row_items;
  int mt_inv, nt, mt_fwd, chunks;
  long long N;
  long long off_phase;   // uint8
  long long off_er;      // float2, Ky * NC * Kx
  long long off_t1;      // float2, ny * NC * Kx (T1 and T1p use the same offsets)
  long long off_h;       // hidx / hn
  long long off_kx;      // int (kx values), float (fac)
  long long off_ky;      // int (ky mod ny)
  long long off_part;    // double, chunks
  long long off_spart;   // double, row_items * 6
  int tab_x, tab_y;      // offsets into the twiddle buffer
  FastDiv dKx, dnx;      // division by Kx and Nx
  int fft;               // row items use FFTs along x (Nx = 2^b or 3 2^b), else the pruned DFT
  int warp;              // row items use warp-resident FFTs (Nx in {64, 96, 128, 192, 256})
  int pad_w;
  int fft_y, cy;         // y transforms by FFT over groups of cy line columns (Ny = 2^b, 3 2^b)
  long long zero_base;   // ER offset (within the RVE) of the zero frequency
  float lam0, mu0, inv2mu0, cgam;
};

struct BStat {
  int done, iters, nonfinite, max_iter;
  int diverged, pad;
  double tol, enorm, inv_n2, last_r, rmin;
  double ebar[6];
  double sbar[6];
};

struct BArgs {
  const BDesc* d;
  BStat* st;
  const int2* items;
  int n_items;
  const uint8_t* phase;
  float2* ER;
  float2* T1;
  float2* T1p;
  float2* OUT;
  const HIdx* hidx;
  const float4* hn;
  const int* kx;
  const float* fac;
  const int* kym;
  const float2* tab;
  double* part;
  double* spart;
  int* n_done;
  LawParams law;
  int final_pass;
  // while-loop graph: the decision kernel's last block clears the loop condition when every
  // RVE is done
  unsigned* counter;
  cudaGraphConditionalHandle cond;
  int use_cond;
};

__device__ __forceinline__ bool rve_done(const BArgs& a, int r) { return a.st[r].done != 0; }

// out[m][n] = sum_k w(m, k) in[k][n] for one 32 x 64 tile (same tile body as the unbatched
// transform kernel): inverse (sign +1): m = y, k over ky; forward (sign -1): m over ky, k = y
__device__ void dft_tile(const float2* in, float2* out, int M, int N, int K, const int* mvals,
                         const int* kvals, const float2* tab, int L, int sign, int m0, int n0,
                         float2 (*xs)[64], float2 (*ws)[33]) {
  constexpr int MT = 8;
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6, tid = threadIdx.x;
  float accr[MT], acci[MT];
#pragma unroll
  for (int i = 0; i < MT; ++i) accr[i] = acci[i] = 0.f;
  for (int kb = 0; kb < K; kb += 32) {
    for (int i = tid; i < 32 * 64; i += 256) {
      const int kk = i >> 6, nn = i & 63, k = kb + kk, n = n0 + nn;
      xs[kk][nn] = (k < K && n < N) ? in[(long long)k * N + n] : make_float2(0.f, 0.f);
    }
    for (int i = tid; i < 32 * 32; i += 256) {
      const int mm = i >> 5, kk = i & 31, m = m0 + mm, k = kb + kk;
      float2 w = make_float2(0.f, 0.f);
      if (m < M && k < K) {
        const int mv = mvals ? mvals[m] : m;
        const int kv = kvals ? kvals[k] : k;
        w = tab[(int)(((long long)mv * kv) % L)];
        if (sign < 0) w.y = -w.y;
      }
      ws[mm][kk] = w;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      const float2 x = xs[kk][tx];
#pragma unroll
      for (int i = 0; i < MT; ++i) {
        const float2 w = ws[ty * MT + i][kk];
        accr[i] = fmaf(w.x, x.x, fmaf(-w.y, x.y, accr[i]));
        acci[i] = fmaf(w.x, x.y, fmaf(w.y, x.x, acci[i]));
      }
    }
    __syncthreads();
  }
  const int n = n0 + tx;
  if (n < N) {
#pragma unroll
    for (int i = 0; i < MT; ++i) {
      const int m = m0 + ty * MT + i;
      if (m < M) out[(long long)m * N + n] = make_float2(accr[i], acci[i]);
    }
  }
}

// Column item by FFTs along y: cy consecutive line columns (of the NC Kx per row) of one RVE.
// Inverse: the pattern's ky rows of ER scattered into full columns, FFT, all Ny rows of T1.
// Forward: all Ny rows of T1p, FFT, the pattern's ky rows into OUT. Loads in batches of 8.
__device__ void col_item_fft(const BArgs& a, int g, const BDesc& d, unsigned char* smem,
                             int sign) {
  using namespace fftc;
  const int L = d.ny, NCK = NC * d.Kx;
  const int c0 = g * d.cy, cc_n = min(d.cy, NCK - c0);
  const int span = span_of(cc_n * L);
  float2* tw = reinterpret_cast<float2*>(smem);
  float2* b0 = tw + L;
  float2* b1 = b0 + span;
  copy_twiddles(a.tab + d.tab_y, L, tw);
  const int* kym = a.kym + d.off_ky;
  if (sign > 0)
    for (int i = threadIdx.x; i < span; i += blockDim.x) b0[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const float2* src = sign > 0 ? a.ER + d.off_er : a.T1p + d.off_t1;
  const int rows_in = sign > 0 ? d.Ky : L;
  const int tot = rows_in * cc_n;
  for (int i0 = threadIdx.x; i0 < tot; i0 += 8 * blockDim.x) {
    float2 v[8];
    int dst[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * blockDim.x;
      dst[u] = -1;
      v[u] = make_float2(0.f, 0.f);
      if (i < tot) {
        const int r = i / cc_n, cc = i - r * cc_n;
        v[u] = src[(long long)r * NCK + c0 + cc];
        dst[u] = cc * L + (sign > 0 ? kym[r] : r);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (dst[u] >= 0) b0[sw(dst[u])] = v[u];
  }
  __syncthreads();
  const float2* z = fft_block(b0, b1, tw, L, cc_n, sign);
  float2* dstg = sign > 0 ? a.T1 + d.off_t1 : a.OUT + d.off_er;
  const int rows_out = sign > 0 ? L : d.Ky;
  for (int i = threadIdx.x; i < rows_out * cc_n; i += blockDim.x) {
    const int r = i / cc_n, cc = i - r * cc_n;
    dstg[(long long)r * NCK + c0 + cc] = z[sw(cc * L + (sign > 0 ? r : kym[r]))];
  }
  __syncthreads();   // the next item reuses the buffers
}

constexpr int kColFft = 1 << 30;   // item flag: FFT column group (else a DFT tile index)

__global__ __launch_bounds__(256) void kb_inv_y(BArgs a) {
  __shared__ float2 xs[32][64];
  __shared__ float2 ws[32][33];
  extern __shared__ __align__(16) unsigned char csm[];
  for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const int2 w = a.items[it];
    if (!a.final_pass && rve_done(a, w.x)) continue;   // the final pass covers every RVE
    const BDesc d = a.d[w.x];
    if (w.y & kColFft) {
      col_item_fft(a, w.y & ~kColFft, d, csm, +1);
      continue;
    }
    const int mt = w.y / d.nt, nt = w.y % d.nt;
    dft_tile(a.ER + d.off_er, a.T1 + d.off_t1, d.ny, NC * d.Kx, d.Ky, nullptr, a.kym + d.off_ky,
             a.tab + d.tab_y, d.ny, +1, mt * 32, nt * 64, xs, ws);
  }
}

__global__ __launch_bounds__(256) void kb_fwd_y(BArgs a) {
  __shared__ float2 xs[32][64];
  __shared__ float2 ws[32][33];
  extern __shared__ __align__(16) unsigned char csm[];
  for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const int2 w = a.items[it];
    if (rve_done(a, w.x)) continue;
    const BDesc d = a.d[w.x];
    if (w.y & kColFft) {
      col_item_fft(a, w.y & ~kColFft, d, csm, -1);
      continue;
    }
    const int mt = w.y / d.nt, nt = w.y % d.nt;
    dft_tile(a.T1p + d.off_t1, a.OUT + d.off_er, d.Ky, NC * d.Kx, d.ny, a.kym + d.off_ky,
             nullptr, a.tab + d.tab_y, d.ny, -1, mt * 32, nt * 64, xs, ws);
  }
}

// row tiles: R rows of one RVE; inverse x transform, law, forward x transform (FINAL: stress
// partials instead of the forward transform)
// Row item by FFTs along x (the transform mode of the single-RVE solver, for Nx = 2^b or 3 2^b):
// two real lines per complex sequence, Hermitian completion of the lines' kx >= 0 coefficients,
// inverse FFT, elastic law and polarization per voxel, forward FFT, separation of the two lines'
// spectra at the pattern's kx columns. Final pass: homogenised-stress partials instead.
__device__ void row_item_fft(const BArgs& a, int2 w, const BDesc& d, unsigned char* smem,
                             double* red) {
  using namespace fftc;
  const int L = d.nx, Kx = d.Kx, R = d.R;
  const int row0 = w.y * R;
  const int nr = min(R, d.rows - row0);
  const int S = nr * NC, P = (S + 1) / 2;
  const int span = span_of(P * L);
  float2* tw = reinterpret_cast<float2*>(smem);
  float2* b0 = tw + L;
  float2* b1 = b0 + span;
  int* kxs = reinterpret_cast<int*>(b1 + span);
  const int tid = threadIdx.x;
  copy_twiddles(a.tab + d.tab_x, L, tw);
  for (int i = tid; i < Kx; i += blockDim.x) kxs[i] = a.kx[d.off_kx + i];
  for (int i = tid; i < span; i += blockDim.x) b0[i] = make_float2(0.f, 0.f);
  __syncthreads();
  // z_p = line 2p + i line 2p+1: z[k] = ta + i tb, z[L - k] = conj(ta) + i conj(tb); the
  // coefficients are loaded four (p, j) at a time before they are scattered
  const float2* Tg = a.T1 + d.off_t1 + (long long)row0 * NC * Kx;
  for (int u0 = tid; u0 < P * Kx; u0 += 4 * blockDim.x) {
    float2 ta[4], tb[4];
    int jj[4], pp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int u = u0 + q * blockDim.x;
      pp[q] = -1;
      if (u < P * Kx) {
        const int p = fdiv(u, d.dKx), j = u - p * Kx;
        const int s0 = 2 * p, s1 = s0 + 1;
        ta[q] = Tg[(long long)s0 * Kx + j];   // line s = r NC + c is row r, component c
        tb[q] = s1 < S ? Tg[(long long)s1 * Kx + j] : make_float2(0.f, 0.f);
        pp[q] = p;
        jj[q] = j;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (pp[q] < 0) continue;
      const int k = kxs[jj[q]];
      const bool self = (k == 0) || (2 * k == L);
      if (self) {
        ta[q].y = 0.f;
        tb[q].y = 0.f;
      }
      b0[sw(pp[q] * L + k)] = make_float2(ta[q].x - tb[q].y, ta[q].y + tb[q].x);
      if (!self) b0[sw(pp[q] * L + L - k)] = make_float2(ta[q].x + tb[q].y, tb[q].x - ta[q].y);
    }
  }
  __syncthreads();
  float2* zb = fft_block(b0, b1, tw, L, P, +1);
  float2* other = (zb == b0) ? b1 : b0;
  const float invN = 1.f / (float)d.N;
  double sb[6] = {0, 0, 0, 0, 0, 0};
  // phase ids four voxels at a time, loaded before the law runs on them
  for (int v0 = tid; v0 < nr * L; v0 += 4 * blockDim.x) {
    uint8_t pid[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int v = v0 + q * blockDim.x;
      pid[q] = 0;
      if (v < nr * L) {
        const int r = fdiv(v, d.dnx), x = v - r * L;
        pid[q] = a.phase[d.off_phase + (long long)(row0 + r) * L + x];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int v = v0 + q * blockDim.x;
      if (v >= nr * L) continue;
      const int r = fdiv(v, d.dnx), x = v - r * L;
      float e[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int sl = r * NC + c;
        const float2 z = zb[sw((sl >> 1) * L + x)];
        e[c] = ((sl & 1) ? z.y : z.x) * invN;
      }
      float e6[6];
      comp_to6<NC>(e, e6);
      const DevPhase ph = a.law.ph[pid[q]];
      float ep[6] = {0, 0, 0, 0, 0, 0};
      LawOut o;
      stress6<false>(e6, ph, ep, 0.f, o);
      if (a.final_pass) {
#pragma unroll
        for (int i = 0; i < 6; ++i) sb[i] += (double)o.s[i];
      } else {
        const float tr = e6[0] + e6[1] + e6[2];
        float tau6[6];
#pragma unroll
        for (int i = 0; i < 3; ++i) tau6[i] = o.s[i] - (d.lam0 * tr + 2.f * d.mu0 * e6[i]);
#pragma unroll
        for (int i = 3; i < 6; ++i) tau6[i] = o.s[i] - 2.f * d.mu0 * e6[i];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int sl = r * NC + c;
          float* dst = reinterpret_cast<float*>(other + sw((sl >> 1) * L + x));
          dst[sl & 1] = tau6[comp6<NC>(c)];
        }
      }
    }
  }
  if (a.final_pass) {
    for (int i = 0; i < 6; ++i) {
      const double t = block_sum_d(sb[i], red);
      if (tid == 0) a.spart[d.off_spart + (long long)w.y * 6 + i] = t;
    }
    return;
  }
  if (S & 1)
    for (int x = tid; x < L; x += blockDim.x) other[sw((P - 1) * L + x)].y = 0.f;
  __syncthreads();
  float2* zf = fft_block(other, zb, tw, L, P, -1);
  float2* To = a.T1p + d.off_t1 + (long long)row0 * NC * Kx;
  for (int u = tid; u < S * Kx; u += blockDim.x) {
    const int sl = fdiv(u, d.dKx), j = u - sl * Kx;
    const int k = kxs[j];
    const int base = (sl >> 1) * L;
    const float2 zk = zf[sw(base + k)], zm = zf[sw(base + (k == 0 ? 0 : L - k))];
    float2 out;
    if ((sl & 1) == 0) out = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    else out = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    To[(long long)sl * Kx + j] = out;
  }
}

// ---- row items with warp-resident FFTs (rows of L = 32 P voxels, P in {2, 3, 4, 6, 8})
//
// A warp transforms S = 32 / P packed sequences (two real lines each) of length L at once: lane
// n2 holds entries 32 n1 + n2 of sequence s in v[s P + n1]; a P-point DFT per sequence in
// registers, the twiddle exp(sign 2 pi i k1 n2 / L), a transpose through a padded warp region
// (row s P + k1 to lane s P + k1), and a 32-point DFT per lane: lane s P + k1 then holds entries
// k1 + P k2 of sequence s's transform in v[k2]. The item's rows are staged in the warps'
// regions between the transforms, and the law runs on every voxel of the item.

constexpr int kWRegion = 32 * 33;   // a warp's region (entries): transposes and S sequences

// P-point DFT of v[0 .. P) in natural order in and out, kernel exp(sign 2 pi i k n / P)
template <int P>
__device__ __forceinline__ void dft_small(float2* v, int sign) {
  const float sg = sign < 0 ? -1.f : 1.f;
  if constexpr (P == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = make_float2(a.x + b.x, a.y + b.y);
    v[1] = make_float2(a.x - b.x, a.y - b.y);
  } else if constexpr (P == 3) {
    // X1,2 = a - (b + c) / 2 +- i sign sqrt(3)/2 (b - c)
    const float2 a = v[0], b = v[1], c = v[2];
    const float2 t1 = make_float2(b.x + c.x, b.y + c.y);
    const float2 t2 = make_float2(a.x - 0.5f * t1.x, a.y - 0.5f * t1.y);
    const float h = 0.86602540378443865f * sg;
    const float2 t3 = make_float2(h * (b.x - c.x), h * (b.y - c.y));
    v[0] = make_float2(a.x + t1.x, a.y + t1.y);
    v[1] = make_float2(t2.x - t3.y, t2.y + t3.x);
    v[2] = make_float2(t2.x + t3.y, t2.y - t3.x);
  } else if constexpr (P == 4) {
    fftc::dft4(v[0], v[1], v[2], v[3], sign);
  } else if constexpr (P == 6) {
    // n = 3 n1 + n2, k = k1 + 2 k2: 2-point DFTs over n1, twiddles exp(sign 2 pi i n2 k1 / 6),
    // 3-point DFTs over n2
    float2 y0[3], y1[3];
#pragma unroll
    for (int n2 = 0; n2 < 3; ++n2) {
      const float2 a = v[n2], b = v[3 + n2];
      y0[n2] = make_float2(a.x + b.x, a.y + b.y);
      y1[n2] = make_float2(a.x - b.x, a.y - b.y);
    }
    const float h = 0.86602540378443865f * sg;
    y1[1] = fftc::cmul(y1[1], make_float2(0.5f, h));    // exp(sign i pi / 3)
    y1[2] = fftc::cmul(y1[2], make_float2(-0.5f, h));   // exp(sign 2 i pi / 3)
    dft_small<3>(y0, sign);
    dft_small<3>(y1, sign);
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2) {
      v[2 * k2] = y0[k2];
      v[2 * k2 + 1] = y1[k2];
    }
  } else {
    static_assert(P == 8, "P");
    float2 e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    fftc::dft4(e[0], e[1], e[2], e[3], sign);
    fftc::dft4(o[0], o[1], o[2], o[3], sign);
    const float r = 0.70710678118654752f;
    const float2 w[4] = {make_float2(1.f, 0.f), make_float2(r, sg * r), make_float2(0.f, sg),
                         make_float2(-r, sg * r)};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float2 t = k == 0 ? o[0] : fftc::cmul(o[k], w[k]);
      v[k] = make_float2(e[k].x + t.x, e[k].y + t.y);
      v[k + 4] = make_float2(e[k].x - t.x, e[k].y - t.y);
    }
  }
}

// 32-point DFT in registers (natural order in and out): even and odd samples through two
// 16-point DFTs and a radix-2 step
__device__ __forceinline__ void dft32_regs(float2* v, int sign) {
  float2 e[16], o[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    e[m] = v[2 * m];
    o[m] = v[2 * m + 1];
  }
  fftc::dft16(e, sign);
  fftc::dft16(o, sign);
  const float c[9] = {1.f,
                      0.98078528040323044912f,
                      0.92387953251128675613f,
                      0.83146961230254523708f,
                      0.70710678118654752440f,
                      0.55557023301960222474f,
                      0.38268343236508977173f,
                      0.19509032201612826785f,
                      0.f};
  const float sg = sign < 0 ? -1.f : 1.f;
#pragma unroll
  for (int q = 0; q < 16; ++q) {
    const int i = 4 * (q & 3) + (q >> 2);   // where the 16-point kernel leaves its output q
    const float cs = q <= 8 ? c[q] : -c[16 - q];
    const float sn = q <= 8 ? c[8 - q] : c[q - 8];
    const float2 O = fftc::cmul(o[i], make_float2(cs, sg * sn));
    v[q] = make_float2(e[i].x + O.x, e[i].y + O.y);
    v[q + 16] = make_float2(e[i].x - O.x, e[i].y - O.y);
  }
}

// Forward transforms (exp(-2 pi i k n / L), L = 32 P) of the first SU of the S = 32 / P
// sequences a warp holds (layout above; the others are left as zeros); tab[t] = exp(+2 pi i t /
// L); T: the warp's region (32 rows of 33), free again when after_transpose() runs (before the
// 32-point DFTs).
template <int P, int SU = 32 / P, class F>
__device__ __forceinline__ void fwd_batch_cb(float2* v, float2* T, const float2* __restrict__ tab,
                                             int lane, F&& after_transpose) {
  static_assert(SU >= 1 && SU <= 32 / P, "sequences");
#pragma unroll
  for (int s = 0; s < SU; ++s) dft_small<P>(v + s * P, -1);
#pragma unroll
  for (int s = 0; s < SU; ++s)
#pragma unroll
    for (int k1 = 1; k1 < P; ++k1) {
      float2 w = __ldg(tab + k1 * lane);
      w.y = -w.y;
      v[s * P + k1] = fftc::cmul(v[s * P + k1], w);
    }
  __syncwarp();
#pragma unroll
  for (int r = 0; r < SU * P; ++r) T[r * 33 + lane] = v[r];
  __syncwarp();
#pragma unroll
  for (int n2 = 0; n2 < 32; ++n2) v[n2] = lane < SU * P ? T[lane * 33 + n2] : make_float2(0.f, 0.f);
  __syncwarp();
  after_transpose();
  dft32_regs(v, -1);
}

template <int P>
__device__ __forceinline__ void fwd_batch(float2* v, float2* T, const float2* __restrict__ tab,
                                          int lane) {
  fwd_batch_cb<P>(v, T, tab, lane, [] {});
}

// Row item with warp-resident FFTs (FINAL: homogenised-stress partials after the law). Sequence
// p = (line 2p) + i (line 2p + 1) of the item's 3 nr lines (line s = r NC + c) lives in warp
// p / S at p % S; between the transforms the region holds it in space at s (L + P) + x (the
// padded stride keeps the transform's scattered writes free of bank conflicts).
template <int P, bool FINAL>
__device__ void row_item_warp(const BArgs& a, int2 w, const BDesc& d, unsigned char* smem,
                              double* red) {
  constexpr int L = 32 * P, S = 32 / P, LS = L + P;   // sequence stride: conflict-free writes
  const int Kx = d.Kx, R = d.R;
  const int row0 = w.y * R;
  const int nr = min(R, d.rows - row0);
  const int nl = nr * NC, nseq = (nl + 1) / 2;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  int* kxs = reinterpret_cast<int*>(smem);
  float2* W0 = reinterpret_cast<float2*>(smem + (((size_t)Kx * sizeof(int) + 15) & ~(size_t)15));
  float2* Wr = W0 + (size_t)wp * kWRegion;   // this warp's region
  const float2* tab = a.tab + d.tab_x;
  for (int i = tid; i < Kx; i += blockDim.x) kxs[i] = a.kx[d.off_kx + i];
  for (int i = lane; i < kWRegion; i += 32) Wr[i] = make_float2(0.f, 0.f);
  __syncthreads();
  // spectra: z_p[k] = ta + i tb, z_p[L - k] = conj(ta) + i conj(tb)
  const float2* Tg = a.T1 + d.off_t1 + (long long)row0 * NC * Kx;
  for (int u0 = tid; u0 < nseq * Kx; u0 += 4 * blockDim.x) {
    float2 ta[4], tb[4];
    int jj[4], pp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int u = u0 + q * blockDim.x;
      pp[q] = -1;
      if (u < nseq * Kx) {
        const int p = fdiv(u, d.dKx), j = u - p * Kx;
        const int s0 = 2 * p, s1 = s0 + 1;
        ta[q] = Tg[(long long)s0 * Kx + j];
        tb[q] = s1 < nl ? Tg[(long long)s1 * Kx + j] : make_float2(0.f, 0.f);
        pp[q] = p;
        jj[q] = j;
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (pp[q] < 0) continue;
      const int k = kxs[jj[q]];
      const bool self = (k == 0) || (2 * k == L);
      if (self) {
        ta[q].y = 0.f;
        tb[q].y = 0.f;
      }
      float2* z = W0 + (size_t)(pp[q] / S) * kWRegion + (pp[q] % S) * LS;
      z[k] = make_float2(ta[q].x - tb[q].y, ta[q].y + tb[q].x);
      if (!self) z[L - k] = make_float2(ta[q].x + tb[q].y, tb[q].x - ta[q].y);
    }
  }
  __syncthreads();
  float2 v[32];
  const bool busy = wp * S < nseq;   // a warp with sequences
  if (busy) {
    // to space: the conjugate of the forward transform of the conjugate spectra
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) {
        const float2 z = Wr[s * LS + 32 * n1 + lane];
        v[s * P + n1] = make_float2(z.x, -z.y);
      }
#pragma unroll
    for (int r = S * P; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
    fwd_batch<P>(v, Wr, tab, lane);
    if (lane < S * P) {
      const int s = lane / P, k1 = lane - s * P;
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) Wr[s * LS + k1 + P * k2] = make_float2(v[k2].x, -v[k2].y);
    }
  }
  __syncthreads();
  // the law on every voxel of the item
  const float invN = 1.f / (float)d.N;
  double sb[6] = {0, 0, 0, 0, 0, 0};
  for (int vx = tid; vx < nr * L; vx += blockDim.x) {
    const int r = vx / L, x = vx - r * L;
    const uint8_t pid = a.phase[d.off_phase + (long long)(row0 + r) * L + x];
    float e[NC];
    float* at[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int sl = r * NC + c, p = sl >> 1;
      at[c] = reinterpret_cast<float*>(W0 + (size_t)(p / S) * kWRegion + (p % S) * LS + x) +
              (sl & 1);
      e[c] = *at[c] * invN;
    }
    float e6[6];
    comp_to6<NC>(e, e6);
    const DevPhase ph = a.law.ph[pid];
    float ep[6] = {0, 0, 0, 0, 0, 0};
    LawOut o;
    stress6<false>(e6, ph, ep, 0.f, o);
    if (FINAL) {
#pragma unroll
      for (int i = 0; i < 6; ++i) sb[i] += (double)o.s[i];
    } else {
      const float tr = e6[0] + e6[1] + e6[2];
      float tau6[6];
#pragma unroll
      for (int i = 0; i < 3; ++i) tau6[i] = o.s[i] - (d.lam0 * tr + 2.f * d.mu0 * e6[i]);
#pragma unroll
      for (int i = 3; i < 6; ++i) tau6[i] = o.s[i] - 2.f * d.mu0 * e6[i];
#pragma unroll
      for (int c = 0; c < NC; ++c) *at[c] = tau6[comp6<NC>(c)];
    }
  }
  if (FINAL) {
    for (int i = 0; i < 6; ++i) {
      const double t = block_sum_d(sb[i], red);
      if (tid == 0) a.spart[d.off_spart + (long long)w.y * 6 + i] = t;
    }
    return;
  }
  // an odd line count leaves the last sequence's imaginary carrier unused: zero it
  if (nl & 1) {
    const int p = nseq - 1;
    float2* z = W0 + (size_t)(p / S) * kWRegion + (p % S) * LS;
    for (int x = tid; x < L; x += blockDim.x) z[x].y = 0.f;
  }
  __syncthreads();
  if (busy) {
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) v[s * P + n1] = Wr[s * LS + 32 * n1 + lane];
#pragma unroll
    for (int r = S * P; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
    fwd_batch<P>(v, Wr, tab, lane);
    if (lane < S * P) {
      const int s = lane / P, k1 = lane - s * P;
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) Wr[s * LS + k1 + P * k2] = v[k2];
    }
  }
  __syncthreads();
  float2* To = a.T1p + d.off_t1 + (long long)row0 * NC * Kx;
  for (int u = tid; u < nl * Kx; u += blockDim.x) {
    const int sl = fdiv(u, d.dKx), j = u - sl * Kx;
    const int k = kxs[j], p = sl >> 1;
    const float2* z = W0 + (size_t)(p / S) * kWRegion + (p % S) * LS;
    const float2 zk = z[k], zm = z[k == 0 ? 0 : L - k];
    float2 out;
    if ((sl & 1) == 0) out = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    else out = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    To[(long long)sl * Kx + j] = out;
  }
}

// Column item with warp-resident FFTs along y (column length L = 32 P): 8 S consecutive line
// columns (of the NC Kx per row) of one RVE, S = 32 / P per warp. Inverse (sign +1): the
// pattern's ky rows of ER scattered into zeroed columns, transformed, all L rows of T1.
// Forward: all L rows of T1p, transformed, the pattern's ky rows into OUT.
template <int P>
__device__ void col_item_warp(const BArgs& a, int g, const BDesc& d, unsigned char* smem,
                              int sign) {
  constexpr int L = 32 * P, S = 32 / P, G = 8 * S, LS = L + P;
  const int NCK = NC * d.Kx;
  const int c0 = g * G, cc_n = min(G, NCK - c0);
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  float2* W0 = reinterpret_cast<float2*>(smem);
  float2* Wr = W0 + (size_t)wp * kWRegion;
  const float2* tab = a.tab + d.tab_y;
  const int* kym = a.kym + d.off_ky;
  if (sign > 0)
    for (int i = lane; i < kWRegion; i += 32) Wr[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const float2* src = sign > 0 ? a.ER + d.off_er : a.T1p + d.off_t1;
  const int rows_in = sign > 0 ? d.Ky : L;
  const int tot = rows_in * cc_n;
  for (int i0 = tid; i0 < tot; i0 += 8 * blockDim.x) {
    float2 v[8];
    int dst[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int i = i0 + u * blockDim.x;
      dst[u] = -1;
      if (i < tot) {
        const int r = i / cc_n, cc = i - r * cc_n;
        v[u] = src[(long long)r * NCK + c0 + cc];
        dst[u] = (cc / S) * kWRegion + (cc % S) * LS + (sign > 0 ? kym[r] : r);
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (dst[u] >= 0) W0[dst[u]] = v[u];
  }
  __syncthreads();
  if (wp * S < cc_n) {
    float2 v[32];
    const float cj = sign > 0 ? -1.f : 1.f;   // the inverse as the conjugate of the forward
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) {
        const float2 z = Wr[s * LS + 32 * n1 + lane];
        v[s * P + n1] = make_float2(z.x, cj * z.y);
      }
#pragma unroll
    for (int r = S * P; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
    fwd_batch<P>(v, Wr, tab, lane);
    if (lane < S * P) {
      const int s = lane / P, k1 = lane - s * P;
#pragma unroll
      for (int k2 = 0; k2 < 32; ++k2) Wr[s * LS + k1 + P * k2] = make_float2(v[k2].x, cj * v[k2].y);
    }
  }
  __syncthreads();
  float2* dstg = sign > 0 ? a.T1 + d.off_t1 : a.OUT + d.off_er;
  const int rows_out = sign > 0 ? L : d.Ky;
  for (int i = tid; i < rows_out * cc_n; i += blockDim.x) {
    const int r = i / cc_n, cc = i - r * cc_n;
    dstg[(long long)r * NCK + c0 + cc] =
        W0[(cc / S) * kWRegion + (cc % S) * LS + (sign > 0 ? r : kym[r])];
  }
  __syncthreads();   // the next item reuses the regions
}

// warp-FFT column items of one column length (a kernel per P and direction)
template <int P, int SIGN>
__global__ __launch_bounds__(256, 2) void kb_y_w(BArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const int2 w = a.items[it];
    if (!a.final_pass && rve_done(a, w.x)) continue;   // the final pass covers every RVE
    const BDesc d = a.d[w.x];
    col_item_warp<P>(a, w.y, d, smem, SIGN);
  }
}

// warp-FFT row items of one row length L = 32 P (their own work list, a kernel per P: each
// has its own register budget)
template <int P>
__global__ __launch_bounds__(256, 2) void kb_row_w(BArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[8];
  for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const int2 w = a.items[it];
    if (!a.final_pass && rve_done(a, w.x)) continue;
    const BDesc d = a.d[w.x];
    __syncthreads();   // the previous item's shared-memory reads are done
    if (a.final_pass) row_item_warp<P, true>(a, w, d, smem, red);
    else row_item_warp<P, false>(a, w, d, smem, red);
    __syncthreads();
  }
}

// ---- RVE-resident solve: a block holds one RVE for every update of its solve
//
// Each block of kResWarps warps takes RVEs from a queue (largest first) and runs all updates of
// its RVE back to back (each the update of Sec. 4, steps d, a, b, c in that order, and the
// convergence test): the inverse y transforms of the coefficients (S line columns per warp),
// the row passes (R_w rows per warp: their 3 R_w lines as packed pairs, inverse x transform,
// law, forward x transform, the coefficients at the pattern's kx), the forward y transforms,
// the Green step with the FP64 measure (a partial per thread, one block sum), and the decision
// (the rules of kb_decide); then the final pass (homogenised stress). Block barriers separate the phases; no
// block waits for another. The line transforms live in the block's scratch slot in global
// memory, [Ny][NC Kx] (the RVE's working set, L2-resident while the block holds it); the RVE's
// parameters, the phase table and the pattern's index maps sit in shared memory.

constexpr int kResWarps = 8;
constexpr int kResThreads = 32 * kResWarps;
constexpr int kResMaxL = 256;
constexpr int kResPhaseBytes = 640;   // a warp item's phase ids (at most 10 rows of 64, 5 of 128)

struct ResCtx {
  float2* T;            // the block's line transforms, [Ny][NC Kx]
  float2* ER;           // the RVE's coefficients, [Ky][NC Kx]
  const float2* tab;    // exp(2 pi i t / L)
  const uint8_t* phase;
  const HIdx* hidx;
  const float4* hn;
  BStat* st;
  int Kx, Ky, Kh, NCK, chunks, pad;   // chunks: as in BDesc (kept for the layout)
  FastDiv dKx;
  float invN, lam0, mu0, inv2mu0, cgam, pad2;
  double N;
};

struct ResShared {
  ResCtx c;
  DevPhase ph[kMaxPhases];
  float2 dph[kMaxPhases];   // per phase (lambda - lambda0, 2 (mu - mu0)) of the RVE's medium
  double sb[kResWarps][6];   // per-warp stress sums of the final pass
  double red[kResWarps];
  int kxs[kResMaxL / 2 + 1];
  int inv_ky[kResMaxL];   // position of ky (mod Ny) in the pattern's ky list, or -1
  int next, done;
  __align__(16) uint8_t phs[kResWarps][kResPhaseBytes];
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
// 8 bytes, zero-filled when bytes = 0 (nothing is read then)
__device__ __forceinline__ void cp_async8(void* dst, const void* src, int bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// y transforms of the NC Kx line columns, S adjacent columns per warp. Inverse (conjugate of the
// forward transform of the conjugate): the pattern's ky rows of ER gathered straight into the
// transform layout, all L rows written to T. Forward: all L rows of T, the pattern's ky rows
// written back in place (row i of T holds the i-th ky of the list afterwards).
template <int P>
__device__ __noinline__ void res_cols(ResShared& sh, float2* Wr, int lane, int wp, bool inverse) {
  constexpr int L = 32 * P, S = 32 / P;
  const ResCtx& c = sh.c;
  const int NCK = c.NCK, groups = (NCK + S - 1) / S;
  const float cj = inverse ? -1.f : 1.f;
  const float2* src = inverse ? c.ER : c.T;
  float2* T = c.T;
  const float2* tab = c.tab;
  // group g's inputs into the region at s L + y by asynchronous copies (zero where the column
  // or the pattern row is absent); the next group's are issued once the transpose has read the
  // region, so they arrive while the 32-point DFTs and the stores run
  auto stage = [&](int g) {
    const int q0 = g * S, ns = min(S, NCK - q0);
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) {
      const int y = 32 * n1 + lane;
      const int row = inverse ? sh.inv_ky[y] : y;
      const float2* p = src + (long long)max(row, 0) * NCK + q0;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const bool ok = row >= 0 && s < ns;
        cp_async8(Wr + s * L + y, ok ? p + s : src, ok ? 8 : 0);
      }
    }
  };
  if (wp < groups) stage(wp);
  for (int g = wp; g < groups; g += kResWarps) {
    const int q0 = g * S, ns = min(S, NCK - q0);
    cp_async_wait_all();
    __syncwarp();
    float2 v[32];
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int n1 = 0; n1 < P; ++n1) {
        const float2 z = Wr[s * L + 32 * n1 + lane];
        v[s * P + n1] = make_float2(z.x, cj * z.y);
      }
#pragma unroll
    for (int r = S * P; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
    fwd_batch_cb<P>(v, Wr, tab, lane, [&] {
      if (g + kResWarps < groups) stage(g + kResWarps);
    });
    if (lane < S * P) {
      const int s = lane / P, k1 = lane - s * P;
      if (s < ns) {
        float2* col = T + q0 + s;
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2) {
          const int y = k1 + P * k2;
          const int row = inverse ? y : sh.inv_ky[y];
          if (row >= 0) col[(long long)row * NCK] = make_float2(v[k2].x, cj * v[k2].y);
        }
      }
    }
  }
}

// row passes: warp items of R_w = 2 S / 3 rows (3 R_w lines, packed in pairs into at most S
// sequences at a stride of L + P entries, which keeps the transform's scattered writes free of
// bank conflicts), each warp on its own items; one transform body for both directions. Final
// pass: homogenised-stress sums per warp instead of the forward transform.
template <int P>
__device__ __noinline__ void res_rows(ResShared& sh, float2* Wr, int lane, int wp, bool final) {
  constexpr int L = 32 * P, S = 32 / P, RW = (2 * S) / 3, LS = L + P;
  constexpr int SU = (3 * RW + 1) / 2;   // sequences in use (3 of 4 at P = 8)
  static_assert(S * LS <= kWRegion && RW * L <= kResPhaseBytes, "region");
  const ResCtx& c = sh.c;
  const int Kx = c.Kx, NCK = c.NCK;
  const float2* tab = c.tab;
  uint8_t* phs = sh.phs[wp];
  const int items = (L + RW - 1) / RW;
  for (int it = wp; it < items; it += kResWarps) {
    const int y0 = it * RW, nr = min(RW, L - y0), nl = nr * NC, nseq = (nl + 1) / 2;
    // the item's phase ids: asynchronous 16-byte copies, waited for before the law
    for (int k = lane; k < nr * L / 16; k += 32)
      cp_async16(phs + 16 * k, c.phase + (long long)y0 * L + 16 * k);
    for (int i = lane; i < SU * LS; i += 32) Wr[i] = make_float2(0.f, 0.f);
    __syncwarp();
    // z_p = line 2p + i line 2p+1 (line s = r NC + c of the item): z[k] = ta + i tb,
    // z[L - k] = conj(ta) + i conj(tb)
    float2* Tg = c.T + (long long)y0 * NCK;
    for (int u0 = lane; u0 < nseq * Kx; u0 += 4 * 32) {
      float2 ta[4], tb[4];
      int jj[4], pp[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int u = u0 + q * 32;
        pp[q] = -1;
        if (u < nseq * Kx) {
          const int p = fdiv(u, c.dKx), j = u - p * Kx;
          const int s0 = 2 * p, s1 = s0 + 1;
          ta[q] = Tg[s0 * Kx + j];
          tb[q] = s1 < nl ? Tg[s1 * Kx + j] : make_float2(0.f, 0.f);
          pp[q] = p;
          jj[q] = j;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (pp[q] < 0) continue;
        const int k = sh.kxs[jj[q]];
        const bool self = (k == 0) || (2 * k == L);
        if (self) {
          ta[q].y = 0.f;
          tb[q].y = 0.f;
        }
        float2* z = Wr + pp[q] * LS;
        z[k] = make_float2(ta[q].x - tb[q].y, ta[q].y + tb[q].x);
        if (!self) z[L - k] = make_float2(ta[q].x + tb[q].y, tb[q].x - ta[q].y);
      }
    }
    __syncwarp();
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const float cj = pass == 0 ? -1.f : 1.f;   // pass 0: inverse, as the conjugate trick
      float2 v[32];
#pragma unroll
      for (int s = 0; s < SU; ++s)
#pragma unroll
        for (int n1 = 0; n1 < P; ++n1) {
          const float2 z = Wr[s * LS + 32 * n1 + lane];
          v[s * P + n1] = make_float2(z.x, cj * z.y);
        }
#pragma unroll
      for (int r = SU * P; r < 32; ++r) v[r] = make_float2(0.f, 0.f);
      fwd_batch_cb<P, SU>(v, Wr, tab, lane, [] {});
      if (lane < SU * P) {
        const int s = lane / P, k1 = lane - s * P;
#pragma unroll
        for (int k2 = 0; k2 < 32; ++k2)
          Wr[s * LS + k1 + P * k2] = make_float2(v[k2].x, cj * v[k2].y);
      }
      __syncwarp();
      if (pass == 1) break;
      cp_async_wait_all();
      __syncwarp();
      // the law on the item's voxels, two rows at a time: rows 2m and 2m + 1 hold lines
      // 6m .. 6m + 5, i.e. whole sequences 3m, 3m + 1 and 3m + 2 (read and written as float2);
      // a missing row 2m + 1 leaves zeros in its carriers
      double s6[6] = {0, 0, 0, 0, 0, 0};
      for (int vx = lane; vx < (nr + 1) / 2 * L; vx += 32) {
        const int m = vx / L, x = vx - m * L;
        const bool two = 2 * m + 1 < nr;
        float2* zA = Wr + 3 * m * LS + x;
        const float2 A = zA[0], B = zA[LS];
        const float2 Cz = two ? zA[2 * LS] : make_float2(0.f, 0.f);
        const float ev[2][NC] = {{A.x, A.y, B.x}, {B.y, Cz.x, Cz.y}};
        float tv[2][NC] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (h == 1 && !two) break;
          float e[NC];
#pragma unroll
          for (int cc = 0; cc < NC; ++cc) e[cc] = ev[h][cc] * c.invN;
          const int pid = phs[(2 * m + h) * L + x];
          if (final) {
            float e6[6];
            comp_to6<NC>(e, e6);
            const DevPhase ph = sh.ph[pid];
            float ep[6] = {0, 0, 0, 0, 0, 0};
            LawOut o;
            stress6<false>(e6, ph, ep, 0.f, o);
#pragma unroll
            for (int i = 0; i < 6; ++i) s6[i] += (double)o.s[i];
          } else {
            // elastic phases in plane strain: tau = sigma - C0 : eps
            //   = (lambda - lambda0) tr(eps) 1 + 2 (mu - mu0) eps, components 11, 22, 12
            const float2 dm = sh.dph[pid];
            const float tr = e[0] + e[1];
            tv[h][0] = fmaf(dm.y, e[0], dm.x * tr);
            tv[h][1] = fmaf(dm.y, e[1], dm.x * tr);
            tv[h][2] = dm.y * e[2];
          }
        }
        if (!final) {
          zA[0] = make_float2(tv[0][0], tv[0][1]);
          zA[LS] = make_float2(tv[0][2], tv[1][0]);
          if (two) zA[2 * LS] = make_float2(tv[1][1], tv[1][2]);
        }
      }
      if (final) {
#pragma unroll
        for (int i = 0; i < 6; ++i) {
          double t = s6[i];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
          if (lane == 0) sh.sb[wp][i] += t;
        }
        break;
      }
      __syncwarp();
    }
    if (!final) {
      for (int u = lane; u < nl * Kx; u += 32) {
        const int sl = fdiv(u, c.dKx), j = u - sl * Kx;
        const int k = sh.kxs[j];
        const float2* z = Wr + (sl >> 1) * LS;
        const float2 zk = z[k], zm = z[k == 0 ? 0 : L - k];
        float2 out;
        if ((sl & 1) == 0) out = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
        else out = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
        Tg[sl * Kx + j] = out;
      }
    }
    __syncwarp();   // the next item rewrites the region and the phase bytes
  }
}

// Green step at the RVE's half-pattern entries (thread t takes entries t, t + kResThreads, ...),
// ER updated, the squared-increment measure summed in FP64 per thread and over the block in a
// fixed order; the sum is valid in thread 0
__device__ __noinline__ double res_green(ResShared& sh) {
  const ResCtx& c = sh.c;
  const int NCK = c.NCK, Kx = c.Kx;
  const double* ebar = c.st->ebar;
  double s = 0.0;
  for (int h = threadIdx.x; h < c.Kh; h += kResThreads) {
    const HIdx hi = c.hidx[h];
    const float4 n = c.hn[h];
    const long long base = (long long)hi.iy * NCK + hi.j;
    float2 tv[NC], old[NC];
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
      tv[cc] = c.T[base + cc * Kx];
      old[cc] = c.ER[base + cc * Kx];
    }
    float er[NC], ei[NC];
    green_update<NC>(hi.kind, n, tv, ebar, c.N, c.inv2mu0, c.cgam, er, ei);
    float diff = 0.f;
#pragma unroll
    for (int cc = 0; cc < NC; ++cc) {
      const float dr = er[cc] - old[cc].x, di = ei[cc] - old[cc].y;
      const float wc = (comp6<NC>(cc) >= 3) ? 2.f : 1.f;
      diff = fmaf(n.w * wc, dr * dr + di * di, diff);
      c.ER[base + cc * Kx] = make_float2(er[cc], ei[cc]);
    }
    s += (double)diff;
  }
  return block_sum_d(s, sh.red);
}

// the decision of kb_decide for one RVE (thread 0)
__device__ bool res_decide(BStat& st, int* n_done, double s) {
  double rr = sqrt(s * st.inv_n2);
  if (st.enorm > 0.0) rr /= st.enorm;
  st.iters += 1;
  st.last_r = rr;
  st.rmin = fmin(st.rmin, rr);
  if (!isfinite(rr)) {
    st.nonfinite = 1;
    st.done = 1;
  } else if (rr > kDivergeRatio * st.rmin && rr > kDivergeFloor) {
    st.diverged = 1;
    st.done = 1;
  } else if (rr < st.tol || st.iters >= st.max_iter) {
    st.done = 1;
  }
  if (st.done) atomicAdd(n_done, 1);
  return st.done != 0;
}

template <int P>
__device__ __noinline__ void res_solve(ResShared& sh, float2* Wr, int* n_done) {
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  for (;;) {
    res_cols<P>(sh, Wr, lane, wp, true);
    __syncthreads();
    res_rows<P>(sh, Wr, lane, wp, false);
    __syncthreads();
    res_cols<P>(sh, Wr, lane, wp, false);
    __syncthreads();
    const double s = res_green(sh);
    if (threadIdx.x == 0) sh.done = res_decide(*sh.c.st, n_done, s) ? 1 : 0;
    __syncthreads();
    if (sh.done) break;
  }
  // final pass: fields of the converged coefficients, homogenised stress
  res_cols<P>(sh, Wr, lane, wp, true);
  __syncthreads();
  res_rows<P>(sh, Wr, lane, wp, true);
  __syncthreads();
  if (threadIdx.x < 6) {
    double t = 0.0;
    for (int w = 0; w < kResWarps; ++w) t += sh.sb[w][threadIdx.x];
    sh.c.st->sbar[threadIdx.x] = t / sh.c.N;
  }
}

// whole solves of the RVEs order[0 .. n_order) (square, sides 64, 96, 128, 192 or 256), a
// block per RVE at a time from the queue counter; T slots of slot float2 per block
__global__ __launch_bounds__(kResThreads, 2) void kb_resident(BArgs a, const int* order,
                                                              int n_order, unsigned* queue,
                                                              float2* scratch, long long slot) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ ResShared sh;
  float2* Wr = reinterpret_cast<float2*>(smem) + (size_t)(threadIdx.x >> 5) * kWRegion;
  if (threadIdx.x < kMaxPhases) sh.ph[threadIdx.x] = a.law.ph[threadIdx.x];
  for (;;) {
    if (threadIdx.x == 0) sh.next = (int)atomicAdd(queue, 1u);
    __syncthreads();
    const int q = sh.next;
    if (q >= n_order) break;
    const int r = order[q];
    const BDesc& d = a.d[r];
    const int nx = d.nx;
    if (threadIdx.x == 0) {
      ResCtx& c = sh.c;
      c.T = scratch + (long long)blockIdx.x * slot;
      c.ER = a.ER + d.off_er;
      c.tab = a.tab + d.tab_x;
      c.phase = a.phase + d.off_phase;
      c.hidx = a.hidx + d.off_h;
      c.hn = a.hn + d.off_h;
      c.st = a.st + r;
      c.Kx = d.Kx;
      c.Ky = d.Ky;
      c.Kh = d.Kh;
      c.NCK = NC * d.Kx;
      c.chunks = d.chunks;
      c.dKx = d.dKx;
      c.invN = 1.f / (float)d.N;
      c.lam0 = d.lam0;
      c.mu0 = d.mu0;
      c.inv2mu0 = d.inv2mu0;
      c.cgam = d.cgam;
      c.N = (double)d.N;
    }
    if (threadIdx.x < kResWarps * 6) sh.sb[threadIdx.x / 6][threadIdx.x % 6] = 0.0;
    if (threadIdx.x < kMaxPhases)
      sh.dph[threadIdx.x] = make_float2(sh.ph[threadIdx.x].lam - d.lam0,
                                        2.f * (sh.ph[threadIdx.x].mu - d.mu0));
    for (int i = threadIdx.x; i < d.Kx; i += kResThreads) sh.kxs[i] = a.kx[d.off_kx + i];
    for (int i = threadIdx.x; i < d.ny; i += kResThreads) sh.inv_ky[i] = -1;
    __syncthreads();
    for (int i = threadIdx.x; i < d.Ky; i += kResThreads) sh.inv_ky[a.kym[d.off_ky + i]] = i;
    __syncthreads();
    switch (nx) {
      case 64: res_solve<2>(sh, Wr, a.n_done); break;
      case 96: res_solve<3>(sh, Wr, a.n_done); break;
      case 128: res_solve<4>(sh, Wr, a.n_done); break;
      case 192: res_solve<6>(sh, Wr, a.n_done); break;
      default: res_solve<8>(sh, Wr, a.n_done); break;
    }
    __syncthreads();   // sh is rewritten for the next RVE
  }
}

__global__ __launch_bounds__(256) void kb_row(BArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[8];
  for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const int2 w = a.items[it];
    if (!a.final_pass && rve_done(a, w.x)) continue;
    const BDesc d = a.d[w.x];
    if (d.fft) {
      __syncthreads();   // the previous item's shared-memory reads are done
      row_item_fft(a, w, d, smem, red);
      __syncthreads();
      continue;
    }
    const int Nx = d.nx, Kx = d.Kx, R = d.R;
    const int row0 = w.y * R;
    const int nr = min(R, d.rows - row0);
    float2* tab = reinterpret_cast<float2*>(smem);
    float2* Ts = tab + Nx;
    int* kxs = reinterpret_cast<int*>(Ts + R * NC * Kx);
    float* fac = reinterpret_cast<float*>(kxs + Kx);
    float* taus = fac + Kx;
    const int tid = threadIdx.x;
    for (int i = tid; i < Nx; i += blockDim.x) tab[i] = a.tab[d.tab_x + i];
    for (int i = tid; i < Kx; i += blockDim.x) {
      kxs[i] = a.kx[d.off_kx + i];
      fac[i] = a.fac[d.off_kx + i];
    }
    const float2* Tg = a.T1 + d.off_t1 + (long long)row0 * NC * Kx;
    for (int i = tid; i < nr * NC * Kx; i += blockDim.x) Ts[i] = Tg[i];
    __syncthreads();
    double sb[6] = {0, 0, 0, 0, 0, 0};
    for (int v = tid; v < nr * Nx; v += blockDim.x) {
      const int r = v / Nx, x = v - r * Nx;
      float e[NC] = {0.f, 0.f, 0.f};
      const float2* Tr = Ts + r * NC * Kx;
      for (int j = 0; j < Kx; ++j) {
        const int m = (kxs[j] * x) % Nx;
        const float2 tw = tab[m];
        const float cr = fac[j] * tw.x, ci = fac[j] * tw.y;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float2 t = Tr[c * Kx + j];
          e[c] = fmaf(t.x, cr, fmaf(-t.y, ci, e[c]));
        }
      }
      float e6[6];
      comp_to6<NC>(e, e6);
      const long long g = (long long)(row0 + r) * Nx + x;
      const DevPhase ph = a.law.ph[a.phase[d.off_phase + g]];
      float ep[6] = {0, 0, 0, 0, 0, 0};
      LawOut o;
      stress6<false>(e6, ph, ep, 0.f, o);
      if (a.final_pass) {
#pragma unroll
        for (int i = 0; i < 6; ++i) sb[i] += (double)o.s[i];
      } else {
        const float tr = e6[0] + e6[1] + e6[2];
        float tau6[6];
#pragma unroll
        for (int i = 0; i < 3; ++i) tau6[i] = o.s[i] - (d.lam0 * tr + 2.f * d.mu0 * e6[i]);
#pragma unroll
        for (int i = 3; i < 6; ++i) tau6[i] = o.s[i] - 2.f * d.mu0 * e6[i];
#pragma unroll
        for (int c = 0; c < NC; ++c) taus[(r * NC + c) * Nx + x] = tau6[comp6<NC>(c)];
      }
    }
    if (a.final_pass) {
      for (int i = 0; i < 6; ++i) {
        const double t = block_sum_d(sb[i], red);
        if (tid == 0) a.spart[d.off_spart + (long long)w.y * 6 + i] = t;
      }
      __syncthreads();
      continue;
    }
    __syncthreads();
    for (int u = tid; u < nr * Kx; u += blockDim.x) {
      const int r = u / Kx, j = u - r * Kx;
      const int kxj = kxs[j];
      const float* tr_ = taus + r * NC * Nx;
      float ar[NC] = {0.f, 0.f, 0.f}, ai[NC] = {0.f, 0.f, 0.f};
      int m = 0;
      for (int x = 0; x < Nx; ++x) {
        const float2 tw = tab[m];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float t = tr_[c * Nx + x];
          ar[c] = fmaf(t, tw.x, ar[c]);
          ai[c] = fmaf(-t, tw.y, ai[c]);
        }
        m += kxj;
        if (m >= Nx) m -= Nx;
      }
      float2* o = a.T1p + d.off_t1 + ((long long)(row0 + r) * NC) * Kx + j;
#pragma unroll
      for (int c = 0; c < NC; ++c) o[c * Kx] = make_float2(ar[c], ai[c]);
    }
    __syncthreads();
  }
}

// Green operator on chunks of 256 half-pattern frequencies, squared-increment partials
__global__ __launch_bounds__(256) void kb_gamma(BArgs a) {
  __shared__ double red[8];
  for (int it = blockIdx.x; it < a.n_items; it += gridDim.x) {
    const int2 w = a.items[it];
    if (rve_done(a, w.x)) continue;
    const BDesc d = a.d[w.x];
    const BStat& st = a.st[w.x];
    const int h = w.y * 256 + threadIdx.x;
    float diff = 0.f;
    if (h < d.Kh) {
      const HIdx hi = a.hidx[d.off_h + h];
      const float4 n = a.hn[d.off_h + h];
      const long long base = ((long long)hi.iy * NC) * d.Kx + hi.j;
      float2* erp = a.ER + d.off_er + base;
      const float2* outp = a.OUT + d.off_er + base;
      float2 tv[NC], old[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        tv[c] = outp[c * d.Kx];
        old[c] = erp[c * d.Kx];
      }
      float er[NC], ei[NC];
      green_update<NC>(hi.kind, n, tv, st.ebar, (double)d.N, d.inv2mu0, d.cgam, er, ei);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float dr = er[c] - old[c].x, di = ei[c] - old[c].y;
        const float wc = (comp6<NC>(c) >= 3) ? 2.f : 1.f;
        diff = fmaf(n.w * wc, dr * dr + di * di, diff);
        erp[c * d.Kx] = make_float2(er[c], ei[c]);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) diff += __shfl_down_sync(0xffffffffu, diff, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)diff;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < 8; ++k) t += red[k];
      a.part[d.off_part + w.y] = t;
    }
    __syncthreads();
  }
}

// one thread per RVE: convergence measure from its partials (fixed order), decision (the rules
// of the single-RVE solver: non-finite, diverged, converged or capped)
__global__ void kb_decide(BArgs a, int n_rve) {
  __shared__ bool last;
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rve; r += gridDim.x * blockDim.x) {
    BStat& st = a.st[r];
    if (st.done) continue;
    const BDesc d = a.d[r];
    double s = 0.0;
    for (int k = 0; k < d.chunks; ++k) s += a.part[d.off_part + k];
    double rr = sqrt(s * st.inv_n2);
    if (st.enorm > 0.0) rr /= st.enorm;
    st.iters += 1;
    st.last_r = rr;
    st.rmin = fmin(st.rmin, rr);
    if (!isfinite(rr)) {
      st.nonfinite = 1;
      st.done = 1;
    } else if (rr > kDivergeRatio * st.rmin && rr > kDivergeFloor) {
      st.diverged = 1;
      st.done = 1;
    } else if (rr < st.tol || st.iters >= st.max_iter) {
      st.done = 1;
    }
    if (st.done) atomicAdd(a.n_done, 1);
  }
  if (!a.use_cond) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    *a.counter = 0u;
    // the only call site of the loop condition: one thread of one block per update
    if (atomicAdd(a.n_done, 0) >= n_rve) cudaGraphSetConditional(a.cond, 0u);
  }
}

// homogenised stress per RVE from the final pass partials
__global__ void kb_sbar(BArgs a, int n_rve) {
  for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n_rve; r += gridDim.x * blockDim.x) {
    const BDesc d = a.d[r];
    for (int i = 0; i < 6; ++i) {
      double s = 0.0;
      for (int k = 0; k < d.row_items; ++k) s += a.spart[d.off_spart + (long long)k * 6 + i];
      a.st[r].sbar[i] = s / (double)d.N;
    }
  }
}

// starting coefficients: zero except the zero frequency N ebar, or projected warm starts
// Warm starts come either per half entry in the six-component layout (warm + warm_off[r],
// host-reordered) or, when pwarm is set, from the device slot layout: components 11, 22, 12 of
// half entry h of RVE r at pwarm[(off_h + h) 3 + c].
__global__ void kb_init(BArgs a, int n_rve, const float2* warm, const long long* warm_off,
                        const float2* pwarm) {
  const int r = blockIdx.x;
  if (r >= n_rve) return;
  const BDesc d = a.d[r];
  const BStat& st = a.st[r];
  float2* er = a.ER + d.off_er;
  const long long rect = (long long)d.Ky * NC * d.Kx;
  for (long long i = threadIdx.x; i < rect; i += blockDim.x) er[i] = make_float2(0.f, 0.f);
  __syncthreads();
  if ((warm && warm_off[r] >= 0) || pwarm) {
    const float lam0 = d.lam0, mu0 = d.mu0;
    for (int h = threadIdx.x; h < d.Kh; h += blockDim.x) {
      const HIdx hi = a.hidx[d.off_h + h];
      const float4 n = a.hn[d.off_h + h];
      float outr[6] = {0, 0, 0, 0, 0, 0}, outi[6] = {0, 0, 0, 0, 0, 0};
      if (hi.kind == 0) {
        float e_r[6] = {0, 0, 0, 0, 0, 0}, e_i[6] = {0, 0, 0, 0, 0, 0};
        if (pwarm) {
          const float2* w3 = pwarm + (d.off_h + h) * 3;
          for (int c = 0; c < NC; ++c) {
            e_r[comp6<NC>(c)] = w3[c].x;
            e_i[comp6<NC>(c)] = w3[c].y;
          }
        } else {
          const float2* w6 = warm + warm_off[r] + (long long)h * 6;
          for (int i = 0; i < 6; ++i) {
            e_r[i] = w6[i].x;
            e_i[i] = w6[i].y;
          }
        }
        e_r[2] = e_r[3] = e_r[4] = e_i[2] = e_i[3] = e_i[4] = 0.f;
        float sr[6], si[6];
        const float trr = e_r[0] + e_r[1], tri = e_i[0] + e_i[1];
        for (int i = 0; i < 6; ++i) {
          sr[i] = 2.f * mu0 * e_r[i] + (i < 3 ? lam0 * trr : 0.f);
          si[i] = 2.f * mu0 * e_i[i] + (i < 3 ? lam0 * tri : 0.f);
        }
        gamma6(n, sr, d.inv2mu0, d.cgam, outr);
        gamma6(n, si, d.inv2mu0, d.cgam, outi);
      }
      if (hi.kind != 1) {
        const long long base = ((long long)hi.iy * NC) * d.Kx + hi.j;
        for (int c = 0; c < NC; ++c)
          er[base + (long long)c * d.Kx] = make_float2(outr[comp6<NC>(c)], outi[comp6<NC>(c)]);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < NC) {
    const int c = threadIdx.x;
    er[d.zero_base + (long long)c * d.Kx] =
        make_float2((float)((double)d.N * st.ebar[comp6<NC>(c)]), 0.f);
  }
}

// Network inputs of RVE r (one CTA per RVE). gamma(k) = g^(k) / N at every half entry by
// separable sums: the x transform of a chunk of rows for every kx in [0, nx/2], then the y sum
// per entry, accumulated in the slot table. Then the 48 descriptors from the slots, with
// per-value sums in a fixed order (radial bins decided in FP64 without contraction).
constexpr int kFeatRows = 32;
constexpr int kDescChunk = 512;

__device__ __forceinline__ int radial_bin(int kx, int ky, int nx, int ny) {
  const double a = __ddiv_rn((double)kx, (double)nx), b = __ddiv_rn((double)ky, (double)ny);
  const double r = __dsqrt_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)));
  const double f = floor(__dmul_rn(96.0, r));
  return f >= 23.0 ? 23 : (int)f;
}

__host__ __device__ inline bool desc_fft(int n) {
  const int p2 = (n % 3 == 0) ? n / 3 : n;
  return n >= 2 && (p2 & (p2 - 1)) == 0;
}

__global__ void kb_descriptors(BArgs a, int incl, int rve_base, float* X, rf_slot* slots) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const int r = blockIdx.x;
  const BDesc d = a.d[r];
  const int nx = d.nx, ny = d.ny, Kx = d.Kx;
  // gamma at the half pattern: DFT of the indicator along x at the pattern's kx values for a
  // chunk of rows, then along y at each entry's ky; accumulators stay in shared memory
  // FFT rows for sides 2^b and 3 2^b: twiddles [stage_len(nx)], two packed-row buffers of
  // kFeatRows / 2 sequences; otherwise the indicator rows [kFeatRows][nx] for the DFT
  const bool fft = desc_fft(nx);
  const int spanf = fftc::span_of((kFeatRows / 2) * nx);
  float2* R = reinterpret_cast<float2*>(fsm);                 // [kFeatRows][Kx]
  float* accr = reinterpret_cast<float*>(R + kFeatRows * Kx);  // [Kh]
  float* acci = accr + d.Kh;                                   // [Kh]
  unsigned char* work = reinterpret_cast<unsigned char*>(acci + d.Kh);
  work += (16 - (reinterpret_cast<uintptr_t>(work) & 15)) & 15;
  float* gch = reinterpret_cast<float*>(work);                 // DFT rows
  float2* tw = reinterpret_cast<float2*>(work);                // FFT rows
  float2* f0 = tw + fftc::stage_len(nx);
  float2* f1 = f0 + spanf;
  if (fft) fftc::copy_twiddles(a.tab + d.tab_x, nx, tw);
  const float2* twx = a.tab + d.tab_x;
  const float2* twy = a.tab + d.tab_y;
  const uint8_t* pm = a.phase + d.off_phase;
  const int* kxl = a.kx + d.off_kx;
  rf_slot* sl = slots + d.off_h;
  const float invN = 1.f / (float)d.N;
  for (int h = threadIdx.x; h < d.Kh; h += blockDim.x) {
    const HIdx hi = a.hidx[d.off_h + h];
    const int kx = kxl[hi.j];
    const int kym = a.kym[d.off_ky + hi.iy];
    const int ky = kym <= ny / 2 ? kym : kym - ny;
    rf_slot t;
    t.g_re = 0.f;
    t.g_im = 0.f;
    t.a = (float)kx / (float)nx;
    t.b = (float)ky / (float)ny;
    t.weight = hi.kind == 0 ? a.hn[d.off_h + h].w : 0.f;
    t.inv_n = invN;
    t.rve = rve_base + r;
    t.kind = hi.kind;
    sl[h] = t;
    accr[h] = 0.f;
    acci[h] = 0.f;
  }
  for (int y0 = 0; y0 < ny; y0 += kFeatRows) {
    const int nr = min(kFeatRows, ny - y0);
    __syncthreads();
    if (fft) {
      // rows 2p and 2p + 1 as the real and imaginary carriers of sequence p
      const int P = (nr + 1) / 2;
      for (int i = threadIdx.x; i < P * nx; i += blockDim.x) {
        const int p = i / nx, x = i - p * nx;
        const int ya = 2 * p, yb = ya + 1;
        const float ga = pm[(long long)(y0 + ya) * nx + x] == incl ? 1.f : 0.f;
        const float gb = yb < nr && pm[(long long)(y0 + yb) * nx + x] == incl ? 1.f : 0.f;
        f0[fftc::sw(i)] = make_float2(ga, gb);
      }
      __syncthreads();
      const float2* z = fftc::fft_block(f0, f1, tw, nx, P, -1);
      for (int i = threadIdx.x; i < nr * Kx; i += blockDim.x) {
        const int yy = i / Kx, j = i - yy * Kx;
        const int k = kxl[j], base = (yy >> 1) * nx;
        const float2 zk = z[fftc::sw(base + k)], zm = z[fftc::sw(base + (k == 0 ? 0 : nx - k))];
        R[yy * Kx + j] = (yy & 1) == 0 ? make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y))
                                       : make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
      }
    } else {
      for (int i = threadIdx.x; i < nr * nx; i += blockDim.x)
        gch[i] = pm[(long long)y0 * nx + i] == incl ? 1.f : 0.f;
      __syncthreads();
      for (int i = threadIdx.x; i < nr * Kx; i += blockDim.x) {
        const int yy = i / Kx, j = i - yy * Kx;
        const int kx = kxl[j];
        const float* gr = gch + yy * nx;
        float re = 0.f, im = 0.f;
        int m = 0;
        for (int x = 0; x < nx; ++x) {
          const float gv = gr[x];
          const float2 w = twx[m];   // (cos, sin)(2 pi m / nx)
          re = fmaf(gv, w.x, re);
          im = fmaf(-gv, w.y, im);
          m += kx;
          if (m >= nx) m -= nx;
        }
        R[yy * Kx + j] = make_float2(re, im);
      }
    }
    __syncthreads();
    for (int h = threadIdx.x; h < d.Kh; h += blockDim.x) {
      const HIdx hi = a.hidx[d.off_h + h];
      const int kym = a.kym[d.off_ky + hi.iy];
      float gr = accr[h], gi = acci[h];
      int m = (int)(((long long)kym * y0) % ny);
      for (int yy = 0; yy < nr; ++yy) {
        const float2 v = R[yy * Kx + hi.j];
        const float2 w = twy[m];
        // (v.x + i v.y) (cos - i sin)
        gr = fmaf(v.x, w.x, fmaf(v.y, w.y, gr));
        gi = fmaf(v.y, w.x, fmaf(-v.x, w.y, gi));
        m += kym;
        if (m >= ny) m -= ny;
      }
      accr[h] = gr;
      acci[h] = gi;
    }
  }
  __syncthreads();
  for (int h = threadIdx.x; h < d.Kh; h += blockDim.x) {
    sl[h].g_re = accr[h] * invN;
    sl[h].g_im = acci[h] * invN;
  }
  __syncthreads();
  // descriptors: 24 bin sums and 4 x 4 band anisotropy sums over the nonzero frequencies
  // (half entries weighted by multiplicity), each summed by one lane group in a fixed order
  float* cb = reinterpret_cast<float*>(fsm);        // reuse: [kDescChunk] p, [4][kDescChunk] h
  int* cbin = reinterpret_cast<int*>(cb + 5 * kDescChunk);
  __shared__ float sums[40];
  __shared__ float vf;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  float acc[5] = {0.f, 0.f, 0.f, 0.f, 0.f};   // this warp's values v = warp + nw q, q < 5
  for (int c0 = 0; c0 < d.Kh; c0 += kDescChunk) {
    const int m = min(kDescChunk, d.Kh - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      const int h = c0 + i;
      const HIdx hi = a.hidx[d.off_h + h];
      const rf_slot t = sl[h];
      if (hi.kind == 1) {
        vf = t.g_re;
        cb[i] = 0.f;
        cbin[i] = 0;
        for (int q = 0; q < 4; ++q) cb[(1 + q) * kDescChunk + i] = 0.f;
        continue;
      }
      const int kx = a.kx[d.off_kx + hi.j];
      const int kym = a.kym[d.off_ky + hi.iy];
      const int ky = kym <= ny / 2 ? kym : kym - ny;
      cb[i] = a.hn[d.off_h + h].w * (t.g_re * t.g_re + t.g_im * t.g_im);
      cbin[i] = radial_bin(kx, ky, nx, ny);
      const float aa = t.a, bb = t.b, r2 = aa * aa + bb * bb;
      const float c2 = (aa * aa - bb * bb) / r2, s2 = 2.f * aa * bb / r2;
      cb[kDescChunk + i] = c2;
      cb[2 * kDescChunk + i] = s2;
      cb[3 * kDescChunk + i] = c2 * c2 - s2 * s2;
      cb[4 * kDescChunk + i] = 2.f * s2 * c2;
    }
    __syncthreads();
    for (int q = 0; q < 5; ++q) {
      const int v = warp + nw * q;
      if (v >= 40) break;
      float s = 0.f;
      if (v < 24) {
        for (int i = lane; i < m; i += 32)
          if (cbin[i] == v) s += cb[i];
      } else {
        const int band = (v - 24) >> 2, hm = (v - 24) & 3;
        for (int i = lane; i < m; i += 32)
          if (cbin[i] / 6 == band) s += cb[i] * cb[(1 + hm) * kDescChunk + i];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      acc[q] += s;
    }
  }
  if (lane == 0)
    for (int q = 0; q < 5; ++q) {
      const int v = warp + nw * q;
      if (v < 40) sums[v] = acc[q];
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    float* x = X + (long long)r * RF_MLP_IN;
    float tot = 0.f;
    x[0] = vf;
    for (int i = 0; i < 24; ++i) {
      x[1 + i] = sqrtf(sums[i]);
      tot += sums[i];
    }
    for (int j = 0; j < 4; ++j) {
      float bt = 0.f;
      for (int i = 6 * j; i < 6 * j + 6; ++i) bt += sums[i];
      for (int q = 0; q < 4; ++q) x[25 + 4 * j + q] = sums[24 + 4 * j + q] / (bt + 1e-12f);
    }
    x[41] = sqrtf(tot);
    for (int i = 42; i < RF_MLP_IN; ++i) x[i] = 0.f;
  }
}

// coefficients of the last solve at the slots: out[(off_h + h) 3 + c] (components 11, 22, 12)
__global__ void kb_reduced_strain(BArgs a, float2* out) {
  const int r = blockIdx.x;
  const BDesc d = a.d[r];
  const float2* er = a.ER + d.off_er;
  for (int h = threadIdx.x; h < d.Kh; h += blockDim.x) {
    const HIdx hi = a.hidx[d.off_h + h];
    const long long base = ((long long)hi.iy * NC) * d.Kx + hi.j;
    for (int c = 0; c < NC; ++c) out[(d.off_h + h) * 3 + c] = er[base + (long long)c * d.Kx];
  }
}

}  // namespace

}  // namespace rfk

// ------------------------------------------------------------------------------------------
// host side
struct rf_batch {
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int n = 0;
  rf_options opt{};
  rfk::LawParams law{};
  std::vector<rfk::BDesc> desc;
  std::vector<std::vector<int32_t>> patterns;  // as given
  std::vector<std::vector<long long>> h_src;   // per RVE: half index -> pattern entry
  rfk::BDesc* d_desc = nullptr;
  rfk::BStat* d_stat = nullptr;
  rfk::BStat* h_stat = nullptr;   // pinned
  uint8_t* d_phase = nullptr;
  float2 *d_ER = nullptr, *d_T1 = nullptr, *d_T1p = nullptr, *d_OUT = nullptr;
  rfk::HIdx* d_hidx = nullptr;
  float4* d_hn = nullptr;
  int* d_kx = nullptr;
  float* d_fac = nullptr;
  int* d_kym = nullptr;
  float2* d_tab = nullptr;
  double *d_part = nullptr, *d_spart = nullptr;
  int* d_ndone = nullptr;
  int* h_ndone = nullptr;   // pinned
  // work lists: 0 inverse y, 1 rows, 2 forward y, 3 Green, 4 warp-FFT rows, 5 warp-FFT columns
  int2* d_items[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int n_items[6] = {0, 0, 0, 0, 0, 0};
  int col_warp = 0;                    // 1: warp-FFT column items where the column length allows
  int y_off[6] = {0, 0, 0, 0, 0, 0};   // work list 5: groups of column length 32 P, P = kWP[i]
  float2* d_warm = nullptr;
  long long* d_warm_off = nullptr;
  long long n_slots = 0;    // half entries of all RVEs
  int max_nx = 0;
  long long warm_total = 0;
  int grid = 0;
  size_t row_smem = 0;
  size_t row_w_smem = 0;   // warp-FFT row items (work list 4, grouped by row length)
  int w_off[6] = {0, 0, 0, 0, 0, 0};   // work list 4: items of row length 32 P for P = kWP[i]
  int R_choice[5] = {0, 0, 0, 0, 0};   // rows per row item, per size class (autotuned)
  bool use_fft = true;                 // FFT row and column items where the sides allow
  size_t col_smem = 0;                 // dynamic shared memory of the column kernels
  std::vector<std::pair<int, cudaGraphExec_t>> graphs;
  // one-launch solve: conditional while node over kBatchBody updates
  cudaGraphExec_t while_exec = nullptr;
  cudaGraphConditionalHandle while_cond = 0;
  bool while_failed = false;
  bool capturing_while = false;
  bool last_while = false;         // the last solve ran as the while graph
  unsigned* d_counter = nullptr;   // finished blocks of the decision kernel
  long long launches = 0;
  int last_max_iters = 0;
  // RVE-resident solve (kb_resident): every RVE square with a side of 64, 96, 128, 192 or 256
  bool res_ok = false;             // the batch qualifies
  int resident = 0;                // 1: solves run as kb_resident
  int res_grid = 0;
  long long res_slot = 0;          // float2 per block's line-transform slot
  int* d_order = nullptr;          // RVEs, largest first
  unsigned* d_queue = nullptr;
  float2* d_scratch = nullptr;
};

using namespace rfk;

namespace {

int bfail(cudaError_t e, const char* what) { return cuda_fail(e, what); }

template <class T>
int balloc(T** p, size_t n, const char* what) {
  *p = nullptr;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), std::max<size_t>(n, 1) * sizeof(T));
  return e == cudaSuccess ? RF_OK : bfail(e, what);
}

BArgs batch_args(rf_batch* b, int stage) {
  BArgs a{};
  a.d = b->d_desc;
  a.st = b->d_stat;
  a.items = stage >= 0 ? b->d_items[stage] : nullptr;
  a.n_items = stage >= 0 ? b->n_items[stage] : 0;
  a.phase = b->d_phase;
  a.ER = b->d_ER;
  a.T1 = b->d_T1;
  a.T1p = b->d_T1p;
  a.OUT = b->d_OUT;
  a.hidx = b->d_hidx;
  a.hn = b->d_hn;
  a.kx = b->d_kx;
  a.fac = b->d_fac;
  a.kym = b->d_kym;
  a.tab = b->d_tab;
  a.part = b->d_part;
  a.spart = b->d_spart;
  a.n_done = b->d_ndone;
  a.law = b->law;
  a.counter = b->d_counter;
  a.cond = b->while_cond;
  a.use_cond = b->capturing_while ? 1 : 0;
  return a;
}

constexpr int kWP[5] = {2, 3, 4, 6, 8};   // P of the warp-FFT row lengths 64, 96, 128, 192, 256

int warp_row_kernels(const rf_batch* b) {
  int n = 0;
  for (int i = 0; i < 5; ++i) n += b->w_off[i + 1] > b->w_off[i] ? 1 : 0;
  return n;
}

// the warp-FFT row items, one launch per row length present
void launch_warp_rows(rf_batch* b, bool final_pass) {
  for (int i = 0; i < 5; ++i) {
    const int n = b->w_off[i + 1] - b->w_off[i];
    if (n <= 0) continue;
    BArgs a = batch_args(b, 4);
    a.items = b->d_items[4] + b->w_off[i];
    a.n_items = n;
    a.final_pass = final_pass ? 1 : 0;
    switch (kWP[i]) {
      case 2: kb_row_w<2><<<b->grid, 256, b->row_w_smem, b->stream>>>(a); break;
      case 3: kb_row_w<3><<<b->grid, 256, b->row_w_smem, b->stream>>>(a); break;
      case 4: kb_row_w<4><<<b->grid, 256, b->row_w_smem, b->stream>>>(a); break;
      case 6: kb_row_w<6><<<b->grid, 256, b->row_w_smem, b->stream>>>(a); break;
      default: kb_row_w<8><<<b->grid, 256, b->row_w_smem, b->stream>>>(a); break;
    }
  }
}

int warp_col_kernels(const rf_batch* b) {
  int n = 0;
  for (int i = 0; i < 5; ++i) n += b->y_off[i + 1] > b->y_off[i] ? 1 : 0;
  return n;
}

// the warp-FFT column items of one direction, one launch per column length present
void launch_warp_cols(rf_batch* b, int sign, bool final_pass) {
  for (int i = 0; i < 5; ++i) {
    const int n = b->y_off[i + 1] - b->y_off[i];
    if (n <= 0) continue;
    BArgs a = batch_args(b, 5);
    a.items = b->d_items[5] + b->y_off[i];
    a.n_items = n;
    a.final_pass = final_pass ? 1 : 0;
    const size_t sm = 8 * (size_t)kWRegion * sizeof(float2);
#define RF_YW(PP)                                                                          \
  (sign > 0 ? (kb_y_w<PP, 1><<<b->grid, 256, sm, b->stream>>>(a), 0)                      \
            : (kb_y_w<PP, -1><<<b->grid, 256, sm, b->stream>>>(a), 0))
    switch (kWP[i]) {
      case 2: RF_YW(2); break;
      case 3: RF_YW(3); break;
      case 4: RF_YW(4); break;
      case 6: RF_YW(6); break;
      default: RF_YW(8); break;
    }
#undef RF_YW
  }
}

// kernels of one update: y transforms both ways, the row kernels with items, Green, decision
int update_kernels(const rf_batch* b) {
  return 2 + (b->n_items[0] > 0 ? 1 : 0) + (b->n_items[2] > 0 ? 1 : 0) +
         (b->n_items[1] > 0 ? 1 : 0) + warp_row_kernels(b) + 2 * warp_col_kernels(b);
}

int launch_update(rf_batch* b) {
  const int G = b->grid;
  if (b->n_items[0] > 0) kb_inv_y<<<G, 256, b->col_smem, b->stream>>>(batch_args(b, 0));
  launch_warp_cols(b, +1, false);
  if (b->n_items[1] > 0) kb_row<<<G, 256, b->row_smem, b->stream>>>(batch_args(b, 1));
  launch_warp_rows(b, false);
  if (b->n_items[2] > 0) kb_fwd_y<<<G, 256, b->col_smem, b->stream>>>(batch_args(b, 2));
  launch_warp_cols(b, -1, false);
  kb_gamma<<<G, 256, 0, b->stream>>>(batch_args(b, 3));
  kb_decide<<<(b->n + 255) / 256, 256, 0, b->stream>>>(batch_args(b, -1), b->n);
  b->launches += update_kernels(b);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RF_OK : bfail(e, "batch update");
}

constexpr int kSides[5] = {64, 96, 128, 192, 256};   // the size classes' sides

int size_class(int side) {
  static const int sides[5] = {64, 96, 128, 192, 256};
  for (int i = 0; i < 5; ++i)
    if (side <= sides[i]) return i;
  return 4;
}

// groups of 8 S line columns per warp-FFT column item for columns of ny voxels, 0 where that
// path does not apply
int warp_col_group(const BDesc& d) {
  const int ny = d.ny;
  if (!d.fft_y || (ny != 64 && ny != 96 && ny != 128 && ny != 192 && ny != 256)) return 0;
  return 8 * (32 / (ny / 32));
}

// the y-transform work lists: shared-memory FFT groups or DFT tiles (lists 0 and 2), and with
// b->col_warp the warp-FFT column groups (list 5, grouped by column length)
int build_col_items(rf_batch* b) {
  std::vector<int> order(b->n);
  for (int i = 0; i < b->n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->desc[x].N > b->desc[y].N; });
  std::vector<int2> inv, fwd, yw;
  for (int r : order) {
    const BDesc& d = b->desc[r];
    const int G = b->col_warp ? warp_col_group(d) : 0;
    if (G > 0) {
      for (int k = 0; k < (NC * d.Kx + G - 1) / G; ++k) yw.push_back(make_int2(r, k));
    } else if (d.fft_y) {
      const int groups = (NC * d.Kx + d.cy - 1) / d.cy;
      for (int k = 0; k < groups; ++k) {
        inv.push_back(make_int2(r, k | kColFft));
        fwd.push_back(make_int2(r, k | kColFft));
      }
    } else {
      for (int k = 0; k < d.mt_inv * d.nt; ++k) inv.push_back(make_int2(r, k));
      for (int k = 0; k < d.mt_fwd * d.nt; ++k) fwd.push_back(make_int2(r, k));
    }
  }
  std::stable_sort(yw.begin(), yw.end(), [&](const int2& x, const int2& y) {
    return b->desc[x.x].ny < b->desc[y.x].ny;
  });
  for (int i = 0; i < 6; ++i) b->y_off[i] = 0;
  for (const int2& it : yw) {
    const int P = b->desc[it.x].ny / 32;
    for (int i = 0; i < 5; ++i)
      if (kWP[i] == P) b->y_off[i + 1] += 1;
  }
  for (int i = 0; i < 5; ++i) b->y_off[i + 1] += b->y_off[i];
  std::vector<int2>* lists[3] = {&inv, &fwd, &yw};
  const int slot[3] = {0, 2, 5};
  for (int q = 0; q < 3; ++q) {
    const int st = slot[q];
    if (b->d_items[st]) cudaFree(b->d_items[st]);
    b->d_items[st] = nullptr;
    if (int e = balloc(&b->d_items[st], std::max<size_t>(lists[q]->size(), 1), "batch items"))
      return e;
    b->n_items[st] = (int)lists[q]->size();
    if (!lists[q]->empty()) {
      cudaError_t e = cudaMemcpy(b->d_items[st], lists[q]->data(),
                                 sizeof(int2) * lists[q]->size(), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return bfail(e, "batch upload");
    }
  }
  return RF_OK;
}

// rows per warp-FFT row item for rows of nx voxels (the item's 3 R lines pair into sequences
// that fill the block's eight warps, 32 / P sequences each), 0 where that path does not apply
int warp_rows(int nx) {
  if (nx != 64 && nx != 96 && nx != 128 && nx != 192 && nx != 256) return 0;
  const int S = 32 / (nx / 32);
  return (16 * S) / 3;
}

// row items for a given rows-per-item choice per size class (-1: warp-FFT row items where
// the row length allows them); sets desc R / row_items
int build_row_items(rf_batch* b) {
  std::vector<int2> items, witems;
  std::vector<int> order(b->n);
  for (int i = 0; i < b->n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return b->desc[x].N > b->desc[y].N; });
  size_t smem = 0, wsmem = 0;
  long long spart = 0;
  for (int r : order) {
    BDesc& d = b->desc[r];
    const int choice = b->R_choice[size_class(std::max(d.nx, d.ny))];
    d.warp = (choice < 0 && b->use_fft && warp_rows(d.nx) > 0) ? 1 : 0;
    d.R = d.warp ? std::min(warp_rows(d.nx), d.rows)
                 : std::max(1, std::min(choice < 0 ? 2 : choice, d.rows));
    d.row_items = (d.rows + d.R - 1) / d.R;
    for (int k = 0; k < d.row_items; ++k) (d.warp ? witems : items).push_back(make_int2(r, k));
    const size_t s_dft = (size_t)d.nx * sizeof(float2) + (size_t)d.R * NC * d.Kx * sizeof(float2) +
                         (size_t)d.Kx * 8 + (size_t)d.R * NC * d.nx * sizeof(float) + 64;
    const int P = (d.R * NC + 1) / 2;
    const size_t span = (size_t)fftc::span_of(P * d.nx);
    const size_t s_fft = (size_t)d.nx * sizeof(float2) + 2 * span * sizeof(float2) +
                         (size_t)d.Kx * sizeof(int) + 64;
    const int p2 = d.nx % 3 == 0 ? d.nx / 3 : d.nx;
    d.fft = (b->use_fft && p2 >= 1 && (p2 & (p2 - 1)) == 0 && s_fft <= 160 * 1024) ? 1 : 0;
    const size_t s_warp = (((size_t)d.Kx * sizeof(int) + 15) & ~(size_t)15) +
                          8 * (size_t)kWRegion * sizeof(float2);
    if (d.warp) wsmem = std::max(wsmem, s_warp);
    else smem = std::max(smem, d.fft ? s_fft : s_dft);
  }
  for (int r = 0; r < b->n; ++r) {
    b->desc[r].off_spart = spart;
    spart += (long long)b->desc[r].row_items * 6;
  }
  if (b->d_items[1]) cudaFree(b->d_items[1]);
  if (b->d_items[4]) cudaFree(b->d_items[4]);
  b->d_items[1] = b->d_items[4] = nullptr;
  if (b->d_spart) cudaFree(b->d_spart);
  if (int e = balloc(&b->d_items[1], std::max<size_t>(items.size(), 1), "batch items")) return e;
  if (int e = balloc(&b->d_items[4], std::max<size_t>(witems.size(), 1), "batch items")) return e;
  if (int e = balloc(&b->d_spart, (size_t)spart, "batch partials")) return e;
  b->n_items[1] = (int)items.size();
  b->n_items[4] = (int)witems.size();
  b->row_w_smem = wsmem;
  // group the warp items by row length (stable: largest RVEs first within each)
  std::stable_sort(witems.begin(), witems.end(), [&](const int2& x, const int2& y) {
    return b->desc[x.x].nx < b->desc[y.x].nx;
  });
  for (int i = 0; i < 6; ++i) b->w_off[i] = 0;
  for (const int2& it : witems) {
    const int P = b->desc[it.x].nx / 32;
    for (int i = 0; i < 5; ++i)
      if (kWP[i] == P) b->w_off[i + 1] += 1;
  }
  for (int i = 0; i < 5; ++i) b->w_off[i + 1] += b->w_off[i];
  if (smem > 200 * 1024) {
    set_error("batch: row tile too large for shared memory");
    return RF_ERR_INVALID;
  }
  b->row_smem = smem;
  cudaError_t e = items.empty() ? cudaSuccess
                                : cudaMemcpy(b->d_items[1], items.data(),
                                             sizeof(int2) * items.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !witems.empty())
    e = cudaMemcpy(b->d_items[4], witems.data(), sizeof(int2) * witems.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_desc, b->desc.data(), sizeof(BDesc) * b->n, cudaMemcpyHostToDevice);
  return e == cudaSuccess ? RF_OK : bfail(e, "batch upload");
}

void free_graphs(rf_batch* b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.second);
  b->graphs.clear();
  if (b->while_exec) cudaGraphExecDestroy(b->while_exec);
  b->while_exec = nullptr;
  b->while_failed = false;
}

// One graph for a whole batched solve: a conditional while node whose body is kBatchBody
// updates; the decision kernel's last block clears the condition once every RVE is done, so the
// loop ends with the body in which the last RVE finished (later updates skip every item). If
// the graph cannot be built, the solve replays chunks of updates and polls the done count.
constexpr int kBatchBody = 4;

int while_graph(rf_batch* b) {
  if (b->while_exec || b->while_failed) return RF_OK;
  cudaGraph_t graph = nullptr;
  auto give_up = [&]() {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    b->while_failed = true;
    return RF_OK;
  };
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) return give_up();
  cudaGraphConditionalHandle h = 0;
  if (cudaGraphConditionalHandleCreate(&h, graph, 1u, cudaGraphCondAssignDefault) != cudaSuccess)
    return give_up();
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeWhile;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &p) != cudaSuccess) return give_up();
  cudaGraph_t body = p.conditional.phGraph_out[0];
  b->while_cond = h;
  if (cudaStreamBeginCaptureToGraph(b->stream, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return give_up();
  const long long launched = b->launches;
  b->capturing_while = true;
  int err = RF_OK;
  for (int i = 0; i < kBatchBody && !err; ++i) err = launch_update(b);
  b->capturing_while = false;
  b->launches = launched;
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(b->stream, &captured);
  if (err || ce != cudaSuccess) {
    set_error("");
    return give_up();
  }
  cudaGraphExec_t exec = nullptr;
  if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) return give_up();
  cudaGraphDestroy(graph);
  b->while_exec = exec;
  return RF_OK;
}

int graph_for(rf_batch* b, int chunk, cudaGraphExec_t* out) {
  for (auto& g : b->graphs)
    if (g.first == chunk) {
      *out = g.second;
      return RF_OK;
    }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return bfail(e, "batch capture");
  int err = RF_OK;
  const long long launched = b->launches;   // captured kernels are counted at each replay
  for (int i = 0; i < chunk && !err; ++i) err = launch_update(b);
  b->launches = launched;
  e = cudaStreamEndCapture(b->stream, &graph);
  if (!err && e != cudaSuccess) err = bfail(e, "batch end capture");
  cudaGraphExec_t ex = nullptr;
  if (!err) {
    e = cudaGraphInstantiate(&ex, graph, 0);
    if (e != cudaSuccess) err = bfail(e, "batch instantiate");
  }
  if (graph) cudaGraphDestroy(graph);
  if (err) return err;
  b->graphs.push_back({chunk, ex});
  *out = ex;
  return RF_OK;
}

int set_status(rf_batch* b, const double* macro, int max_iter = 0) {
  for (int r = 0; r < b->n; ++r) {
    BStat& s = b->h_stat[r];
    std::memset(&s, 0, sizeof(s));
    s.max_iter = max_iter > 0 ? max_iter : b->opt.max_iter;
    s.tol = max_iter > 0 ? 0.0 : b->opt.tol;
    const double* m = macro + 6 * r;
    for (int i = 0; i < 6; ++i) s.ebar[i] = m[i];
    s.enorm = std::sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2] +
                        2.0 * (m[3] * m[3] + m[4] * m[4] + m[5] * m[5]));
    const double N = (double)b->desc[r].N;
    s.inv_n2 = 1.0 / (N * N);
    s.rmin = HUGE_VAL;
  }
  cudaError_t e = cudaMemcpyAsync(b->d_stat, b->h_stat, sizeof(BStat) * b->n,
                                  cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_ndone, 0, sizeof(int), b->stream);
  return e == cudaSuccess ? RF_OK : bfail(e, "batch status");
}

// iterate until every RVE is done: one while-graph launch, or replayed chunks of updates with
// a host read of the done count after each
int iterate(rf_batch* b) {
  if (int e = while_graph(b)) return e;
  if (b->while_exec) {
    cudaError_t e = cudaGraphLaunch(b->while_exec, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->h_ndone, b->d_ndone, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(e, "batch iterate");
    b->last_while = true;   // kernels launched are counted from the iterations in finish_solve
    return RF_OK;
  }
  b->last_while = false;
  const int maxchunk = b->opt.check_every > 0 ? b->opt.check_every : 16;
  int chunk = std::min(4, maxchunk);
  for (;;) {
    cudaGraphExec_t ex;
    if (int e = graph_for(b, chunk, &ex)) return e;
    cudaError_t e = cudaGraphLaunch(ex, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->h_ndone, b->d_ndone, sizeof(int), cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bfail(e, "batch iterate");
    b->launches += (long long)update_kernels(b) * chunk;
    if (*b->h_ndone >= b->n) break;
    chunk = std::min(chunk * 2, maxchunk);
  }
  return RF_OK;
}

constexpr size_t kResSmem = (size_t)kResWarps * kWRegion * sizeof(float2);

// every RVE's whole solve (updates and final pass) in one kb_resident launch
int launch_resident(rf_batch* b) {
  cudaError_t e = cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned), b->stream);
  if (e != cudaSuccess) return bfail(e, "batch resident");
  kb_resident<<<b->res_grid, kResThreads, kResSmem, b->stream>>>(
      batch_args(b, -1), b->d_order, b->n, b->d_queue, b->d_scratch, b->res_slot);
  b->launches += 1;
  e = cudaGetLastError();
  return e == cudaSuccess ? RF_OK : bfail(e, "batch resident");
}

int run_solve(rf_batch* b, const double* macro, bool use_warm, const float2* pwarm = nullptr) {
  if (int e = set_status(b, macro)) return e;
  BArgs a = batch_args(b, -1);
  kb_init<<<b->n, 256, 0, b->stream>>>(a, b->n, use_warm ? b->d_warm : nullptr, b->d_warm_off,
                                       pwarm);
  b->launches += 1;
  if (cudaGetLastError() != cudaSuccess) return bfail(cudaGetLastError(), "batch init");
  if (b->resident) {
    b->last_while = false;
    return launch_resident(b);
  }
  return iterate(b);
}

// Autotuner: rows per row item for each size class present (coordinate descent: one class at
// a time, the others held), then the persistent grid size, each candidate timed as the fastest
// of three groups of two updates of the whole batch (CUDA events on the batch's stream).
int autotune(rf_batch* b, const double* macro) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev);
  const int Rc[5] = {1, 2, 4, 8, -1};   // -1: warp-FFT row items
  const int Gc[3] = {2, 4, 8};
  bool present[5] = {false, false, false, false, false};
  for (const BDesc& d : b->desc) present[size_class(std::max(d.nx, d.ny))] = true;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return bfail(cudaGetLastError(), "batch tuner");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return bfail(cudaGetLastError(), "batch tuner");
  }
  auto time_updates = [&](float* ms) -> int {
    if (int e = set_status(b, macro)) return e;
    kb_init<<<b->n, 256, 0, b->stream>>>(batch_args(b, -1), b->n, nullptr, b->d_warm_off,
                                         nullptr);
    if (int e = launch_update(b)) return e;   // warm-up
    *ms = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0, b->stream);
      for (int i = 0; i < 2; ++i)
        if (int e = launch_update(b)) return e;
      cudaEventRecord(e1, b->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) return bfail(cudaGetLastError(), "batch tuner");
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      *ms = std::min(*ms, t);
    }
    return RF_OK;
  };
  int err = RF_OK;
  for (int k = 0; k < 5; ++k) b->R_choice[k] = 2;
  b->grid = sms * 4;
  for (int k = 0; k < 5 && !err; ++k) {
    if (!present[k]) continue;
    float best = 1e30f;
    int bestR = b->R_choice[k];
    for (int R : Rc) {
      // options.fft_row_warps: -1 never the warp-FFT items, > 0 only them (where they apply)
      const int ow = b->opt.fft_row_warps;
      if (R < 0 && (!b->use_fft || ow < 0)) continue;
      if (R > 0 && ow > 0 && b->use_fft && warp_rows(kSides[k]) > 0) continue;
      b->R_choice[k] = R;
      float ms = 0.f;
      err = build_row_items(b);
      if (!err) err = time_updates(&ms);
      if (err) break;
      if (ms < best) {
        best = ms;
        bestR = R;
      }
    }
    b->R_choice[k] = bestR;
  }
  if (!err) err = build_row_items(b);
  if (!err && b->use_fft && b->opt.fft_row_warps != 0) {
    b->col_warp = b->opt.fft_row_warps > 0 ? 1 : 0;
    err = build_col_items(b);
  } else if (!err && b->use_fft) {
    // warp-FFT column items against the shared-memory ones
    float t1 = 1e30f, t0 = 1e30f;
    b->col_warp = 1;
    err = build_col_items(b);
    if (!err) err = time_updates(&t1);
    if (!err) {
      b->col_warp = 0;
      err = build_col_items(b);
      if (!err) err = time_updates(&t0);
    }
    if (!err) {
      b->col_warp = t1 < t0 ? 1 : 0;
      err = build_col_items(b);
    }
  }
  if (!err) {
    float best = 1e30f;
    int bestG = 4;
    for (int G : Gc) {
      b->grid = sms * G;
      float ms = 0.f;
      err = time_updates(&ms);
      if (err) break;
      if (ms < best) {
        best = ms;
        bestG = G;
      }
    }
    b->grid = sms * bestG;
  }
  // options.batch_resident: -1 never, 1 always (where the batch qualifies), 0 the faster of a
  // three-update solve each way (the sweeps without their final pass, the resident kernel with)
  b->resident = 0;
  if (!err && b->res_ok && b->opt.batch_resident > 0) b->resident = 1;
  if (!err && b->res_ok && b->opt.batch_resident == 0) {
    auto time_solve = [&](bool res, float* ms) -> int {
      *ms = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        if (int e = set_status(b, macro, 3)) return e;
        cudaEventRecord(e0, b->stream);
        kb_init<<<b->n, 256, 0, b->stream>>>(batch_args(b, -1), b->n, nullptr, b->d_warm_off,
                                             nullptr);
        if (res) {
          if (int e = launch_resident(b)) return e;
        } else {
          for (int i = 0; i < 3; ++i)
            if (int e = launch_update(b)) return e;
        }
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess)
          return bfail(cudaGetLastError(), "batch tuner");
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = std::min(*ms, t);
      }
      return RF_OK;
    };
    float t_sweep = 0.f, t_res = 0.f;
    err = time_solve(false, &t_sweep);
    if (!err) err = time_solve(true, &t_res);
    if (!err) b->resident = t_res < t_sweep ? 1 : 0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return err;
}

// final pass: fields of the converged coefficients -> homogenised stresses; per-RVE outputs
int finish_solve(rf_batch* b, double* hom_stress, int32_t* iters, double* residuals,
                 int32_t* status) {
  // final pass: fields of the converged coefficients -> homogenised stresses (kb_resident
  // ran its own)
  if (!b->resident) {
    BArgs a0 = batch_args(b, 0);
    a0.final_pass = 1;
    if (b->n_items[0] > 0) kb_inv_y<<<b->grid, 256, b->col_smem, b->stream>>>(a0);
    launch_warp_cols(b, +1, true);
    BArgs a1 = batch_args(b, 1);
    a1.final_pass = 1;
    if (b->n_items[1] > 0) kb_row<<<b->grid, 256, b->row_smem, b->stream>>>(a1);
    launch_warp_rows(b, true);
    kb_sbar<<<(b->n + 255) / 256, 256, 0, b->stream>>>(batch_args(b, -1), b->n);
    b->launches += 1 + (b->n_items[0] > 0 ? 1 : 0) + warp_col_kernels(b) +
                   (b->n_items[1] > 0 ? 1 : 0) + warp_row_kernels(b);
  }
  cudaError_t e = cudaMemcpyAsync(b->h_stat, b->d_stat, sizeof(BStat) * b->n,
                                  cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bfail(e, "batch final pass");
  int code = RF_OK;
  b->last_max_iters = 0;
  for (int r = 0; r < b->n; ++r) {
    const BStat& s = b->h_stat[r];
    if (hom_stress)
      for (int i = 0; i < 6; ++i) hom_stress[6 * r + i] = s.sbar[i];
    if (iters) iters[r] = s.iters;
    if (residuals) residuals[r] = s.last_r;
    const int st = s.nonfinite ? RF_ERR_NONFINITE
                   : s.diverged ? RF_ERR_DIVERGED
                                : (s.last_r < b->opt.tol ? RF_OK : RF_NOT_CONVERGED);
    if (status) status[r] = st;
    if (st != RF_OK && code == RF_OK) code = RF_NOT_CONVERGED;
    b->last_max_iters = std::max(b->last_max_iters, s.iters);
  }
  if (b->last_while)   // bodies of kBatchBody updates
    b->launches += (long long)update_kernels(b) * kBatchBody *
                   ((b->last_max_iters + kBatchBody - 1) / kBatchBody);
  return code;
}

}  // namespace

extern "C" {

int rf_batch_create(rf_batch** out, int32_t n_rve, const rf_grid* grids,
                    const uint8_t* const* phase_maps, int32_t n_phases, const rf_phase* phases,
                    const int32_t* const* patterns, const int64_t* K, const rf_options* opt,
                    void* stream) {
  set_error("");
  if (!out || n_rve < 1 || !grids || !phase_maps || !phases || !patterns || !K || !opt) {
    set_error("rf_batch_create: invalid arguments");
    return RF_ERR_INVALID;
  }
  *out = nullptr;
  if (n_phases < 1 || n_phases > kMaxPhases) {
    set_error("rf_batch_create: n_phases must be in [1, 16]");
    return RF_ERR_INVALID;
  }
  for (int p = 0; p < n_phases; ++p) {
    if (!std::isfinite(phases[p].lambda) || !std::isfinite(phases[p].mu)) {
      set_error("rf_batch_create: phase moduli must be finite");
      return RF_ERR_NONFINITE;
    }
    if (phases[p].plastic || !(phases[p].mu > 0.0) ||
        !(phases[p].lambda + 2.0 * phases[p].mu / 3.0 > 0.0)) {
      set_error("rf_batch_create: elastic phases with mu > 0, lambda + 2 mu / 3 > 0 only");
      return RF_ERR_INVALID;
    }
  }
  if ((opt->transform != RF_TRANSFORM_DFT && opt->transform != RF_TRANSFORM_FFT) ||
      opt->precision != RF_PREC_FP32 || opt->max_iter < 1 || !(opt->tol >= 0.0) ||
      (opt->green != 0 && opt->green != 1) ||
      (opt->ref_medium != RF_REF_MINMAX && opt->ref_medium != RF_REF_VOLUME) ||
      opt->batch_resident < -1 || opt->batch_resident > 1) {
    set_error("rf_batch_create: options must select FP32 precision, the DFT or FFT transform, "
              "tol >= 0, max_iter >= 1, a known Green operator and reference medium, and "
              "batch_resident -1, 0 or 1");
    return RF_ERR_INVALID;
  }
  rf_batch* b = new rf_batch();
  cudaGetDevice(&b->dev);
  b->n = n_rve;
  b->opt = *opt;
  b->use_fft = opt->transform == RF_TRANSFORM_FFT;
  b->stream = static_cast<cudaStream_t>(stream);
  if (!b->stream) {
    cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    b->own_stream = true;
  }
  for (int p = 0; p < n_phases; ++p) {
    b->law.ph[p].lam = (float)phases[p].lambda;
    b->law.ph[p].mu = (float)phases[p].mu;
  }
  // per-RVE pattern bookkeeping (same rules as rf_set_pattern)
  std::vector<uint8_t> all_phase;
  std::vector<int> kx_all, kym_all;
  std::vector<float> fac_all;
  std::vector<HIdx> hidx_all;
  std::vector<int> hk_all;        // kx, ky, kz, mult per half entry
  std::vector<int> tab_sizes;     // distinct sizes
  std::map<int, int> tab_off;
  long long off_er = 0, off_t1 = 0, off_h = 0, off_kx = 0, off_ky = 0, off_part = 0;

  b->desc.resize(n_rve);
  b->h_src.resize(n_rve);
  auto fail = [&](const char* msg) {
    set_error(msg);
    rf_batch_destroy(b);
    return RF_ERR_INVALID;
  };
  for (int r = 0; r < n_rve; ++r) {
    const rf_grid& g = grids[r];
    if (g.dim != 2 || g.n[2] != 1 || g.n[0] < 2 || g.n[1] < 2 || g.n[0] > 1024 || g.n[1] > 1024)
      return fail("rf_batch_create: 2D grids with sides in [2, 1024] only");
    const int nx = g.n[0], ny = g.n[1];
    const long long N = (long long)nx * ny;
    BDesc& d = b->desc[r];
    std::memset(&d, 0, sizeof(d));
    d.nx = nx;
    d.ny = ny;
    d.N = N;
    d.rows = ny;
    d.off_phase = (long long)all_phase.size();
    unsigned long long present = 0;
    for (long long i = 0; i < N; ++i) {
      const uint8_t v = phase_maps[r][i];
      if (v >= n_phases) return fail("rf_batch_create: phase id >= n_phases");
      present |= 1ull << v;
      all_phase.push_back(v);
    }
    double lmin = 1e300, lmax = -1e300, mmin = 1e300, mmax = -1e300;
    for (int p = 0; p < n_phases; ++p)
      if (present & (1ull << p)) {
        lmin = std::min(lmin, phases[p].lambda);
        lmax = std::max(lmax, phases[p].lambda);
        mmin = std::min(mmin, phases[p].mu);
        mmax = std::max(mmax, phases[p].mu);
      }
    double lam0 = 0.5 * (lmin + lmax), mu0 = 0.5 * (mmin + mmax);
    if (opt->ref_medium == RF_REF_VOLUME) {
      double ls = 0, ms = 0;
      for (long long i = 0; i < N; ++i) {
        ls += phases[phase_maps[r][i]].lambda;
        ms += phases[phase_maps[r][i]].mu;
      }
      lam0 = ls / N;
      mu0 = ms / N;
    }
    d.lam0 = (float)lam0;
    d.mu0 = (float)mu0;
    d.inv2mu0 = (float)(0.5 / mu0);
    d.cgam = (float)((lam0 + mu0) / (mu0 * (lam0 + 2.0 * mu0)));
    // pattern
    const long long Kr = K[r];
    if (Kr < 1 || Kr > N) return fail("rf_batch_create: K must be in [1, N]");
    std::map<std::tuple<int, int>, long long> index;
    int zeros = 0;
    for (long long p = 0; p < Kr; ++p) {
      const int kx = patterns[r][3 * p], ky = patterns[r][3 * p + 1], kz = patterns[r][3 * p + 2];
      if (kz != 0 || kx < -((nx - 1) / 2) || kx > nx / 2 || ky < -((ny - 1) / 2) || ky > ny / 2)
        return fail("rf_batch_create: frequency outside the signed range");
      if (!index.emplace(std::make_tuple(kx, ky), p).second)
        return fail("rf_batch_create: duplicate frequency");
      if (kx == 0 && ky == 0) ++zeros;
    }
    if (zeros != 1) return fail("rf_batch_create: the zero frequency must be present");
    auto sgn = [](int i, int n) { return i <= n / 2 ? i : i - n; };
    auto wrp = [](int k, int n) { return ((k % n) + n) % n; };
    for (auto& kv : index) {
      auto [kx, ky] = kv.first;
      if (!index.count(std::make_tuple(sgn(wrp(-kx, nx), nx), sgn(wrp(-ky, ny), ny))))
        return fail("rf_batch_create: pattern is not closed under k -> -k");
    }
    std::vector<std::tuple<int, int>> H;
    for (auto& kv : index)
      if (std::get<0>(kv.first) >= 0) H.push_back(kv.first);
    std::sort(H.begin(), H.end());
    std::vector<int> xs, ys;
    for (auto& t : H) {
      xs.push_back(std::get<0>(t));
      ys.push_back(std::get<1>(t));
    }
    std::sort(xs.begin(), xs.end());
    xs.erase(std::unique(xs.begin(), xs.end()), xs.end());
    std::sort(ys.begin(), ys.end());
    ys.erase(std::unique(ys.begin(), ys.end()), ys.end());
    d.Kx = (int)xs.size();
    d.Ky = (int)ys.size();
    d.Kh = (int)H.size();
    auto pos = [](const std::vector<int>& v, int x) {
      return (int)(std::lower_bound(v.begin(), v.end(), x) - v.begin());
    };
    d.off_er = off_er;
    d.off_t1 = off_t1;
    d.off_h = off_h;
    d.off_kx = off_kx;
    d.off_ky = off_ky;
    d.off_part = off_part;
    d.chunks = (d.Kh + 255) / 256;
    d.nt = (NC * d.Kx + 63) / 64;
    d.mt_inv = (ny + 31) / 32;
    d.mt_fwd = (d.Ky + 31) / 32;
    {
      const int p2 = ny % 3 == 0 ? ny / 3 : ny;
      d.cy = std::max(1, std::min(16, 4096 / ny));
      const size_t cs = ((size_t)ny + 2 * (size_t)fftc::span_of(d.cy * ny)) * sizeof(float2);
      d.fft_y = (b->use_fft && (p2 & (p2 - 1)) == 0 && cs <= 120 * 1024) ? 1 : 0;
      if (d.fft_y) b->col_smem = std::max(b->col_smem, cs);
    }
    d.zero_base = ((long long)pos(ys, 0) * NC) * d.Kx + pos(xs, 0);
    std::map<std::tuple<int, int>, long long> hpos;
    b->h_src[r].assign(d.Kh, 0);
    for (int h = 0; h < d.Kh; ++h) {
      auto [kx, ky] = H[h];
      hpos[H[h]] = h;
      const bool self = (kx == 0) || (nx % 2 == 0 && kx == nx / 2);
      hidx_all.push_back(HIdx{pos(xs, kx), pos(ys, ky), 0, 0});
      hk_all.insert(hk_all.end(), {kx, ky, 0, self ? 1 : 2});
    }
    for (long long p = 0; p < Kr; ++p) {
      const int kx = patterns[r][3 * p], ky = patterns[r][3 * p + 1];
      if (kx >= 0) b->h_src[r][hpos[std::make_tuple(kx, ky)]] = p;
    }
    b->max_nx = std::max(b->max_nx, nx);
    for (int j = 0; j < d.Kx; ++j) {
      kx_all.push_back(xs[j]);
      const bool self = (xs[j] == 0) || (nx % 2 == 0 && xs[j] == nx / 2);
      fac_all.push_back((float)((self ? 1.0 : 2.0) / (double)N));
    }
    for (int i = 0; i < d.Ky; ++i) kym_all.push_back(wrp(ys[i], ny));
    for (int L : {nx, ny})
      if (!tab_off.count(L)) {
        tab_off[L] = 0;
        tab_sizes.push_back(L);
      }
    off_er += (long long)d.Ky * NC * d.Kx;
    off_t1 += (long long)ny * NC * d.Kx;
    off_h += d.Kh;
    off_kx += d.Kx;
    off_ky += d.Ky;
    off_part += d.chunks;
    b->patterns.emplace_back(patterns[r], patterns[r] + 3 * Kr);
  }
  long long tab_total = 0;
  for (int L : tab_sizes) {   // even lengths keep every stage table 16-byte aligned
    tab_off[L] = (int)tab_total;
    tab_total += fftc::table_len(L);
  }
  for (auto& d : b->desc) {
    d.tab_x = tab_off[d.nx];
    d.tab_y = tab_off[d.ny];
    d.dKx = make_fastdiv((unsigned)std::max(1, d.Kx));
    d.dnx = make_fastdiv((unsigned)d.nx);
  }
  int err = RF_OK;
  int* d_hk = nullptr;
  if (!err) err = balloc(&b->d_desc, n_rve, "batch");
  if (!err) err = balloc(&b->d_stat, n_rve, "batch");
  if (!err) err = cudaMallocHost(&b->h_stat, sizeof(BStat) * n_rve) == cudaSuccess ? RF_OK : RF_ERR_OOM;
  if (!err) err = cudaMallocHost(&b->h_ndone, sizeof(int)) == cudaSuccess ? RF_OK : RF_ERR_OOM;
  if (!err) err = balloc(&b->d_phase, all_phase.size(), "batch phase maps");
  if (!err) err = balloc(&b->d_ER, off_er, "batch coefficients");
  if (!err) err = balloc(&b->d_OUT, off_er, "batch coefficients");
  if (!err) err = balloc(&b->d_T1, off_t1, "batch line transforms");
  if (!err) err = balloc(&b->d_T1p, off_t1, "batch line transforms");
  if (!err) err = balloc(&b->d_hidx, off_h, "batch pattern");
  if (!err) err = balloc(&b->d_hn, off_h, "batch pattern");
  if (!err) err = balloc(&d_hk, hk_all.size(), "batch pattern");
  if (!err) err = balloc(&b->d_kx, off_kx, "batch pattern");
  if (!err) err = balloc(&b->d_fac, off_kx, "batch pattern");
  if (!err) err = balloc(&b->d_kym, off_ky, "batch pattern");
  if (!err) err = balloc(&b->d_tab, tab_total, "batch tables");
  if (!err) err = balloc(&b->d_part, off_part, "batch partials");
  if (!err) err = balloc(&b->d_ndone, 1, "batch");
  if (!err) err = balloc(&b->d_counter, 1, "batch");
  if (!err && cudaMemset(b->d_counter, 0, sizeof(unsigned)) != cudaSuccess)
    err = bfail(cudaGetLastError(), "batch");
  if (!err) err = balloc(&b->d_warm_off, n_rve, "batch");
  b->n_slots = off_h;
  auto up = [&](void* dst, const void* src, size_t bytes) {
    if (err) return;
    cudaError_t e = cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) err = bfail(e, "batch upload");
  };
  up(b->d_phase, all_phase.data(), all_phase.size());
  up(b->d_hidx, hidx_all.data(), sizeof(HIdx) * hidx_all.size());
  up(d_hk, hk_all.data(), sizeof(int) * hk_all.size());
  up(b->d_kx, kx_all.data(), sizeof(int) * kx_all.size());
  up(b->d_fac, fac_all.data(), sizeof(float) * fac_all.size());
  up(b->d_kym, kym_all.data(), sizeof(int) * kym_all.size());
  if (!err) {
    // twiddle tables and wave vectors via the single-RVE setup kernels
    rf_ctx tmp;
    tmp.stream = b->stream;
    for (int L : tab_sizes) {
      tmp.nx = tmp.ny = tmp.nz = L;
      tmp.d_twx = tmp.d_twy = tmp.d_twz = b->d_tab + tab_off[L];
      if (!err) err = launch_setup_tables(&tmp);
    }
    long long h0 = 0;
    for (int r = 0; r < n_rve && !err; ++r) {
      const BDesc& d = b->desc[r];
      tmp.nx = d.nx;
      tmp.ny = d.ny;
      tmp.nz = 1;
      tmp.opt.green = opt->green;
      tmp.d_hidx = b->d_hidx + h0;
      tmp.d_hn = b->d_hn + h0;
      err = launch_hinfo(&tmp, d_hk + 4 * h0, d.Kh);
      h0 += d.Kh;
    }
    b->launches += tmp.launches;
    tmp.d_twx = tmp.d_twy = tmp.d_twz = nullptr;
    tmp.d_hidx = nullptr;
    tmp.d_hn = nullptr;
    if (!err && cudaStreamSynchronize(b->stream) != cudaSuccess) err = RF_ERR_CUDA;
  }
  if (d_hk) cudaFree(d_hk);
  // work lists for the transform, Green and (initial) row stages
  if (!err) {
    std::vector<int> order(n_rve);
    for (int i = 0; i < n_rve; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b->desc[x].N > b->desc[y].N; });
    std::vector<int2> gam;
    for (int r : order) {
      const BDesc& d = b->desc[r];
      for (int k = 0; k < d.chunks; ++k) gam.push_back(make_int2(r, k));
    }
    if (!err) err = balloc(&b->d_items[3], gam.size(), "batch items");
    up(b->d_items[3], gam.data(), sizeof(int2) * gam.size());
    b->n_items[3] = (int)gam.size();
    b->col_warp = (b->use_fft && opt->fft_row_warps >= 0) ? 1 : 0;
    if (!err) err = build_col_items(b);
    std::vector<long long> none(n_rve, -1);
    up(b->d_warm_off, none.data(), sizeof(long long) * n_rve);
    cudaFuncSetAttribute(kb_row, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    for (const void* k : {(const void*)kb_row_w<2>, (const void*)kb_row_w<3>,
                          (const void*)kb_row_w<4>, (const void*)kb_row_w<6>,
                          (const void*)kb_row_w<8>})
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    cudaFuncSetAttribute(kb_inv_y, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    for (const void* k :
         {(const void*)kb_y_w<2, 1>, (const void*)kb_y_w<3, 1>, (const void*)kb_y_w<4, 1>,
          (const void*)kb_y_w<6, 1>, (const void*)kb_y_w<8, 1>, (const void*)kb_y_w<2, -1>,
          (const void*)kb_y_w<3, -1>, (const void*)kb_y_w<4, -1>, (const void*)kb_y_w<6, -1>,
          (const void*)kb_y_w<8, -1>})
      cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    cudaFuncSetAttribute(kb_fwd_y, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
    // the RVE-resident solve: square RVEs with sides of the warp-FFT lengths
    b->res_ok = b->use_fft && opt->batch_resident >= 0;
    long long slot = 0;
    for (const BDesc& d : b->desc) {
      if (d.nx != d.ny || warp_rows(d.nx) == 0) b->res_ok = false;
      slot = std::max(slot, (long long)d.ny * NC * d.Kx);
    }
    if (b->res_ok) {
      cudaFuncSetAttribute(kb_resident, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kResSmem);
      int sms = 152, per_sm = 0;
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kb_resident, kResThreads, kResSmem);
      b->res_grid = sms * std::max(1, per_sm);
      b->res_slot = (slot + 1) & ~1LL;   // 16-byte aligned slots
      if (!err) err = balloc(&b->d_order, order.size(), "batch queue");
      up(b->d_order, order.data(), sizeof(int) * order.size());
      if (!err) err = balloc(&b->d_queue, 1, "batch queue");
      if (!err) err = balloc(&b->d_scratch, (size_t)b->res_grid * b->res_slot, "batch scratch");
    }
  }
  if (!err) {
    std::vector<double> macro0(6 * (size_t)n_rve, 0.0);
    for (int r = 0; r < n_rve; ++r) macro0[6 * r] = 0.01;
    err = autotune(b, macro0.data());
  }
  if (err) {
    std::string keep = rf_last_error();
    rf_batch_destroy(b);
    set_error(keep);
    return err;
  }
  *out = b;
  return RF_OK;
}

int rf_batch_solve(rf_batch* b, const double* macro, const float* const* warm,
                   double* hom_stress, int32_t* iters, double* residuals, int32_t* status) {
  if (!b || !macro) {
    set_error("rf_batch_solve: null argument");
    return RF_ERR_INVALID;
  }
  for (int i = 0; i < 6 * b->n; ++i)
    if (!std::isfinite(macro[i])) {
      set_error("rf_batch_solve: macroscopic strain is not finite");
      return RF_ERR_NONFINITE;
    }
  for (int r = 0; r < b->n; ++r)
    for (int i = 2; i < 5; ++i)
      if (macro[6 * r + i] != 0.0) {
        set_error("rf_batch_solve: plane strain needs macro components 33, 23, 13 = 0");
        return RF_ERR_INVALID;
      }
  bool use_warm = false;
  if (warm) {
    std::vector<long long> off(b->n, -1);
    long long total = 0;
    for (int r = 0; r < b->n; ++r)
      if (warm[r]) {
        off[r] = total;
        total += (long long)b->desc[r].Kh * 6;
      }
    if (total > b->warm_total) {
      if (b->d_warm) cudaFree(b->d_warm);
      if (int e = balloc(&b->d_warm, total, "batch warm")) return e;
      b->warm_total = total;
    }
    std::vector<float2> w6((size_t)std::max(total, 1LL));
    for (int r = 0; r < b->n; ++r) {
      if (!warm[r]) continue;
      for (int h = 0; h < b->desc[r].Kh; ++h) {
        const long long p = b->h_src[r][h];
        for (int i = 0; i < 6; ++i)
          w6[off[r] + (long long)h * 6 + i] =
              make_float2(warm[r][(p * 6 + i) * 2], warm[r][(p * 6 + i) * 2 + 1]);
      }
    }
    cudaError_t e = cudaMemcpy(b->d_warm, w6.data(), sizeof(float2) * std::max(total, 1LL),
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(b->d_warm_off, off.data(), sizeof(long long) * b->n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bfail(e, "batch warm upload");
    use_warm = true;
  }
  if (int e = run_solve(b, macro, use_warm)) return e;
  return finish_solve(b, hom_stress, iters, residuals, status);
}

int rf_batch_slots(const rf_batch* b, int64_t* n_slots, int64_t* offsets) {
  if (!b || !n_slots) {
    set_error("rf_batch_slots: null argument");
    return RF_ERR_INVALID;
  }
  *n_slots = b->n_slots;
  if (offsets) {
    for (int r = 0; r < b->n; ++r) offsets[r] = b->desc[r].off_h;
    offsets[b->n] = b->n_slots;
  }
  return RF_OK;
}

int rf_batch_descriptors(rf_batch* b, int32_t inclusion_phase, int32_t rve_base, float* d_x,
                         rf_slot* d_slots) {
  if (!b || !d_x || !d_slots || inclusion_phase < 0 || inclusion_phase > 255 || rve_base < 0 ||
      (reinterpret_cast<uintptr_t>(d_x) & 15) || (reinterpret_cast<uintptr_t>(d_slots) & 15)) {
    set_error("rf_batch_descriptors: invalid argument");
    return RF_ERR_INVALID;
  }
  size_t smem_dft = 0;
  for (const BDesc& d : b->desc) {
    const size_t rows = desc_fft(d.nx) ? ((size_t)fftc::stage_len(d.nx) +
                                 2 * (size_t)fftc::span_of((kFeatRows / 2) * d.nx)) *
                                    sizeof(float2)
                              : sizeof(float) * (size_t)kFeatRows * d.nx;
    smem_dft = std::max(smem_dft, sizeof(float2) * (size_t)kFeatRows * d.Kx +
                                      sizeof(float) * 2 * (size_t)d.Kh + 16 + rows);
  }
  const size_t smem_desc = (5 * sizeof(float) + sizeof(int)) * (size_t)kDescChunk;
  const size_t smem = std::max(smem_dft, smem_desc);
  cudaFuncSetAttribute(kb_descriptors, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  kb_descriptors<<<b->n, 256, smem, b->stream>>>(batch_args(b, -1), inclusion_phase, rve_base,
                                                  d_x, d_slots);
  b->launches += 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RF_OK : bfail(e, "rf_batch_descriptors");
}

int rf_batch_reduced_strain(rf_batch* b, float* d_coeffs) {
  if (!b || !d_coeffs || (reinterpret_cast<uintptr_t>(d_coeffs) & 15)) {
    set_error("rf_batch_reduced_strain: invalid argument");
    return RF_ERR_INVALID;
  }
  kb_reduced_strain<<<b->n, 256, 0, b->stream>>>(batch_args(b, -1),
                                                  reinterpret_cast<float2*>(d_coeffs));
  b->launches += 1;
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? RF_OK : bfail(e, "rf_batch_reduced_strain");
}

int rf_batch_solve_warm(rf_batch* b, const double* macro, const float* d_warm, double* hom_stress,
                        int32_t* iters, double* residuals, int32_t* status) {
  if (!b || !macro || !d_warm || (reinterpret_cast<uintptr_t>(d_warm) & 7)) {
    set_error("rf_batch_solve_warm: invalid argument");
    return RF_ERR_INVALID;
  }
  for (int i = 0; i < 6 * b->n; ++i)
    if (!std::isfinite(macro[i])) {
      set_error("rf_batch_solve_warm: macroscopic strain is not finite");
      return RF_ERR_NONFINITE;
    }
  for (int r = 0; r < b->n; ++r)
    for (int i = 2; i < 5; ++i)
      if (macro[6 * r + i] != 0.0) {
        set_error("rf_batch_solve_warm: plane strain needs macro components 33, 23, 13 = 0");
        return RF_ERR_INVALID;
      }
  if (int e = run_solve(b, macro, false, reinterpret_cast<const float2*>(d_warm))) return e;
  return finish_solve(b, hom_stress, iters, residuals, status);
}

int rf_batch_info(const rf_batch* b, int64_t* kernel_launches, int32_t* rows_per_item,
                  int32_t* grid) {
  if (!b) {
    set_error("rf_batch_info: null batch");
    return RF_ERR_INVALID;
  }
  if (kernel_launches) *kernel_launches = b->launches;
  if (rows_per_item) {
    static const int sides[5] = {64, 96, 128, 192, 256};
    for (int k = 0; k < 5; ++k)
      rows_per_item[k] = b->R_choice[k] < 0 ? warp_rows(sides[k]) : b->R_choice[k];
  }
  if (grid) *grid = b->grid;
  return RF_OK;
}

int rf_batch_mode(const rf_batch* b, int32_t* resident) {
  if (!b || !resident) {
    set_error("rf_batch_mode: null argument");
    return RF_ERR_INVALID;
  }
  *resident = b->resident;
  return RF_OK;
}

int rf_batch_destroy(rf_batch* b) {
  if (!b) return RF_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  free_graphs(b);
  cudaFree(b->d_desc);
  cudaFree(b->d_stat);
  cudaFree(b->d_phase);
  cudaFree(b->d_ER);
  cudaFree(b->d_T1);
  cudaFree(b->d_T1p);
  cudaFree(b->d_OUT);
  cudaFree(b->d_hidx);
  cudaFree(b->d_hn);
  cudaFree(b->d_kx);
  cudaFree(b->d_fac);
  cudaFree(b->d_kym);
  cudaFree(b->d_tab);
  cudaFree(b->d_part);
  cudaFree(b->d_spart);
  cudaFree(b->d_ndone);
  cudaFree(b->d_counter);
  cudaFree(b->d_warm);
  cudaFree(b->d_warm_off);
  cudaFree(b->d_order);
  cudaFree(b->d_queue);
  cudaFree(b->d_scratch);
  for (int s = 0; s < 6; ++s) cudaFree(b->d_items[s]);
  if (b->h_stat) cudaFreeHost(b->h_stat);
  if (b->h_ndone) cudaFreeHost(b->h_ndone);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return RF_OK;
}

}  // extern "C"
