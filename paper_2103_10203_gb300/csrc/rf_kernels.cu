// Solver kernels of the reduced fixed-point scheme (Sec. 4, steps a-d), FP32 SIMT path.
//
// One iteration is a chain of kernels on the context's stream:
//   [3D] inverse transform along z  (ER -> T2)            step d), part 1
//   inverse transform along y       (ER or T2 -> T1)       step d), part 2
//   row kernel: inverse transform along x, constitutive law, polarization stress,
//               forward transform along x (T1 -> T1p)      steps d) part 3, a), b) part 1
//   forward transform along y       (T1p -> OUT or T2f)    step b), part 2
//   [3D] forward transform along z  (T2f -> OUT)           step b), part 3
//   Green operator update + squared-increment partials     step c)
//   finalize: convergence measure (FP64), device flag      criterion of Sec. 3
// Every kernel returns at once when the device flag says the solve is done, so the host can
// enqueue several iterations between checks without changing the result.
#include <algorithm>
#include <cmath>
#include <cstdio>

#include "rf_fftcore.cuh"
#include "rf_internal.cuh"
#include "rf_law.cuh"

namespace rfk {

// ------------------------------------------------------------------------------------------
// tables and per-frequency data
__global__ void k_twiddle(float2* t, int L) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L) {
    double s, c;
    sincospi(2.0 * (double)i / (double)L, &s, &c);
    t[i] = make_float2((float)c, (float)s);
  }
}

// Stage-major table of a twiddle buffer (rf_fftcore.cuh), one block, after k_twiddle wrote tab.
__global__ void k_stage_table(float2* buf, int L) {
  float2* st = buf + fftc::stage_offset(L);
  fftc::stage_twiddles(buf, L, st);
  for (int i = fftc::twiddle_count(L) + threadIdx.x; i < fftc::stage_len(L); i += blockDim.x)
    st[i] = make_float2(0.f, 0.f);
}

// hk: [Kh][4] = (kx, ky, kz, multiplicity). Writes unit wave vector and the frequency kind.
__global__ void k_hinfo(const int* hk, long long Kh, int nx, int ny, int nz, int green,
                        HIdx* hidx, float4* hn) {
  long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (h >= Kh) return;
  int k[3] = {hk[4 * h], hk[4 * h + 1], hk[4 * h + 2]};
  int n[3] = {nx, ny, nz};
  bool zero = (k[0] == 0 && k[1] == 0 && k[2] == 0);
  int nyq = 0;
  for (int j = 0; j < 3; ++j)
    if (n[j] > 1 && (n[j] % 2) == 0 && k[j] == n[j] / 2) ++nyq;
  double q[3];
  bool null;
  if (green == RF_GREEN_ROTATED) {
    double s[3], c[3];
    for (int j = 0; j < 3; ++j) sincospi((double)k[j] / (double)n[j], &s[j], &c[j]);
    q[0] = 2.0 * s[0] * c[1] * c[2];
    q[1] = 2.0 * s[1] * c[0] * c[2];
    q[2] = 2.0 * s[2] * c[0] * c[1];
    null = !zero && nyq >= 2;   // q = 0 exactly when two components sit at Nyquist
  } else {
    for (int j = 0; j < 3; ++j) q[j] = 2.0 * M_PI * (double)k[j] / (double)n[j];
    null = !zero && nyq >= 1;
  }
  double nn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
  float4 out = make_float4(0.f, 0.f, 0.f, (float)hk[4 * h + 3]);
  if (!zero && !null) {
    out.x = (float)(q[0] / nn);
    out.y = (float)(q[1] / nn);
    out.z = (float)(q[2] / nn);
  }
  hn[h] = out;
  hidx[h].kind = zero ? 1 : (null ? 2 : 0);
}

// ------------------------------------------------------------------------------------------
// line transform along one axis as a batched complex product with generated twiddles:
//   out[s][b][m][n] = sum_{k in split s} w(m, k) * (sum_t in[t][b][k][n]),
//   w(m, k) = exp(sign * 2 pi i * (mv(m) * kv(k) mod L) / L).
// Block: 64 n-columns x 32 m-rows, 256 threads, k staged through shared memory in tiles of 32.
template <int MT>
__global__ __launch_bounds__(256) void k_dft_axis(DftAxisArgs a) {
  if (a.done && *a.done) return;
  __shared__ float2 xs[32][64];
  __shared__ float2 ws[4 * MT][33];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 64 + tx;
  const int n0 = blockIdx.x * 64, m0 = blockIdx.y * (4 * MT);
  const int b = blockIdx.z / a.out_splits, s = blockIdx.z % a.out_splits;
  int kchunk = (a.K + a.out_splits - 1) / a.out_splits;
  kchunk = (kchunk + 31) & ~31;
  const int kbeg = s * kchunk;
  const int kend = min(a.K, kbeg + kchunk);
  float accr[MT], acci[MT];
#pragma unroll
  for (int i = 0; i < MT; ++i) accr[i] = acci[i] = 0.f;
  const float2* inb = a.in + (long long)b * a.in_bstride;
  for (int kb = kbeg; kb < kend; kb += 32) {
    for (int i = tid; i < 32 * 64; i += 256) {
      int kk = i >> 6, nn = i & 63;
      int k = kb + kk, n = n0 + nn;
      float2 v = make_float2(0.f, 0.f);
      if (k < kend && n < a.N) {
        const float2* p = inb + (long long)k * a.N + n;
        for (int t = 0; t < a.in_splits; ++t) {
          float2 u = p[t * a.in_split_stride];
          v.x += u.x;
          v.y += u.y;
        }
      }
      xs[kk][nn] = v;
    }
    for (int i = tid; i < 4 * MT * 32; i += 256) {
      int mm = i >> 5, kk = i & 31;
      int m = m0 + mm, k = kb + kk;
      float2 w = make_float2(0.f, 0.f);
      if (m < a.M && k < kend) {
        int mv = a.mvals ? a.mvals[m] : m;
        int kv = a.kvals ? a.kvals[k] : k;
        w = a.table[(int)(((long long)mv * kv) % a.L)];
        if (a.sign < 0) w.y = -w.y;
      }
      ws[mm][kk] = w;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < 32; ++kk) {
      float2 x = xs[kk][tx];
#pragma unroll
      for (int i = 0; i < MT; ++i) {
        float2 w = ws[ty * MT + i][kk];
        accr[i] = fmaf(w.x, x.x, fmaf(-w.y, x.y, accr[i]));
        acci[i] = fmaf(w.x, x.y, fmaf(w.y, x.x, acci[i]));
      }
    }
    __syncthreads();
  }
  const int n = n0 + tx;
  if (n >= a.N) return;
  float2* ob = a.out + (long long)s * a.out_split_stride + (long long)b * a.out_bstride;
#pragma unroll
  for (int i = 0; i < MT; ++i) {
    int m = m0 + ty * MT + i;
    if (m < a.M) ob[(long long)m * a.N + n] = make_float2(accr[i], acci[i]);
  }
}

// ------------------------------------------------------------------------------------------
// constitutive law: rf_law.cuh

// ------------------------------------------------------------------------------------------
// Row kernel: R grid rows (lines along x) per block.
//   phase 1 (per voxel): eps = (1/N) sum_j w_j Re(T_j exp(+2 pi i kx_j x / Nx)), law, tau
//   phase 2 (per row, kx_j): T'_j = sum_x tau(x) exp(-2 pi i kx_j x / Nx)
// FINAL: phase 1 only, with stress, fields, homogenised-stress partials and the J2 commit.
template <int NC, bool PLASTIC, bool FINAL>
__global__ __launch_bounds__(256) void k_row(RowArgs a) {
  if (!FINAL && a.done && *a.done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  float2* tab = reinterpret_cast<float2*>(smem);
  float2* Ts = tab + a.Nx;
  int* kxs = reinterpret_cast<int*>(Ts + a.R * NC * a.Kx);
  float* fac = reinterpret_cast<float*>(kxs + a.Kx);
  float* taus = fac + a.Kx;
  __shared__ double red[8];

  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * a.R;
  const int nr = min(a.R, a.rows - row0);
  for (int i = tid; i < a.Nx; i += blockDim.x) tab[i] = a.table[i];
  for (int i = tid; i < a.Kx; i += blockDim.x) {
    kxs[i] = a.kx[i];
    fac[i] = a.fac[i];
  }
  const float2* Tg = a.T + (long long)row0 * NC * a.Kx;
  for (int i = tid; i < nr * NC * a.Kx; i += blockDim.x) Ts[i] = Tg[i];
  __syncthreads();

  const bool pow2 = (a.Nx & (a.Nx - 1)) == 0;
  const int mask = a.Nx - 1;
  double sb[6] = {0, 0, 0, 0, 0, 0};
  double vmax = 0.0;
  const float lam0 = a.law.lam0, mu0 = a.law.mu0;
  for (int v = tid; v < nr * a.Nx; v += blockDim.x) {
    const int r = v / a.Nx;
    const int x = v - r * a.Nx;
    const long long g = (long long)(row0 + r) * a.Nx + x;
    float e[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) e[c] = 0.f;
    const float2* Tr = Ts + r * NC * a.Kx;
    for (int j = 0; j < a.Kx; ++j) {
      int m = kxs[j] * x;
      m = pow2 ? (m & mask) : (m % a.Nx);
      const float2 w = tab[m];
      const float f = fac[j];
      const float cr = f * w.x, ci = f * w.y;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float2 t = Tr[c * a.Kx + j];
        e[c] = fmaf(t.x, cr, fmaf(-t.y, ci, e[c]));
      }
    }
    float e6[6];
    comp_to6<NC>(e, e6);
    const DevPhase ph = a.law.ph[a.phase[g]];
    float ep[6] = {0, 0, 0, 0, 0, 0};
    float alpha = 0.f;
    if (PLASTIC) load_state<NC>(a.state, a.N, g, ep, alpha);
    LawOut o;
    stress6<PLASTIC>(e6, ph, ep, alpha, o);
    if (!FINAL) {
      const float tr = e6[0] + e6[1] + e6[2];
      float tau6[6];
#pragma unroll
      for (int i = 0; i < 3; ++i) tau6[i] = o.s[i] - (lam0 * tr + 2.f * mu0 * e6[i]);
#pragma unroll
      for (int i = 3; i < 6; ++i) tau6[i] = o.s[i] - 2.f * mu0 * e6[i];
      float* tr_ = taus + r * NC * a.Nx;
#pragma unroll
      for (int c = 0; c < NC; ++c) tr_[c * a.Nx + x] = tau6[comp6<NC>(c)];
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
          // FP64 consistency check of the FP32 return map: sigma_eq(sigma) = sy + H alpha
          double s0 = o.s[0], s1 = o.s[1], s2 = o.s[2];
          double pmd = (s0 + s1 + s2) / 3.0;
          double d0 = s0 - pmd, d1 = s1 - pmd, d2 = s2 - pmd;
          double q = d0 * d0 + d1 * d1 + d2 * d2 +
                     2.0 * ((double)o.s[3] * o.s[3] + (double)o.s[4] * o.s[4] +
                            (double)o.s[5] * o.s[5]);
          double seq = sqrt(1.5 * q);
          double yl = (double)ph.sy + (double)ph.H * (double)o.alpha;
          vmax = fmax(vmax, fabs(seq - yl) / (double)ph.sy);
        }
      } else if (a.alpha_out) {
        a.alpha_out[g] = 0.f;
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
  __syncthreads();
  for (int u = tid; u < nr * a.Kx; u += blockDim.x) {
    const int r = u / a.Kx;
    const int j = u - r * a.Kx;
    const int kxj = kxs[j];
    const float* tr_ = taus + r * NC * a.Nx;
    float ar[NC], ai[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) ar[c] = ai[c] = 0.f;
    int m = 0;
    for (int x = 0; x < a.Nx; ++x) {
      const float2 w = tab[m];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float t = tr_[c * a.Nx + x];
        ar[c] = fmaf(t, w.x, ar[c]);
        ai[c] = fmaf(-t, w.y, ai[c]);
      }
      m += kxj;
      if (m >= a.Nx) m -= a.Nx;
    }
    float2* o = a.Tout + ((long long)(row0 + r) * NC) * a.Kx + j;
#pragma unroll
    for (int c = 0; c < NC; ++c) o[c * a.Kx] = make_float2(ar[c], ai[c]);
  }
}

// ------------------------------------------------------------------------------------------


template <int NC>
__global__ __launch_bounds__(kGammaBlock) void k_gamma(GammaArgs a, double Nd) {
  __shared__ double red[8];
  __shared__ double sh[256];
  __shared__ bool last;
  const long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const bool act = h < a.Kh;
  // the pattern's indices and wave vectors do not depend on the previous kernel: load them
  // before waiting for it
  HIdx hi{0, 0, 0, 2};
  float4 n = make_float4(0.f, 0.f, 0.f, 0.f);
  if (act) {
    hi = a.hidx[h];
    n = a.hn[h];
  }
  grid_dep_wait();
  // the update's inputs are loaded together with the flag (they are discarded if it is set)
  const int dn = a.done ? __ldcg(a.done) : 0;
  const long long base = ((long long)(hi.iz * a.Ky + hi.iy) * NC) * a.Kx + hi.j;
  const float2* __restrict__ out = a.OUT + base;
  float2* __restrict__ er_p = a.ER + base;
  float2 tv[NC], old[NC];
  if (act) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      tv[c] = out[c * a.Kx];
      old[c] = er_p[c * a.Kx];
    }
  }
  if (dn) return;
  float diff = 0.f;
  if (act) {
    for (int s = 1; s < a.splits; ++s) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float2 u = out[s * a.split_stride + c * a.Kx];
        tv[c].x += u.x;
        tv[c].y += u.y;
      }
    }
    float er[NC], ei[NC];
    const double* eb = a.st->ebar;
    double em[6];
    if (hi.kind == 1 && a.st->mixed) {   // the one zero-frequency thread of the update
      mixed_macro<NC>(tv, Nd, a.st, em);
      for (int i = 0; i < 6; ++i) a.status->ebar[i] = em[i];
      eb = em;
    }
    green_update<NC>(hi.kind, n, tv, eb, Nd, a.inv2mu0, a.cgam, er, ei);
    const float mult = n.w;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float dr = er[c] - old[c].x, di = ei[c] - old[c].y;
      const float wc = (comp6<NC>(c) >= 3) ? 2.f : 1.f;   // Frobenius: shear counted twice
      diff = fmaf(mult * wc, dr * dr + di * di, diff);
      er_p[c * a.Kx] = make_float2(er[c], ei[c]);
    }
  }
  // one frequency's squared increment in FP32 (a sum of at most six non-negative terms); the
  // sums over warps and blocks are FP64
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) diff += __shfl_down_sync(0xffffffffu, diff, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)diff;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  // the last block to finish reduces all partials and takes the convergence decision
  if (threadIdx.x == 0) {
    a.part[blockIdx.x] = t;
    __threadfence();
    const unsigned prev = atomicAdd(a.counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (last) {
    __threadfence();
    decide(a.part, gridDim.x, a.status, sh);
    if (threadIdx.x == 0) {
      *a.counter = 0u;
      // the only call site of the loop condition: one thread of one block per update
      if (a.use_cond && a.status->done) cudaGraphSetConditional(a.cond, 0u);
    }
  }
}

__global__ void k_reduce_sbar(const double* part, const double* vpart, int nb, double invN,
                              double* out) {
  __shared__ double sh[256];
  for (int c = 0; c < 7; ++c) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nb; i += 256)
      s = (c < 6) ? s + part[i * 6 + c] : fmax(s, vpart[i]);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (threadIdx.x < w)
        sh[threadIdx.x] = (c < 6) ? sh[threadIdx.x] + sh[threadIdx.x + w]
                                  : fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
      __syncthreads();
    }
    if (threadIdx.x == 0) out[c] = (c < 6) ? sh[0] * invN : sh[0];
    __syncthreads();
  }
}

// zero frequency of ER: set (mode 0) or add (mode 1) N * value
__global__ void k_zero_freq(float2* ER, long long base0, int NC, int Kx, double Nd, double v0,
                            double v1, double v2, double v3, double v4, double v5, int mode) {
  const double v6[6] = {v0, v1, v2, v3, v4, v5};
  for (int c = threadIdx.x; c < NC; c += blockDim.x) {
    const int c6 = (NC == 3) ? (c == 2 ? 5 : c) : c;
    float2* p = ER + base0 + (long long)c * Kx;
    const float val = (float)(Nd * v6[c6]);
    if (mode == 0) *p = make_float2(val, 0.f);
    else p->x = (float)((double)p->x + Nd * v6[c6]);
  }
}

// warm start: project given coefficients onto compatible strains, P(e) = Gamma0 : (C0 : e)
template <int NC>
__global__ void k_warm_project(const float2* w6, float2* ER, const HIdx* hidx, const float4* hn,
                               long long Kh, int Kx, int Ky, float lam0, float mu0,
                               float inv2mu0, float cg, double Nd, double e0, double e1,
                               double e2, double e3, double e4, double e5) {
  const long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (h >= Kh) return;
  const HIdx hi = hidx[h];
  const long long base = ((long long)(hi.iz * Ky + hi.iy) * NC) * Kx + hi.j;
  const double eb[6] = {e0, e1, e2, e3, e4, e5};
  float outr[6], outi[6];
  if (hi.kind == 1) {
    for (int i = 0; i < 6; ++i) {
      outr[i] = (float)(Nd * eb[i]);
      outi[i] = 0.f;
    }
  } else if (hi.kind == 2) {
    for (int i = 0; i < 6; ++i) outr[i] = outi[i] = 0.f;
  } else {
    float er[6], ei[6];
    for (int i = 0; i < 6; ++i) {
      float2 v = w6[h * 6 + i];
      er[i] = v.x;
      ei[i] = v.y;
    }
    if (NC == 3) er[2] = er[3] = er[4] = ei[2] = ei[3] = ei[4] = 0.f;
    float sr[6], si[6];
    const float trr = er[0] + er[1] + er[2], tri = ei[0] + ei[1] + ei[2];
    for (int i = 0; i < 6; ++i) {
      sr[i] = 2.f * mu0 * er[i] + (i < 3 ? lam0 * trr : 0.f);
      si[i] = 2.f * mu0 * ei[i] + (i < 3 ? lam0 * tri : 0.f);
    }
    const float4 n = hn[h];
    gamma6(n, sr, inv2mu0, cg, outr);
    gamma6(n, si, inv2mu0, cg, outi);
  }
  for (int c = 0; c < NC; ++c) {
    const int c6 = (NC == 3) ? (c == 2 ? 5 : c) : c;
    ER[base + (long long)c * Kx] = make_float2(outr[c6], outi[c6]);
  }
}

__global__ void k_phase_hist(const uint8_t* pm, long long N, unsigned long long* hist) {
  __shared__ unsigned int h[256];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N;
       g += (long long)gridDim.x * blockDim.x)
    atomicAdd(&h[pm[g]], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// ------------------------------------------------------------------------------------------
// host-side launchers
static int launch_check(rf_ctx* c, const char* what) {
  c->launches += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, what);
  return RF_OK;
}

static int dft(rf_ctx* c, const float2* in, int in_splits, long long in_split_stride,
               long long in_bstride, float2* out, int out_splits, long long out_split_stride,
               long long out_bstride, int M, int N, int K, int batch, const int* mvals,
               const int* kvals, const float2* tab, int L, int sign, const int* done) {
  DftAxisArgs a;
  a.in = in;
  a.in_splits = in_splits;
  a.in_split_stride = in_split_stride;
  a.in_bstride = in_bstride;
  a.out = out;
  a.out_splits = out_splits;
  a.out_split_stride = out_split_stride;
  a.out_bstride = out_bstride;
  a.M = M;
  a.N = N;
  a.K = K;
  a.batch = batch;
  a.mvals = mvals;
  a.kvals = kvals;
  a.table = tab;
  a.L = L;
  a.sign = sign;
  a.done = done;
  dim3 block(64, 4);
  dim3 grid((N + 63) / 64, (M + 31) / 32, batch * out_splits);
  k_dft_axis<8><<<grid, block, 0, c->stream>>>(a);
  return launch_check(c, "dft_axis");
}

// twiddle buffers of fftc::table_len(n) entries per axis: plain table, then stage-major table
int launch_setup_tables(rf_ctx* c) {
  const int n[3] = {c->nx, c->ny, c->nz};
  float2* t[3] = {c->d_twx, c->d_twy, c->d_twz};
  for (int a = 0; a < 3; ++a) {
    k_twiddle<<<(n[a] + 255) / 256, 256, 0, c->stream>>>(t[a], n[a]);
    if (int e = launch_check(c, "twiddle table")) return e;
    k_stage_table<<<1, 256, 0, c->stream>>>(t[a], n[a]);
    if (int e = launch_check(c, "twiddle stage table")) return e;
  }
  return RF_OK;
}

int launch_hinfo(rf_ctx* c, const int* d_hk, long long Kh) {
  k_hinfo<<<(unsigned)((Kh + 255) / 256), 256, 0, c->stream>>>(d_hk, Kh, c->nx, c->ny, c->nz,
                                                                c->opt.green, c->d_hidx, c->d_hn);
  return launch_check(c, "hinfo");
}

// per-entry data of the half pattern in kx-grouped order (read without an indirection by the
// Green operator inside the inverse y kernel)
__global__ void k_gather_jentries(const int* jlist, const HIdx* hidx, const float4* hn, long long Kh,
                                  int2* ent, float4* nn) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= Kh) return;
  const int h = jlist[e];
  ent[e] = make_int2(hidx[h].iy, hidx[h].kind);
  nn[e] = hn[h];
}

int launch_gather_jentries(rf_ctx* c) {
  if (c->Kh <= 0) return RF_OK;
  k_gather_jentries<<<(unsigned)((c->Kh + 255) / 256), 256, 0, c->stream>>>(
      c->d_jlist, c->d_hidx, c->d_hn, c->Kh, c->d_jent, c->d_jn);
  return launch_check(c, "gather entries");
}

// Coefficients of a reduced context scattered into the rectangle of a full-set context on the
// same grid (whose distinct values are kx = 0..Nx/2, every ky and kz in signed order); the full
// rectangle is zeroed first by the caller.
template <int NC>
__global__ void k_scatter_full(const float2* ER, const HIdx* hidx, const int* kxv, const int* kym,
                               const int* kzm, long long Kh, int Kx, int Ky, int nx, int ny, int nz,
                               int fKx, int fKy, float2* fER) {
  const long long h = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (h >= Kh) return;
  const HIdx hi = hidx[h];
  const int kx = kxv[hi.j];
  const int ky = kym[hi.iy] <= ny / 2 ? kym[hi.iy] : kym[hi.iy] - ny;
  const int kz = kzm[hi.iz] <= nz / 2 ? kzm[hi.iz] : kzm[hi.iz] - nz;
  const long long src = ((long long)(hi.iz * Ky + hi.iy) * NC) * Kx + hi.j;
  const long long dst =
      ((long long)((kz + (nz - 1) / 2) * fKy + (ky + (ny - 1) / 2)) * NC) * fKx + kx;
#pragma unroll
  for (int c = 0; c < NC; ++c) fER[dst + (long long)c * fKx] = ER[src + (long long)c * Kx];
  (void)nx;
}

int launch_scatter_full(rf_ctx* c, rf_ctx* f) {
  const unsigned gb = (unsigned)((c->Kh + 255) / 256);
  if (c->nc == 3)
    k_scatter_full<3><<<gb, 256, 0, c->stream>>>(c->d_ER, c->d_hidx, c->d_kx, c->d_kym, c->d_kzm,
                                                 c->Kh, c->Kx, c->Ky, c->nx, c->ny, c->nz, f->Kx,
                                                 f->Ky, f->d_ER);
  else
    k_scatter_full<6><<<gb, 256, 0, c->stream>>>(c->d_ER, c->d_hidx, c->d_kx, c->d_kym, c->d_kzm,
                                                 c->Kh, c->Kx, c->Ky, c->nx, c->ny, c->nz, f->Kx,
                                                 f->Ky, f->d_ER);
  return launch_check(c, "scatter to the full set");
}

// Error measures of Sec. 5 between two stress fields [6][N] (tensor shear components, counted
// twice in the Frobenius norm): per block, the sum over its voxels of |sig - ref| / |ref| in FP64
// (voxels with |ref| = 0 add nothing), in a fixed order.
__global__ __launch_bounds__(256) void k_stress_err(const float* sig, const float* ref,
                                                    long long N, double* part) {
  __shared__ double red[8];
  double acc = 0.0;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N;
       g += (long long)gridDim.x * blockDim.x) {
    double num = 0.0, den = 0.0;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const double w = i < 3 ? 1.0 : 2.0;
      const double r = ref[i * N + g], d = (double)sig[i * N + g] - r;
      num += w * d * d;
      den += w * r * r;
    }
    if (den > 0.0) acc += sqrt(num) / sqrt(den);
  }
  const double t = block_sum_d(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// E = sum of the block partials / N; Ebar from the two homogenised stresses. out[0] = Ebar,
// out[1] = E.
__global__ void k_stress_err_final(const double* part, int nb, long long N, double a0, double a1,
                                   double a2, double a3, double a4, double a5, double r0,
                                   double r1, double r2, double r3, double r4, double r5,
                                   double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[b];
  const double a[6] = {a0, a1, a2, a3, a4, a5}, r[6] = {r0, r1, r2, r3, r4, r5};
  double num = 0.0, den = 0.0;
  for (int i = 0; i < 6; ++i) {
    const double w = i < 3 ? 1.0 : 2.0;
    num += w * (a[i] - r[i]) * (a[i] - r[i]);
    den += w * r[i] * r[i];
  }
  out[0] = den > 0.0 ? sqrt(num) / sqrt(den) : sqrt(num);
  out[1] = s / (double)N;
}

int launch_stress_errors(rf_ctx* c, const float* sig_ref, const double* sb, const double* sr) {
  k_stress_err<<<kErrBlocks, 256, 0, c->stream>>>(c->d_sig, sig_ref, c->N, c->d_err);
  if (int e = launch_check(c, "stress errors")) return e;
  k_stress_err_final<<<1, 32, 0, c->stream>>>(c->d_err, kErrBlocks, c->N, sb[0], sb[1], sb[2],
                                              sb[3], sb[4], sb[5], sr[0], sr[1], sr[2], sr[3],
                                              sr[4], sr[5], c->d_err + kErrBlocks);
  return launch_check(c, "stress errors");
}

// Constitutive sweep on its own (step a of Sec. 4 unfused): tau = sigma(eps) - C0 : eps per voxel
// from strain planes in device memory, four consecutive voxels per thread with 16-byte loads and
// stores of every plane (N a multiple of 4, planes 16-byte aligned), grid-stride over the
// voxels. State frozen (read only).
template <int NC, bool PLASTIC>
__global__ __launch_bounds__(256) void k_law_sweep(const float* __restrict__ eps,
                                                   const uint8_t* __restrict__ phase,
                                                   const float* __restrict__ state, long long N,
                                                   LawParams law, float* __restrict__ tau,
                                                   float* __restrict__ sig) {
  constexpr int NS = NC == 3 ? 4 : 7;
  __shared__ DevPhase phs[kMaxPhases];
  for (int i = threadIdx.x; i < kMaxPhases; i += blockDim.x) phs[i] = law.ph[i];
  __syncthreads();
  const long long n4 = N >> 2;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n4;
       q += (long long)gridDim.x * blockDim.x) {
    float4 e4[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) e4[c] = __ldcs(reinterpret_cast<const float4*>(eps + c * N) + q);
    const uchar4 p4 = __ldcs(reinterpret_cast<const uchar4*>(phase) + q);
    float4 s4[NS];
    if (PLASTIC) {
#pragma unroll
      for (int i = 0; i < NS; ++i) s4[i] = __ldcs(reinterpret_cast<const float4*>(state + i * N) + q);
    }
    float4 t4[NC], o4[NC];
    const uint8_t pid[4] = {p4.x, p4.y, p4.z, p4.w};
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      auto pick = [v](const float4& f) { return v == 0 ? f.x : v == 1 ? f.y : v == 2 ? f.z : f.w; };
      float e[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) e[c] = pick(e4[c]);
      float e6[6];
      comp_to6<NC>(e, e6);
      float ep[6] = {0, 0, 0, 0, 0, 0};
      float alpha = 0.f;
      if (PLASTIC) {
        if (NC == 3) {
          ep[0] = pick(s4[0]);
          ep[1] = pick(s4[1]);
          ep[5] = pick(s4[2]);
          ep[2] = -(ep[0] + ep[1]);
          alpha = pick(s4[3]);
        } else {
#pragma unroll
          for (int i = 0; i < 6; ++i) ep[i] = pick(s4[i]);
          alpha = pick(s4[6]);
        }
      }
      LawOut o;
      stress6<PLASTIC>(e6, phs[pid[v]], ep, alpha, o);
      const float tr = e6[0] + e6[1] + e6[2];
      float tau6[6];
#pragma unroll
      for (int i = 0; i < 3; ++i) tau6[i] = o.s[i] - (law.lam0 * tr + 2.f * law.mu0 * e6[i]);
#pragma unroll
      for (int i = 3; i < 6; ++i) tau6[i] = o.s[i] - 2.f * law.mu0 * e6[i];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        float* tp = reinterpret_cast<float*>(&t4[c]);
        float* sp = reinterpret_cast<float*>(&o4[c]);
        tp[v] = tau6[comp6<NC>(c)];
        sp[v] = o.s[comp6<NC>(c)];
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      __stcs(reinterpret_cast<float4*>(tau + c * N) + q, t4[c]);
      if (sig) __stcs(reinterpret_cast<float4*>(sig + c * N) + q, o4[c]);
    }
  }
}

int launch_law_sweep(rf_ctx* c, const float* eps, float* tau, float* sig) {
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
  const long long n4 = c->N >> 2;
  const int grid = (int)std::max(1LL, std::min<long long>(8LL * sms, (n4 + 255) / 256));
  const bool pl = c->has_plastic;
  if (c->nc == 3) {
    if (pl) k_law_sweep<3, true><<<grid, 256, 0, c->stream>>>(eps, c->d_phase, c->d_state, c->N, c->law, tau, sig);
    else k_law_sweep<3, false><<<grid, 256, 0, c->stream>>>(eps, c->d_phase, c->d_state, c->N, c->law, tau, sig);
  } else {
    if (pl) k_law_sweep<6, true><<<grid, 256, 0, c->stream>>>(eps, c->d_phase, c->d_state, c->N, c->law, tau, sig);
    else k_law_sweep<6, false><<<grid, 256, 0, c->stream>>>(eps, c->d_phase, c->d_state, c->N, c->law, tau, sig);
  }
  return launch_check(c, "law sweep");
}

int launch_phase_hist(rf_ctx* c, unsigned long long* d_hist) {
  k_phase_hist<<<304, 256, 0, c->stream>>>(c->d_phase, c->N, d_hist);
  return launch_check(c, "phase_hist");
}

static RowArgs row_args(rf_ctx* c, const int* done) {
  RowArgs a{};
  a.T = c->d_T1;
  a.Tout = c->d_T1p;
  a.phase = c->d_phase;
  a.state = c->d_state;
  a.kx = c->d_kx;
  a.fac = c->d_fac;
  a.table = c->d_twx;
  a.Nx = c->nx;
  a.Kx = c->Kx;
  a.rows = c->rows;
  a.R = c->row_R;
  a.N = c->N;
  a.law = c->law;
  a.done = done;
  return a;
}

void init_attributes_kernels() {
  const int s = 200 * 1024;
  cudaFuncSetAttribute(k_row<3, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_row<3, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_row<3, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_row<3, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_row<6, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_row<6, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_row<6, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
  cudaFuncSetAttribute(k_row<6, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
}

template <int NC, bool PL, bool FIN>
static int row_launch(rf_ctx* c, const RowArgs& a) {
  k_row<NC, PL, FIN><<<c->row_blocks, 256, c->row_smem, c->stream>>>(a);
  return launch_check(c, "row");
}

static int row_dispatch(rf_ctx* c, const RowArgs& a, bool final_pass) {
  const bool pl = c->has_plastic;
  if (c->nc == 3) {
    if (final_pass) return pl ? row_launch<3, true, true>(c, a) : row_launch<3, false, true>(c, a);
    return pl ? row_launch<3, true, false>(c, a) : row_launch<3, false, false>(c, a);
  }
  if (final_pass) return pl ? row_launch<6, true, true>(c, a) : row_launch<6, false, true>(c, a);
  return pl ? row_launch<6, true, false>(c, a) : row_launch<6, false, false>(c, a);
}

int launch_gamma_finalize(rf_ctx* c, int splits, const int* done);

// transforms along y and z: tensor cores (split operands) in the split-precision modes, the
// SIMT DFT otherwise
static int axis(rf_ctx* c, const TcAxis& ax, const float2* in, int in_splits, long long iss,
                long long ibs, float2* out, int out_splits, long long oss, long long obs, int M,
                int N, int K, int batch, const int* mvals, const int* kvals, const float2* tab,
                int L, int sign, const int* done) {
  if (c->opt.precision != RF_PREC_FP32)
    return launch_tc_axis(c, ax, in, in_splits, iss, ibs, out, obs, N, batch, done);
  return dft(c, in, in_splits, iss, ibs, out, out_splits, oss, obs, M, N, K, batch, mvals, kvals,
             tab, L, sign, done);
}

static int inverse_stages(rf_ctx* c, const int* done) {
  const int NCK = c->nc * c->Kx;
  if (c->dim == 3) {
    // along z: T2[z][ky][c][kx] = sum_kz exp(+..kz z) ER[kz][ky][c][kx]
    trace_stage(c, 0);
    if (int e = axis(c, c->tc_zi, c->d_ER, 1, 0, 0, c->d_T2, 1, 0, 0, c->nz, c->Ky * NCK, c->Kz,
                     1, nullptr, c->d_kzm, c->d_twz, c->nz, +1, done))
      return e;
    // along y, batched over z
    trace_stage(c, 1);
    return axis(c, c->tc_yi, c->d_T2, 1, 0, (long long)c->Ky * NCK, c->d_T1, 1, 0,
                (long long)c->ny * NCK, c->ny, NCK, c->Ky, c->nz, nullptr, c->d_kym, c->d_twy,
                c->ny, +1, done);
  }
  trace_stage(c, 1);
  return axis(c, c->tc_yi, c->d_ER, 1, 0, 0, c->d_T1, 1, 0, 0, c->ny, NCK, c->Ky, 1, nullptr,
              c->d_kym, c->d_twy, c->ny, +1, done);
}

int launch_iteration(rf_ctx* c) {
  const int* done = &c->d_status->done;
  trace_begin(c, c->launched_iters++);
  const bool fftm = c->opt.transform == RF_TRANSFORM_FFT;
  if (fftm && c->fft_colmode == kColFused) {
    // row pass, then forward y + Green operator + decision + inverse y in one kernel (the
    // inverse of the start coefficients runs once before the first update)
    trace_stage(c, 2);
    if (int e = launch_fft_row(c, done, false, 0)) return e;
    return launch_fft_colphase(c, done);
  }
  if (fftm && c->fft_colmode == kColWarp) {
    // as kColFused, the column phase on the warp-FFT column kernel
    trace_stage(c, 2);
    if (int e = launch_fft_row(c, done, false, 0)) return e;
    return launch_fft_colphase_warp(c, done);
  }
  if (fftm && c->fft_colmode == kColGreenInv) {
    // row pass, forward y, then the Green operator + decision inside the inverse y kernel
    trace_stage(c, 2);
    if (int e = launch_fft_row(c, done, false, 0)) return e;
    if (int e = fft_forward_stages(c, done)) return e;
    return launch_fft_green_inv(c, done);
  }
  if (fftm) {
    if (int e = fft_inverse_stages(c, done)) return e;
    trace_stage(c, 2);
    if (int e = launch_fft_row(c, done, false, 0)) return e;
    if (int e = fft_forward_stages(c, done)) return e;
    return launch_gamma_finalize(c, 1, done);
  }
  if (int e = inverse_stages(c, done)) return e;
  const bool tcm = c->opt.precision != RF_PREC_FP32;
  trace_stage(c, 2);
  if (tcm) {
    if (int e = launch_tc_row(c, done)) return e;
  } else {
    RowArgs ra = row_args(c, done);
    if (int e = row_dispatch(c, ra, false)) return e;
  }
  const int NCK = c->nc * c->Kx;
  const long long outstride = c->rect;
  // the tensor-core row kernel leaves one partial sum per 128-wide x slice
  const float2* fin = tcm ? reinterpret_cast<const float2*>(c->d_Tout) : c->d_T1p;
  const int fsplits = tcm ? c->tc_nXS : 1;
  const long long fstride = (long long)c->rows * NCK;
  trace_stage(c, 3);
  if (c->dim == 3) {
    if (int e = axis(c, c->tc_yf, fin, fsplits, fstride, (long long)c->ny * NCK, c->d_T2f, 1, 0,
                     (long long)c->Ky * NCK, c->Ky, NCK, c->ny, c->nz, c->d_kym, nullptr,
                     c->d_twy, c->ny, -1, done))
      return e;
    trace_stage(c, 4);
    if (int e = axis(c, c->tc_zf, c->d_T2f, 1, 0, 0, c->d_OUT, c->splitC, outstride, 0, c->Kz,
                     c->Ky * NCK, c->nz, 1, c->d_kzm, nullptr, c->d_twz, c->nz, -1, done))
      return e;
  } else {
    if (int e = axis(c, c->tc_yf, fin, fsplits, fstride, 0, c->d_OUT, c->splitB, outstride, 0,
                     c->Ky, NCK, c->ny, 1, c->d_kym, nullptr, c->d_twy, c->ny, -1, done))
      return e;
  }
  return launch_gamma_finalize(c, (c->dim == 3) ? c->splitC : c->splitB, done);
}

int launch_gamma_finalize(rf_ctx* c, int splits, const int* done) {
  GammaArgs g{};
  g.OUT = c->d_OUT;
  g.splits = splits;
  g.split_stride = c->rect;
  g.ER = c->d_ER;
  g.hidx = c->d_hidx;
  g.hn = c->d_hn;
  g.Kh = c->Kh;
  g.Kx = c->Kx;
  g.Ky = c->Ky;
  g.NC = c->nc;
  g.inv2mu0 = (float)(0.5 / c->mu0);
  g.cgam = (float)((c->lam0 + c->mu0) / (c->mu0 * (c->lam0 + 2.0 * c->mu0)));
  g.st = c->d_status;
  g.status = c->d_status;
  g.counter = c->d_counter;
  g.part = c->d_part;
  g.done = done;
  g.cond = c->while_cond;
  g.use_cond = c->capturing_while ? 1 : 0;
  const unsigned gb = (unsigned)((c->Kh + kGammaBlock - 1) / kGammaBlock);
  trace_stage(c, 5);
  const cudaError_t le =
      c->nc == 3 ? launch_pdl(k_gamma<3>, dim3(gb), dim3(kGammaBlock), 0, c->stream, g, (double)c->N)
                 : launch_pdl(k_gamma<6>, dim3(gb), dim3(kGammaBlock), 0, c->stream, g, (double)c->N);
  if (le != cudaSuccess) return cuda_fail(le, "gamma");
  int e = launch_check(c, "gamma");
  trace_end(c);
  return e;
}

int launch_final(rf_ctx* c, int commit) {
  trace_begin(c, -1);
  trace_stage(c, 7);
  const bool tr = c->tracing;
  c->tracing = false;   // the whole final pass is one stage
  if (c->opt.transform == RF_TRANSFORM_FFT && c->fft_colmode == kColPersistent) {
    // the persistent solve leaves the strain lines of the final coefficients in its layout
    const int ie = launch_persist_final(c, commit);
    c->tracing = tr;
    if (ie) return ie;
    k_reduce_sbar<<<1, 256, 0, c->stream>>>(c->d_sbar_part, c->d_viol_part, c->persist_G,
                                            1.0 / (double)c->N, c->d_sbar);
    int e = launch_check(c, "reduce_sbar");
    trace_end(c);
    return e;
  }
  if (c->opt.transform == RF_TRANSFORM_FFT) {
    int ie = fft_inverse_stages(c, nullptr);
    if (!ie) ie = launch_fft_row(c, nullptr, true, commit);
    c->tracing = tr;
    if (ie) return ie;
    k_reduce_sbar<<<1, 256, 0, c->stream>>>(c->d_sbar_part, c->d_viol_part, c->fft_blocks,
                                            1.0 / (double)c->N, c->d_sbar);
    int e = launch_check(c, "reduce_sbar");
    trace_end(c);
    return e;
  }
  int ie = inverse_stages(c, nullptr);
  c->tracing = tr;
  if (ie) return ie;
  RowArgs ra = row_args(c, nullptr);
  ra.eps_out = c->d_eps;
  ra.sig_out = c->d_sig;
  ra.alpha_out = c->d_alpha;
  ra.sbar_part = c->d_sbar_part;
  ra.viol_part = c->d_viol_part;
  ra.commit = commit;
  if (int e = row_dispatch(c, ra, true)) return e;
  k_reduce_sbar<<<1, 256, 0, c->stream>>>(c->d_sbar_part, c->d_viol_part, c->row_blocks,
                                          1.0 / (double)c->N, c->d_sbar);
  int e = launch_check(c, "reduce_sbar");
  trace_end(c);
  return e;
}

int launch_reset_er(rf_ctx* c, const double* ebar6, double mode_add) {
  // mode_add == 0: ER = 0 except the zero frequency = N ebar; otherwise add N * ebar6 there
  if (mode_add == 0.0) {
    cudaError_t e = cudaMemsetAsync(c->d_ER, 0, sizeof(float2) * c->rect, c->stream);
    if (e != cudaSuccess) return cuda_fail(e, "memset ER");
  }
  // zero frequency sits at kx index 0 and the indices of ky = 0, kz = 0 (host-computed base)
  k_zero_freq<<<1, 32, 0, c->stream>>>(c->d_ER, zero_base(c), c->nc, c->Kx, (double)c->N,
                                      ebar6[0], ebar6[1], ebar6[2], ebar6[3], ebar6[4], ebar6[5],
                                      mode_add == 0.0 ? 0 : 1);
  return launch_check(c, "zero_freq");
}

int launch_warm_project(rf_ctx* c, const float2* d_warm6, const double* eb) {
  const float inv2mu0 = (float)(0.5 / c->mu0);
  const float cg = (float)((c->lam0 + c->mu0) / (c->mu0 * (c->lam0 + 2.0 * c->mu0)));
  const unsigned gb = (unsigned)((c->Kh + 255) / 256);
  if (c->nc == 3)
    k_warm_project<3><<<gb, 256, 0, c->stream>>>(d_warm6, c->d_ER, c->d_hidx, c->d_hn, c->Kh,
                                                 c->Kx, c->Ky, (float)c->lam0, (float)c->mu0,
                                                 inv2mu0, cg, (double)c->N, eb[0], eb[1], eb[2],
                                                 eb[3], eb[4], eb[5]);
  else
    k_warm_project<6><<<gb, 256, 0, c->stream>>>(d_warm6, c->d_ER, c->d_hidx, c->d_hn, c->Kh,
                                                 c->Kx, c->Ky, (float)c->lam0, (float)c->mu0,
                                                 inv2mu0, cg, (double)c->N, eb[0], eb[1], eb[2],
                                                 eb[3], eb[4], eb[5]);
  return launch_check(c, "warm_project");
}

int launch_inverse(rf_ctx* c) { return inverse_stages(c, nullptr); }

// ------------------------------------------------------------------------------------------
// tracing
static cudaEvent_t take_event(rf_ctx* c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

// While a graph is being captured the events become event-record nodes of the graph (they are
// recorded on the device timeline at every replay) and belong to the graph.
static void record_event(rf_ctx* c, cudaEvent_t e) {
  if (c->capturing) cudaEventRecordWithFlags(e, c->stream, cudaEventRecordExternal);
  else cudaEventRecord(e, c->stream);
}

void trace_begin(rf_ctx* c, long long idx) {
  if (!c->tracing) return;
  auto& list = c->capturing ? c->graph_traces : c->pending;
  list.push_back(rf_ctx::TraceIter{});
  c->cur = &list.back();
  c->cur->idx = idx;
  c->cur->n = 0;
}

void trace_stage(rf_ctx* c, int stage) {
  if (!c->tracing || !c->cur || c->cur->n >= 8) return;
  cudaEvent_t e = take_event(c);
  record_event(c, e);
  c->cur->stage[c->cur->n] = stage;
  c->cur->ev[c->cur->n] = e;
  c->cur->n += 1;
}

void trace_end(rf_ctx* c) {
  if (!c->tracing || !c->cur) return;
  cudaEvent_t e = take_event(c);
  record_event(c, e);
  c->cur->ev[c->cur->n] = e;
  c->cur = nullptr;
}

// after a replay of graph g (first update index `base`) and a stream synchronize
void trace_collect_graph(rf_ctx* c, const rf_ctx::GraphEntry& g, long long base,
                         long long real_iters) {
  for (size_t i = 0; i < g.trace_first.size(); ++i) {
    if (base + (long long)i >= real_iters) break;
    const rf_ctx::TraceIter& t = c->graph_traces[g.trace_first[i]];
    for (int s = 0; s < t.n; ++s) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, t.ev[s], t.ev[s + 1]) == cudaSuccess) {
        c->stage_ms[t.stage[s]] += ms;
        c->stage_n[t.stage[s]] += 1;
      }
    }
  }
}

int trace_collect(rf_ctx* c, long long real_iters) {
  // call after a stream synchronize: accumulate updates with index < real_iters, and finals
  for (auto& t : c->pending) {
    const bool real = (t.idx < 0) || (t.idx < real_iters);
    for (int i = 0; i < t.n; ++i) {
      if (real) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.ev[i], t.ev[i + 1]) == cudaSuccess) {
          c->stage_ms[t.stage[i]] += ms;
          c->stage_n[t.stage[i]] += 1;
        }
      }
      c->ev_pool.push_back(t.ev[i]);
    }
    if (t.n > 0) c->ev_pool.push_back(t.ev[t.n]);
  }
  c->pending.clear();
  c->cur = nullptr;
  return RF_OK;
}

}  // namespace rfk
