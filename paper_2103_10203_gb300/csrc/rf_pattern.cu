// Sampling patterns (reduced sets of frequencies), computed on the GPU.
//
// Adapted pattern (Sec. 4.2; 3D as in Sec. 5.3): the phase map becomes the step function g
// (1 on the inclusion phase), g is transformed in FP64 axis by axis, and the amplitudes |g^|
// rank the conjugate pairs (k, -k). Ranking key (smaller first): quantised amplitude
// round(|g^| / |g^(0)| * 2^30) descending, |k|^2 ascending, signed linear index ascending.
// Pairs are taken whole until at least k_target frequencies are held; the selection threshold
// is found by radix passes over weighted histograms of the key (device-side counting).
// Radial pattern (Sec. 4.1): L equiangular rasterised lines; the same selection machinery
// ranks pairs by (not on a line, |k|^2, index).
#include <algorithm>
#include <climits>
#include <cmath>
#include <mutex>
#include <vector>

#include "rf_internal.cuh"

namespace rfk {

namespace {

struct Grid3 {
  int nx, ny, nz;
  long long N;
  int hx, hy, hz;
};

__device__ __forceinline__ int sgn_index(int i, int n) { return i <= n / 2 ? i : i - n; }
__device__ __forceinline__ int wrap(int k, int n) {
  int r = k % n;
  return r < 0 ? r + n : r;
}
__device__ __forceinline__ long long signed_lin(int kx, int ky, int kz, const Grid3& g) {
  return ((long long)(kz + g.hz) * g.ny + (ky + g.hy)) * g.nx + (kx + g.hx);
}

__global__ void k_table_f64(double2* t, int L) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L) {
    double s, c;
    sincospi(2.0 * (double)i / (double)L, &s, &c);
    t[i] = make_double2(c, -s);   // exp(-2 pi i t / L)
  }
}

// out[row][kx] = sum_x g(row, x) exp(-2 pi i kx x / nx), one block per row
__global__ void k_g_rows(const uint8_t* pm, int incl, int nx, const double2* tab, double2* out) {
  extern __shared__ __align__(16) unsigned char sm[];
  double2* t = reinterpret_cast<double2*>(sm);
  float* gr = reinterpret_cast<float*>(t + nx);
  const long long row = blockIdx.x;
  for (int i = threadIdx.x; i < nx; i += blockDim.x) {
    t[i] = tab[i];
    gr[i] = pm[row * nx + i] == incl ? 1.f : 0.f;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nx; k += blockDim.x) {
    double re = 0.0, im = 0.0;
    int m = 0;
    for (int x = 0; x < nx; ++x) {
      if (gr[x] != 0.f) {
        re += t[m].x;
        im += t[m].y;
      }
      m += k;
      if (m >= nx) m -= nx;
    }
    out[row * nx + k] = make_double2(re, im);
  }
}

// out[b][m][n] = sum_k exp(-2 pi i m k / L) in[b][k][n]; 4 m per thread, lanes over n
__global__ void k_axis_f64(const double2* in, double2* out, int L, int N, long long bstride,
                           const double2* tab) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  const int m0 = blockIdx.y * 4;
  const long long b = blockIdx.z;
  if (n >= N) return;
  double ar[4] = {0, 0, 0, 0}, ai[4] = {0, 0, 0, 0};
  const double2* ib = in + b * bstride;
  for (int k = 0; k < L; ++k) {
    const double2 v = ib[(long long)k * N + n];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int m = m0 + i;
      if (m < L) {
        const double2 w = tab[(int)(((long long)m * k) % L)];
        ar[i] += w.x * v.x - w.y * v.y;
        ai[i] += w.x * v.y + w.y * v.x;
      }
    }
  }
  double2* ob = out + b * bstride;
#pragma unroll
  for (int i = 0; i < 4; ++i)
    if (m0 + i < L) ob[(long long)(m0 + i) * N + n] = make_double2(ar[i], ai[i]);
}

// FP64 Stockham FFTs (forward, exp(-2 pi i m n / L)) for lengths L = 2^b or 3 * 2^b: radix-4
// stages, one radix-2 stage, then one radix-3 stage. A stage of radix R and sub-transform size
// Ns reads element j + r L / R, multiplies it by exp(-2 pi i r k / (R Ns)) with k = j mod Ns
// (tab[t] = exp(-2 pi i t / L)), takes the R-point DFT and writes output q to
// (j / Ns) R Ns + k + q Ns. The zero frequency only meets the exact factor 1, so for 0/1 data it
// is an exact sum. C sequences of length L lie back to back in both shared buffers; returns
// the buffer holding the result. The whole block calls it.
__device__ __forceinline__ double2 cm64(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 add64(double2 a, double2 b) {
  return make_double2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ double2 sub64(double2 a, double2 b) {
  return make_double2(a.x - b.x, a.y - b.y);
}

__device__ double2* fft64_block(double2* in, double2* out, const double2* tab, int L, int C) {
  const int p2 = (L % 3 == 0) ? L / 3 : L;
  int Ns = 1;
  auto swap = [&] {
    __syncthreads();
    double2* t = in;
    in = out;
    out = t;
  };
  while (Ns * 4 <= p2) {
    const int q = L / 4, step = L / (4 * Ns);
    for (int u = threadIdx.x; u < C * q; u += blockDim.x) {
      const int p = u / q, j = u - p * q, k = j % Ns;
      const double2* src = in + (long long)p * L + j;
      double2 a0 = src[0], a1 = src[q], a2 = src[2 * q], a3 = src[3 * q];
      if (Ns > 1) {
        a1 = cm64(a1, tab[k * step]);
        a2 = cm64(a2, tab[2 * k * step]);
        a3 = cm64(a3, tab[3 * k * step]);
      }
      const double2 s02 = add64(a0, a2), d02 = sub64(a0, a2);
      const double2 s13 = add64(a1, a3), d13 = sub64(a1, a3);
      const double2 md13 = make_double2(d13.y, -d13.x);   // -i (a1 - a3)
      double2* dst = out + (long long)p * L + (j / Ns) * 4 * Ns + k;
      dst[0] = add64(s02, s13);
      dst[Ns] = add64(d02, md13);
      dst[2 * Ns] = sub64(s02, s13);
      dst[3 * Ns] = sub64(d02, md13);
    }
    swap();
    Ns *= 4;
  }
  if (Ns * 2 <= p2) {
    const int q = L / 2, step = L / (2 * Ns);
    for (int u = threadIdx.x; u < C * q; u += blockDim.x) {
      const int p = u / q, j = u - p * q, k = j % Ns;
      const double2* src = in + (long long)p * L + j;
      double2 a0 = src[0], a1 = src[q];
      if (Ns > 1) a1 = cm64(a1, tab[k * step]);
      double2* dst = out + (long long)p * L + (j / Ns) * 2 * Ns + k;
      dst[0] = add64(a0, a1);
      dst[Ns] = sub64(a0, a1);
    }
    swap();
    Ns *= 2;
  }
  if (p2 != L) {   // Ns = L / 3: j = k < Ns, outputs j, j + Ns, j + 2 Ns
    const double h = 0.86602540378443864676;   // sqrt(3) / 2
    for (int u = threadIdx.x; u < C * Ns; u += blockDim.x) {
      const int p = u / Ns, j = u - p * Ns;
      const double2* src = in + (long long)p * L + j;
      double2 a0 = src[0], a1 = src[Ns], a2 = src[2 * Ns];
      if (Ns > 1) {
        a1 = cm64(a1, tab[j]);
        a2 = cm64(a2, tab[2 * j]);
      }
      // X0 = a0 + s, X1,2 = a0 - s / 2 -+ i sqrt(3)/2 (a1 - a2)
      const double2 sm = add64(a1, a2), d = sub64(a1, a2);
      const double2 m = make_double2(a0.x - 0.5 * sm.x, a0.y - 0.5 * sm.y);
      double2* dst = out + (long long)p * L + j;
      dst[0] = add64(a0, sm);
      dst[Ns] = make_double2(m.x + h * d.y, m.y - h * d.x);
      dst[2 * Ns] = make_double2(m.x - h * d.y, m.y + h * d.x);
    }
    swap();
  }
  return in;
}

constexpr size_t kFft64Smem = 96 * 1024;

bool fft64_length(int L) {
  const int p2 = (L % 3 == 0) ? L / 3 : L;
  return L >= 1 && (p2 & (p2 - 1)) == 0 && 2 * (size_t)L * sizeof(double2) <= kFft64Smem;
}

// sequences per block for length L within the shared-memory budget
int fft64_lines(int L, int cap) {
  return std::max(1, std::min(cap, (int)(kFft64Smem / (2 * (size_t)L * sizeof(double2)))));
}

// out[row][kx] = FFT along x of the indicator of `incl` on C rows per block
__global__ void k_g_rows_fft(const uint8_t* pm, int incl, int nx, long long rows, int C,
                             const double2* tab, double2* out) {
  extern __shared__ __align__(16) unsigned char sm[];
  double2* b0 = reinterpret_cast<double2*>(sm);
  double2* b1 = b0 + (size_t)C * nx;
  const long long row0 = (long long)blockIdx.x * C;
  for (int i = threadIdx.x; i < C * nx; i += blockDim.x) {
    const long long g = row0 * nx + i;
    b0[i] = make_double2((row0 + i / nx < rows && pm[g] == incl) ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  const double2* z = fft64_block(b0, b1, tab, nx, C);
  for (int i = threadIdx.x; i < C * nx; i += blockDim.x)
    if (row0 + i / nx < rows) out[row0 * nx + i] = z[i];
}

// out[b][m][n] = sum_k exp(-2 pi i m k / L) in[b][k][n] by FFT, C columns n per block
__global__ void k_cols_fft64(const double2* in, double2* out, int L, int ncols, long long bstride,
                             int C, const double2* tab) {
  extern __shared__ __align__(16) unsigned char sm[];
  double2* b0 = reinterpret_cast<double2*>(sm);
  double2* b1 = b0 + (size_t)C * L;
  const int col0 = blockIdx.x * C;
  const double2* ib = in + blockIdx.y * bstride;
  double2* ob = out + blockIdx.y * bstride;
  for (int i = threadIdx.x; i < C * L; i += blockDim.x) {
    const int y = i / C, c = i - y * C, col = col0 + c;
    b0[c * L + y] = col < ncols ? ib[(long long)y * ncols + col] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const double2* z = fft64_block(b0, b1, tab, L, C);
  for (int i = threadIdx.x; i < C * L; i += blockDim.x) {
    const int y = i / C, c = i - y * C, col = col0 + c;
    if (col < ncols) ob[(long long)y * ncols + col] = z[c * L + y];
  }
}

// keys at canonical pair members (array order [z][y][x]); others get ~0
__global__ void k_keys(const double2* G, const uint8_t* mark, Grid3 g, unsigned long long* key,
                       int* lin, int* size) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // |g^(0)| = number of inclusion voxels, exact in FP64 (a sum of ones)
  const double amax = G ? G[0].x : 0.0;
  if (i >= g.N) return;
  const int ix = (int)(i % g.nx);
  const int iy = (int)((i / g.nx) % g.ny);
  const int iz = (int)(i / ((long long)g.nx * g.ny));
  const int kx = sgn_index(ix, g.nx), ky = sgn_index(iy, g.ny), kz = sgn_index(iz, g.nz);
  const int cx = sgn_index(wrap(-kx, g.nx), g.nx);
  const int cy = sgn_index(wrap(-ky, g.ny), g.ny);
  const int cz = sgn_index(wrap(-kz, g.nz), g.nz);
  const long long l = signed_lin(kx, ky, kz, g);
  const long long lc = signed_lin(cx, cy, cz, g);
  lin[i] = (int)l;
  if (l > lc) {
    key[i] = ~0ull;
    size[i] = 0;
    return;
  }
  size[i] = (l == lc) ? 1 : 2;
  const unsigned long long k2 =
      (unsigned long long)((long long)kx * kx + (long long)ky * ky + (long long)kz * kz);
  unsigned long long primary;
  if (mark) {
    primary = mark[i] ? 0ull : 1ull;
  } else {
    long long aq = 0;
    if (amax > 0.0) {
      const double a = hypot(G[i].x, G[i].y);
      aq = llrint(a / amax * 1073741824.0);
    }
    long long p = 1073741824LL - aq;
    primary = (unsigned long long)(p < 0 ? 0 : p);
  }
  key[i] = (primary << 33) | k2;
}

__global__ void k_count_le(const unsigned long long* key, const int* lin, const int* size,
                           long long N, unsigned long long vhi, int vlin,
                           unsigned long long* out) {
  __shared__ unsigned long long sh[256];
  unsigned long long s = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long k = key[i];
    if (k != ~0ull && (k < vhi || (k == vhi && lin[i] <= vlin))) s += (unsigned long long)size[i];
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && sh[0]) atomicAdd(out, sh[0]);
}

// Weighted histogram for the radix search of the threshold: entries with a valid key and
// (phase 0) key - base in [0, 256 << shift), or (phase 1) key == vhi and lin - base in
// [0, 256 << shift), add their pair size to bucket ((value - base) >> shift).
__global__ void k_key_hist(const unsigned long long* key, const int* lin, const int* size,
                           long long N, int phase, unsigned long long vhi,
                           unsigned long long base, int shift, unsigned long long* hist) {
  __shared__ unsigned long long sh[256];
  sh[threadIdx.x] = 0;
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long k = key[i];
    if (k == ~0ull) continue;
    unsigned long long v;
    if (phase == 0) {
      v = k;
    } else {
      if (k != vhi) continue;
      v = (unsigned long long)(unsigned)lin[i];
    }
    if (v < base) continue;
    const unsigned long long b = (v - base) >> shift;
    if (b < 256) atomicAdd(&sh[b], (unsigned long long)size[i]);
  }
  __syncthreads();
  if (sh[threadIdx.x]) atomicAdd(&hist[threadIdx.x], sh[threadIdx.x]);
}

// flags in signed-linear order
__global__ void k_flags(const unsigned long long* key, const int* lin, Grid3 g,
                        unsigned long long thi, int tlin, int* flags) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.N) return;
  const int kx = (int)(s % g.nx) - g.hx;
  const int ky = (int)((s / g.nx) % g.ny) - g.hy;
  const int kz = (int)(s / ((long long)g.nx * g.ny)) - g.hz;
  const long long ia = ((long long)wrap(kz, g.nz) * g.ny + wrap(ky, g.ny)) * g.nx + wrap(kx, g.nx);
  const long long ic = ((long long)wrap(-kz, g.nz) * g.ny + wrap(-ky, g.ny)) * g.nx +
                       wrap(-kx, g.nx);
  const long long canon = (key[ia] != ~0ull) ? ia : ic;
  const unsigned long long k = key[canon];
  flags[s] = (k < thi || (k == thi && lin[canon] <= tlin)) ? 1 : 0;
}

// three-pass exclusive scan (block totals, scan of totals, write)
__global__ void k_block_totals(const int* flags, long long N, int* tot) {
  __shared__ int sh[1024];
  const long long i = blockIdx.x * 1024LL + threadIdx.x;
  sh[threadIdx.x] = (i < N) ? flags[i] : 0;
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) tot[blockIdx.x] = sh[0];
}

__global__ void k_scan_totals(int* tot, int nb) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    int run = 0;
    for (int b = 0; b < nb; ++b) {
      int t = tot[b];
      tot[b] = run;
      run += t;
    }
    tot[nb] = run;
  }
}

__global__ void k_compact(const int* flags, long long N, const int* tot, Grid3 g, int* out,
                          long long cap) {
  __shared__ int sh[1024];
  const long long i = blockIdx.x * 1024LL + threadIdx.x;
  const int f = (i < N) ? flags[i] : 0;
  sh[threadIdx.x] = f;
  __syncthreads();
  // Hillis-Steele inclusive scan inside the block
  for (int o = 1; o < 1024; o <<= 1) {
    int v = (threadIdx.x >= o) ? sh[threadIdx.x - o] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  if (f) {
    const long long pos = (long long)tot[blockIdx.x] + sh[threadIdx.x] - 1;
    if (pos < cap) {
      out[3 * pos + 0] = (int)(i % g.nx) - g.hx;
      out[3 * pos + 1] = (int)((i / g.nx) % g.ny) - g.hy;
      out[3 * pos + 2] = (int)(i / ((long long)g.nx * g.ny)) - g.hz;
    }
  }
}

__global__ void k_radial_mark(int L, int nx, int ny, uint8_t* mark) {
  const int l = blockIdx.y;
  const int ti = blockIdx.x * blockDim.x + threadIdx.x;
  const double th = M_PI * (double)l / (double)L;
  const double c = cos(th), s = sin(th);
  long long x, y;
  if (fabs(c) >= fabs(s)) {
    const int t = ti - nx / 2;
    if (t > nx / 2) return;
    const double v = (double)t * (s / c);
    x = t;
    y = (long long)copysign(floor(fabs(v) + 0.5), v);
  } else {
    const int t = ti - ny / 2;
    if (t > ny / 2) return;
    const double v = (double)t * (c / s);
    y = t;
    x = (long long)copysign(floor(fabs(v) + 0.5), v);
  }
  if (llabs(x) <= nx / 2 && llabs(y) <= ny / 2) {
    const int ix = (int)(((x % nx) + nx) % nx), iy = (int)(((y % ny) + ny) % ny);
    mark[(long long)iy * nx + ix] = 1;
  }
}

__global__ void k_count_u8(const uint8_t* m, long long N, unsigned long long* out) {
  __shared__ unsigned long long sh[256];
  unsigned long long s = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x)
    s += m[i] ? 1 : 0;
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && sh[0]) atomicAdd(out, sh[0]);
}

// RAII scratch
struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  T* get(size_t n) {
    void* p = nullptr;
    if (cudaMalloc(&p, n * sizeof(T) + 16) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
};

int check(cudaError_t e, const char* what) { return e == cudaSuccess ? RF_OK : cuda_fail(e, what); }

int validate_grid(const rf_grid* g, Grid3& out) {
  if (!g || (g->dim != 2 && g->dim != 3)) {
    set_error("grid: dim must be 2 or 3");
    return RF_ERR_INVALID;
  }
  for (int j = 0; j < 3; ++j)
    if (g->n[j] < 1 || g->n[j] > 4096) {
      set_error("grid: sizes must be in [1, 4096]");
      return RF_ERR_INVALID;
    }
  if (g->dim == 2 && g->n[2] != 1) {
    set_error("grid: Nz must be 1 in 2D");
    return RF_ERR_INVALID;
  }
  out.nx = g->n[0];
  out.ny = g->n[1];
  out.nz = g->n[2];
  out.N = (long long)out.nx * out.ny * out.nz;
  if (out.N >= (1LL << 31)) {
    set_error("grid: too many voxels");
    return RF_ERR_INVALID;
  }
  out.hx = (out.nx - 1) / 2;
  out.hy = (out.ny - 1) / 2;
  out.hz = (out.nz - 1) / 2;
  return RF_OK;
}

// Selection of the pattern from keys already in `key/lin/size`, shared by every entry point.
// The caller provides the scratch: device d_cnt [1], d_hist [256], flags [N], tot [N/1024 + 2]
// and d_out [3 K] (K becomes known after the threshold search, so d_out is asked for through
// `out_buf`), and host h_cnt [1], h_hist [256] (pinned or pageable).
struct SelectScratch {
  unsigned long long* d_cnt;
  unsigned long long* d_hist;
  int* flags;
  int* tot;
  unsigned long long* h_cnt;
  unsigned long long* h_hist;
};

// Threshold of the selection: the smallest (key, lin) in the total order whose weighted count of
// entries at or below it reaches k_target, found by radix passes of 8 bits from the top (one
// weighted histogram and one host read each), first over the whole 64-bit key, then over lin
// among the entries with that key. *K receives the number of frequencies at or below it.
int select_threshold(const Grid3& g, const unsigned long long* key, const int* lin,
                     const int* size, long long k_target, cudaStream_t s,
                     const SelectScratch& ss, unsigned long long* thi_out, int* tlin_out,
                     long long* K) {
  auto count = [&](unsigned long long vhi, int vlin, unsigned long long& res) -> int {
    if (int e = check(cudaMemsetAsync(ss.d_cnt, 0, sizeof(unsigned long long), s), "memset"))
      return e;
    k_count_le<<<304, 256, 0, s>>>(key, lin, size, g.N, vhi, vlin, ss.d_cnt);
    if (int e = check(cudaGetLastError(), "count_le")) return e;
    if (int e = check(cudaMemcpyAsync(ss.h_cnt, ss.d_cnt, sizeof(unsigned long long),
                                      cudaMemcpyDeviceToHost, s), "copy count"))
      return e;
    if (int e = check(cudaStreamSynchronize(s), "sync count")) return e;
    res = *ss.h_cnt;
    return RF_OK;
  };
  unsigned long long total = 0;
  if (int e = count(~0ull - 1, INT_MAX, total)) return e;
  if ((long long)total < k_target) {
    set_error("pattern: k_target exceeds the number of frequencies");
    return RF_ERR_INVALID;
  }
  unsigned long long below = 0;   // weighted count of entries strictly below the current base
  auto radix = [&](int phase, unsigned long long vhi, int top_shift,
                   unsigned long long& base) -> int {
    base = 0;
    for (int shift = top_shift; shift >= 0; shift -= 8) {
      if (int e = check(cudaMemsetAsync(ss.d_hist, 0, 256 * sizeof(unsigned long long), s),
                        "memset"))
        return e;
      k_key_hist<<<304, 256, 0, s>>>(key, lin, size, g.N, phase, vhi, base, shift, ss.d_hist);
      if (int e = check(cudaGetLastError(), "key histogram")) return e;
      if (int e = check(cudaMemcpyAsync(ss.h_hist, ss.d_hist, 256 * sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, s), "copy histogram"))
        return e;
      if (int e = check(cudaStreamSynchronize(s), "sync histogram")) return e;
      int b = 0;
      while (b < 255 && (long long)(below + ss.h_hist[b]) < k_target) below += ss.h_hist[b++];
      base += (unsigned long long)b << shift;
    }
    return RF_OK;
  };
  unsigned long long thi = 0, tl = 0;
  if (int e = radix(0, 0, 56, thi)) return e;   // bits 63..0 of the key
  // `below` now counts the entries with key < thi
  if (int e = radix(1, thi, 24, tl)) return e;  // bits 31..0 of lin
  unsigned long long k = 0;
  if (int e = count(thi, (int)tl, k)) return e;
  if ((long long)k < k_target) {
    set_error("pattern: threshold search ended below k_target");
    return RF_ERR_INVALID;
  }
  *thi_out = thi;
  *tlin_out = (int)tl;
  *K = (long long)k;
  return RF_OK;
}

// Flags of the selected frequencies in signed-linear order, their compaction into d_out [3 K]
// and the copy to the host.
int compact_selection(const Grid3& g, const unsigned long long* key, const int* lin,
                      unsigned long long thi, int tlin, long long K, int* d_out,
                      int32_t* out_host, cudaStream_t s, const SelectScratch& ss) {
  const long long nb = (g.N + 1023) / 1024;
  k_flags<<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(key, lin, g, thi, tlin, ss.flags);
  k_block_totals<<<(unsigned)nb, 1024, 0, s>>>(ss.flags, g.N, ss.tot);
  k_scan_totals<<<1, 32, 0, s>>>(ss.tot, (int)nb);
  k_compact<<<(unsigned)nb, 1024, 0, s>>>(ss.flags, g.N, ss.tot, g, d_out, K);
  if (int e = check(cudaGetLastError(), "compact")) return e;
  if (int e = check(cudaMemcpyAsync(out_host, d_out, sizeof(int) * 3 * K, cudaMemcpyDeviceToHost,
                                    s), "copy pattern"))
    return e;
  return check(cudaStreamSynchronize(s), "sync pattern");
}

// Selection with scratch from cudaMalloc / cudaMallocHost (the allocating entry points).
int select_and_compact(const Grid3& g, unsigned long long* key, int* lin, int* size,
                       long long k_target, int32_t* out_host, long long cap, long long* K_out,
                       cudaStream_t s, Scratch& sc) {
  SelectScratch ss{};
  ss.d_cnt = sc.get<unsigned long long>(1);
  ss.d_hist = sc.get<unsigned long long>(256);
  ss.flags = sc.get<int>(g.N);
  ss.tot = sc.get<int>((g.N + 1023) / 1024 + 2);
  if (!ss.d_cnt || !ss.d_hist || !ss.flags || !ss.tot) {
    set_error("pattern: out of device memory");
    return RF_ERR_OOM;
  }
  if (int e = check(cudaMallocHost(&ss.h_cnt, sizeof(unsigned long long)), "pinned")) return e;
  struct PinFree {
    void* p;
    ~PinFree() {
      if (p) cudaFreeHost(p);
    }
  } pf{ss.h_cnt};
  if (int e = check(cudaMallocHost(&ss.h_hist, 256 * sizeof(unsigned long long)), "pinned"))
    return e;
  PinFree pf2{ss.h_hist};
  unsigned long long thi = 0;
  int tlin = 0;
  long long K = 0;
  if (int e = select_threshold(g, key, lin, size, k_target, s, ss, &thi, &tlin, &K)) return e;
  *K_out = K;
  if (K > cap) {
    set_error("pattern: output capacity too small");
    return RF_ERR_INVALID;
  }
  int* d_out = sc.get<int>(3 * (K > 0 ? K : 1));
  if (!d_out) {
    set_error("pattern: out of device memory");
    return RF_ERR_OOM;
  }
  return compact_selection(g, key, lin, thi, tlin, K, d_out, out_host, s, ss);
}

}  // namespace

// DFT of the inclusion indicator along x, y and z (FP64) from the device phase map: FFTs for
// sides 2^b and 3 * 2^b, dense DFTs (exact table sums along x) otherwise. Uses A and B
// ([N] each) and the tables tx, ty, tz ([side] each); *G receives the buffer holding g^.
int indicator_transform(const Grid3& g, const uint8_t* d_pm, int incl, double2* A, double2* B,
                        double2* tx, double2* ty, double2* tz, double2** G, cudaStream_t s) {
  k_table_f64<<<(g.nx + 255) / 256, 256, 0, s>>>(tx, g.nx);
  k_table_f64<<<(g.ny + 255) / 256, 256, 0, s>>>(ty, g.ny);
  k_table_f64<<<(g.nz + 255) / 256, 256, 0, s>>>(tz, g.nz);
  const long long rows = g.N / g.nx;
  if (fft64_length(g.nx)) {
    const int C = fft64_lines(g.nx, 16);
    if (int e = check(cudaFuncSetAttribute(k_g_rows_fft, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)kFft64Smem), "pattern: smem attribute"))
      return e;
    k_g_rows_fft<<<(unsigned)((rows + C - 1) / C), 256, 2 * (size_t)C * g.nx * sizeof(double2), s>>>(
        d_pm, incl, g.nx, rows, C, tx, A);
  } else {
    const size_t smem = (size_t)g.nx * (sizeof(double2) + sizeof(float));
    if (int e = check(cudaFuncSetAttribute(k_g_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           100 * 1024), "pattern: smem attribute"))
      return e;
    k_g_rows<<<(unsigned)rows, 256, smem, s>>>(d_pm, incl, g.nx, tx, A);
  }
  if (int e = check(cudaGetLastError(), "g rows")) return e;
  if (int e = check(cudaFuncSetAttribute(k_cols_fft64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFft64Smem), "pattern: smem attribute"))
    return e;
  // along y: batch z, k = y, n = kx
  if (fft64_length(g.ny)) {
    const int C = fft64_lines(g.ny, 8);
    dim3 grd((g.nx + C - 1) / C, g.nz);
    k_cols_fft64<<<grd, 256, 2 * (size_t)C * g.ny * sizeof(double2), s>>>(
        A, B, g.ny, g.nx, (long long)g.ny * g.nx, C, ty);
  } else {
    dim3 grd((g.nx + 127) / 128, (g.ny + 3) / 4, g.nz);
    k_axis_f64<<<grd, 128, 0, s>>>(A, B, g.ny, g.nx, (long long)g.ny * g.nx, ty);
  }
  *G = B;
  if (g.nz > 1) {
    const int Nn = g.ny * g.nx;
    if (fft64_length(g.nz)) {
      const int C = fft64_lines(g.nz, 8);
      dim3 grd((Nn + C - 1) / C, 1);
      k_cols_fft64<<<grd, 256, 2 * (size_t)C * g.nz * sizeof(double2), s>>>(B, A, g.nz, Nn, 0, C,
                                                                             tz);
    } else {
      dim3 grd((Nn + 127) / 128, (g.nz + 3) / 4, 1);
      k_axis_f64<<<grd, 128, 0, s>>>(B, A, g.nz, Nn, 0, tz);
    }
    *G = A;
  }
  return check(cudaGetLastError(), "g axes");
}

int pattern_adapted(const rf_grid* grid, const uint8_t* pm_host, int incl, long long k_target,
                    int32_t* out, long long cap, long long* K_out, cudaStream_t s) {
  Grid3 g;
  if (int e = validate_grid(grid, g)) return e;
  if (!pm_host || !out || !K_out || k_target < 1 || k_target > g.N) {
    set_error("pattern_adapted: invalid arguments");
    return RF_ERR_INVALID;
  }
  Scratch sc;
  uint8_t* d_pm = sc.get<uint8_t>(g.N);
  double2* A = sc.get<double2>(g.N);
  double2* B = sc.get<double2>(g.N);
  double2* tx = sc.get<double2>(g.nx);
  double2* ty = sc.get<double2>(g.ny);
  double2* tz = sc.get<double2>(g.nz);
  unsigned long long* key = sc.get<unsigned long long>(g.N);
  int* lin = sc.get<int>(g.N);
  int* size = sc.get<int>(g.N);
  if (!d_pm || !A || !B || !tx || !ty || !tz || !key || !lin || !size) {
    set_error("pattern_adapted: out of device memory");
    return RF_ERR_OOM;
  }
  if (int e = check(cudaMemcpyAsync(d_pm, pm_host, g.N, cudaMemcpyHostToDevice, s), "upload"))
    return e;
  double2* G = nullptr;
  if (int e = indicator_transform(g, d_pm, incl, A, B, tx, ty, tz, &G, s)) return e;
  k_keys<<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(G, nullptr, g, key, lin, size);
  if (int e = check(cudaGetLastError(), "keys")) return e;
  return select_and_compact(g, key, lin, size, k_target, out, cap, K_out, s, sc);
}

int pattern_radial(const rf_grid* grid, long long k_target, int32_t* out, long long cap,
                   long long* K_out, cudaStream_t s) {
  Grid3 g;
  if (int e = validate_grid(grid, g)) return e;
  if (grid->dim != 2) {
    set_error("pattern_radial: 2D only");
    return RF_ERR_INVALID;
  }
  if (!out || !K_out || k_target < 1 || k_target > g.N) {
    set_error("pattern_radial: invalid arguments");
    return RF_ERR_INVALID;
  }
  Scratch sc;
  uint8_t* mark = sc.get<uint8_t>(g.N);
  unsigned long long* d_cnt = sc.get<unsigned long long>(1);
  unsigned long long* key = sc.get<unsigned long long>(g.N);
  int* lin = sc.get<int>(g.N);
  int* size = sc.get<int>(g.N);
  if (!mark || !d_cnt || !key || !lin || !size) {
    set_error("pattern_radial: out of device memory");
    return RF_ERR_OOM;
  }
  const int maxL = 4 * (g.nx > g.ny ? g.nx : g.ny);
  const int tcount = (g.nx > g.ny ? g.nx : g.ny) + 1;
  unsigned long long cnt = 0;
  int L = 1;
  for (; L <= maxL; ++L) {
    if (int e = check(cudaMemsetAsync(mark, 0, g.N, s), "memset mark")) return e;
    dim3 grd((tcount + 127) / 128, L);
    k_radial_mark<<<grd, 128, 0, s>>>(L, g.nx, g.ny, mark);
    if (int e = check(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned long long), s), "memset")) return e;
    k_count_u8<<<304, 256, 0, s>>>(mark, g.N, d_cnt);
    if (int e = check(cudaGetLastError(), "radial")) return e;
    if (int e = check(cudaMemcpyAsync(&cnt, d_cnt, sizeof(cnt), cudaMemcpyDeviceToHost, s), "cp"))
      return e;
    if (int e = check(cudaStreamSynchronize(s), "sync")) return e;
    if ((long long)cnt >= k_target) break;
  }
  if ((long long)cnt < k_target) {
    set_error("pattern_radial: k_target not reachable");
    return RF_ERR_INVALID;
  }
  k_keys<<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(nullptr, mark, g, key, lin, size);
  if (int e = check(cudaGetLastError(), "keys")) return e;
  return select_and_compact(g, key, lin, size, k_target, out, cap, K_out, s, sc);
}

// ------------------------------------------------------------------------------------------
// Allocation-free variant of the adapted pattern.
//
// rf_pattern_adapted allocates its device scratch with cudaMalloc and frees it with cudaFree,
// and cudaFree synchronises the whole device. Callers that share the GPU with other streams
// they must not stall, or whose device memory is owned by another framework's pool allocator,
// cannot make those calls. rf_pattern_adapted_noalloc runs the same kernels with all scratch
// carved from the file-scope array below instead, for grids of at most kNoAllocMaxVoxels.
// Every GPU that loads this library holds the array until the process exits.
namespace {

constexpr long long kNoAllocMaxVoxels = 65536;     // e.g. 256 x 256 or 40 x 40 x 40
constexpr int kNoAllocMaxSide = 4096;
constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kNoAllocBytes =
    align256(kNoAllocMaxVoxels)                                   // phase map
    + 2 * align256(kNoAllocMaxVoxels * sizeof(double2))           // transform buffers
    + 3 * align256(kNoAllocMaxSide * sizeof(double2))             // twiddle tables
    + align256(kNoAllocMaxVoxels * sizeof(unsigned long long))    // keys
    + 3 * align256(kNoAllocMaxVoxels * sizeof(int))               // lin, size, flags
    + align256((kNoAllocMaxVoxels / 1024 + 2) * sizeof(int))      // scan totals
    + align256(sizeof(unsigned long long))                        // counter
    + align256(256 * sizeof(unsigned long long))                  // histogram
    + align256(3 * kNoAllocMaxVoxels * sizeof(int));              // output frequencies

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (looked up once per device).
int noalloc_scratch(unsigned char** out) {
  int dev = 0;
  if (int e = check(cudaGetDevice(&dev), "noalloc: cudaGetDevice")) return e;
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("rf_pattern_adapted_noalloc: device index out of range");
    return RF_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    if (int e = check(cudaGetSymbolAddress(&p, g_noalloc_scratch), "noalloc: scratch address"))
      return e;
    g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return RF_OK;
}

}  // namespace

int pattern_adapted_noalloc(const rf_grid* grid, const uint8_t* pm_host, int incl,
                            long long k_target, int32_t* out_host, long long cap,
                            long long* K_out, cudaStream_t s) {
  Grid3 g;
  if (int e = validate_grid(grid, g)) return e;
  if (!pm_host || !out_host || !K_out || k_target < 1 || k_target > g.N) {
    set_error("rf_pattern_adapted_noalloc: invalid arguments");
    return RF_ERR_INVALID;
  }
  if (g.N > kNoAllocMaxVoxels) {
    set_error("rf_pattern_adapted_noalloc: grid has more than 65536 voxels (the limit of its "
              "static scratch); use rf_pattern_adapted");
    return RF_ERR_INVALID;
  }
  unsigned char* base = nullptr;
  if (int e = noalloc_scratch(&base)) return e;
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += align256(bytes);
    return p;
  };
  uint8_t* d_pm = carve(kNoAllocMaxVoxels);
  double2* A = reinterpret_cast<double2*>(carve(kNoAllocMaxVoxels * sizeof(double2)));
  double2* B = reinterpret_cast<double2*>(carve(kNoAllocMaxVoxels * sizeof(double2)));
  double2* tx = reinterpret_cast<double2*>(carve(kNoAllocMaxSide * sizeof(double2)));
  double2* ty = reinterpret_cast<double2*>(carve(kNoAllocMaxSide * sizeof(double2)));
  double2* tz = reinterpret_cast<double2*>(carve(kNoAllocMaxSide * sizeof(double2)));
  auto* key = reinterpret_cast<unsigned long long*>(
      carve(kNoAllocMaxVoxels * sizeof(unsigned long long)));
  int* lin = reinterpret_cast<int*>(carve(kNoAllocMaxVoxels * sizeof(int)));
  int* size = reinterpret_cast<int*>(carve(kNoAllocMaxVoxels * sizeof(int)));
  int* flags = reinterpret_cast<int*>(carve(kNoAllocMaxVoxels * sizeof(int)));
  int* tot = reinterpret_cast<int*>(carve((kNoAllocMaxVoxels / 1024 + 2) * sizeof(int)));
  auto* d_cnt = reinterpret_cast<unsigned long long*>(carve(sizeof(unsigned long long)));
  auto* d_hist = reinterpret_cast<unsigned long long*>(carve(256 * sizeof(unsigned long long)));
  int* d_out = reinterpret_cast<int*>(carve(3 * kNoAllocMaxVoxels * sizeof(int)));

  // the transform and key kernels of rf_pattern_adapted
  if (int e = check(cudaMemcpyAsync(d_pm, pm_host, g.N, cudaMemcpyHostToDevice, s), "upload"))
    return e;
  double2* G = nullptr;
  if (int e = indicator_transform(g, d_pm, incl, A, B, tx, ty, tz, &G, s)) return e;
  k_keys<<<(unsigned)((g.N + 255) / 256), 256, 0, s>>>(G, nullptr, g, key, lin, size);
  if (int e = check(cudaGetLastError(), "noalloc: keys")) return e;

  // the selection code of rf_pattern_adapted, on carved scratch and host buffers on the stack
  // (pageable: the copies complete before each read); the counter and the histogram, the only
  // scratch that must start at zero, are cleared before every use
  unsigned long long h_cnt = 0, h_hist[256];
  const SelectScratch ss{d_cnt, d_hist, flags, tot, &h_cnt, h_hist};
  unsigned long long thi = 0;
  int tlin = 0;
  long long K = 0;
  if (int e = select_threshold(g, key, lin, size, k_target, s, ss, &thi, &tlin, &K)) return e;
  *K_out = K;
  if (K > cap) {
    set_error("pattern: output capacity too small");
    return RF_ERR_INVALID;
  }
  return compact_selection(g, key, lin, thi, tlin, K, d_out, out_host, s, ss);
}


}  // namespace rfk
