// Persistent 2D solve (FFT transform mode, FP32): the whole fixed-point iteration of one solve
// (Sec. 4, steps a-d, and the convergence decision of Sec. 3) in one cooperative launch.
//
// The grid holds one or two CTAs per SM, all co-resident (cooperative launch). Every update is
//   row phase     each CTA's grid rows: inverse FFT along x of the strain lines (Hermitian
//                 completion, two real lines per complex sequence), law and polarization per
//                 voxel, forward FFT along x, the pattern's kx columns of tau back to the lines
//   grid barrier
//   column phase  per kx of the pattern (one item, the NC line columns of that kx): forward FFT
//                 along y, the Green operator at that kx's pattern entries (new strain
//                 coefficients, squared-increment partial in FP64), inverse FFT along y of the
//                 new coefficients back to the strain lines
//   grid barrier
//   decision      every CTA sums the kx partials in the same fixed order, so all CTAs take the
//                 same decision (converged, capped, non-finite, diverged); CTA 0 records it.
// The start runs the inverse along y of the start coefficients first. A second kernel runs the
// final pass (fields, homogenised-stress partials, J2 commit) over the same row partition.
//
// The line transforms are stored column-major, T[(c Kx + j) Ny + y]: a kx item reads and writes
// whole contiguous columns, and a row CTA reads and writes runs of its consecutive rows. Data
// written by other CTAs during the launch is read through L2 (ld.global.cg), since L1 is not
// coherent across SMs. Grid barriers are bounded spin waits on an arrival counter and a
// generation word; a barrier that runs out sets the status's timeout flag and ends the launch.
#include <algorithm>
#include <vector>

#include "rf_fftcore.cuh"
#include "rf_internal.cuh"
#include "rf_law.cuh"

namespace rfk {

using fftc::fft_block;
using fftc::span_of;
using fftc::stage_len;
using fftc::sw;

struct PersistArgs {
  float2* T1;            // strain lines, [(c Kx + j) Ny + y]
  float2* T1p;           // polarization lines, same layout
  float2* ER;            // [Ky][NC][Kx]
  const uint8_t* phase;
  float* state;
  const int* kx;         // [Kx]
  const float2* twx;     // twiddle buffer of length Nx
  const float2* twy;     // twiddle buffer of length Ny
  const int* jptr;       // [Kx + 1] entries of each kx
  const int2* jent;      // per entry: rectangle row iy, frequency kind
  const float4* jn;      // per entry: unit wave vector, multiplicity
  const int* kym;        // [Ky] ky mod Ny
  int Nx, Ny, Kx;
  int rbase, rextra;     // CTA b holds rows [b rbase + min(b, rextra), ...), rbase (+1) rows
  int span_buf;          // entries of each of the two work buffers
  FastDiv dL, dKx, dNy;
  long long N;
  float invN;
  LawParams law;
  float inv2mu0, cgam;
  double Nd;
  Status* st;
  double* part;          // [Kx] squared-increment partial of each kx item
  double* sbar_part;     // [grid][6] (final pass)
  double* viol_part;     // [grid]
  unsigned* bar;         // [2] arrival count, generation
  long bar_limit;        // polls per barrier wait
  int commit;
  float* eps_out;
  float* sig_out;
  float* alpha_out;
  unsigned long long* trace;   // nullable: [trace_cap][3] global-timer stamps per update
  int trace_cap;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier over the whole (co-resident) grid; false if the wait ran out.
__device__ bool grid_sync(unsigned* bar, long limit, int* s_flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned gen = ld_acquire(bar + 1);
    __threadfence();
    if (atomicAdd(bar, 1u) == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long it = 0;
      while (ld_acquire(bar + 1) == gen) {
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

// Row phase of one CTA (see the top of the file). FINAL: fields, homogenised-stress partials,
// FP64 check of the return map and the commit, instead of the forward transform.
template <bool PLASTIC, bool FINAL, int kVox>
__device__ void p_row(const PersistArgs& a, const float2* tw, float2* b0, float2* b1,
                      const int* kxs, const DevPhase* phs, double* red) {
  constexpr int NC = 3, NS = 4;
  const int L = a.Nx, Ny = a.Ny, Kx = a.Kx;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int row0 = blockIdx.x * a.rbase + min((int)blockIdx.x, a.rextra);
  const int R = a.rbase + ((int)blockIdx.x < a.rextra ? 1 : 0);
  const int S = R * NC, P = (S + 1) / 2;
  const int span = span_of(P * L);
  for (int i = tid; i < span; i += nt) b0[i] = make_float2(0.f, 0.f);
  __syncthreads();
  // line coefficients: item u = q R + r with q = c Kx + j (R consecutive rows of one line column
  // are contiguous); line s = r NC + c is the real (s even) or imaginary (s odd) carrier of
  // sequence s / 2. The two carriers of a sequence can fall in different batches, so both add
  // into the zeroed buffer: per batch the real carriers first, then (after a barrier) the
  // imaginary ones, one writer per location in each pass. The batch loop's trip count is the
  // same for every thread.
  constexpr int kB = 8;
  const int nsc = S * Kx;
  for (int base = 0; base < nsc; base += kB * nt) {
    float2 t[kB];
    int sl[kB], jj[kB];
#pragma unroll
    for (int m = 0; m < kB; ++m) {
      const int u = base + tid + m * nt;
      sl[m] = -1;
      t[m] = make_float2(0.f, 0.f);
      if (u < nsc) {
        const int q = u / R, r = u - q * R;
        const int c = fdiv(q, a.dKx), j = q - c * Kx;
        t[m] = __ldcg(a.T1 + (long long)q * Ny + row0 + r);
        sl[m] = r * NC + c;
        jj[m] = j;
      }
    }
#pragma unroll
    for (int m = 0; m < kB; ++m) {
      if (sl[m] < 0 || (sl[m] & 1)) continue;
      const int k = kxs[jj[m]];
      const bool self = (k == 0) || (2 * k == L);
      float2 v = t[m];
      if (self) v.y = 0.f;
      const int zb0 = (sl[m] >> 1) * L;
      float2& zk = b0[sw(zb0 + k)];   // add v at k and conj(v) at L - k
      zk.x += v.x;
      zk.y += v.y;
      if (!self) {
        float2& zm = b0[sw(zb0 + L - k)];
        zm.x += v.x;
        zm.y -= v.y;
      }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < kB; ++m) {
      if (sl[m] < 0 || !(sl[m] & 1)) continue;
      const int k = kxs[jj[m]];
      const bool self = (k == 0) || (2 * k == L);
      float2 v = t[m];
      if (self) v.y = 0.f;
      const int zb0 = (sl[m] >> 1) * L;
      float2& zk = b0[sw(zb0 + k)];   // add i v at k and i conj(v) at L - k
      zk.x -= v.y;
      zk.y += v.x;
      if (!self) {
        float2& zm = b0[sw(zb0 + L - k)];
        zm.x += v.y;
        zm.y += v.x;
      }
    }
    __syncthreads();
  }
  float2* zb = fft_block(b0, b1, tw, L, P, +1);
  float2* other = (zb == b0) ? b1 : b0;
  double sb[6] = {0, 0, 0, 0, 0, 0};
  double vmax = 0.0;
  const float lam0 = a.law.lam0, mu0 = a.law.mu0;
  for (int vb = 0; vb < R * L; vb += kVox * nt) {
    int pid[kVox];
    float stv[kVox][NS];
#pragma unroll
    for (int u = 0; u < kVox; ++u) {
      const int v = vb + tid + u * nt;
      pid[u] = 0;
      if (v < R * L) {
        const int r = fdiv(v, a.dL), x = v - r * L;
        const long long g = (long long)(row0 + r) * L + x;
        pid[u] = a.phase[g];
        if (PLASTIC) {
#pragma unroll
          for (int i = 0; i < NS; ++i) stv[u][i] = a.state[i * a.N + g];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kVox; ++u) {
      const int v = vb + tid + u * nt;
      if (v >= R * L) continue;
      const int r = fdiv(v, a.dL), x = v - r * L;
      const long long g = (long long)(row0 + r) * L + x;
      float e[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const int s = r * NC + c;
        const float2 z = zb[sw((s >> 1) * L + x)];
        e[c] = ((s & 1) ? z.y : z.x) * a.invN;
      }
      float e6[6];
      comp_to6<NC>(e, e6);
      const DevPhase ph = phs[pid[u]];
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
      stress6<PLASTIC>(e6, ph, ep, alpha, o);
      if (!FINAL) {
        const float tr = e6[0] + e6[1] + e6[2];
        float tau6[6];
#pragma unroll
        for (int i = 0; i < 3; ++i) tau6[i] = o.s[i] - (lam0 * tr + 2.f * mu0 * e6[i]);
#pragma unroll
        for (int i = 3; i < 6; ++i) tau6[i] = o.s[i] - 2.f * mu0 * e6[i];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int s = r * NC + c;
          float* dst = reinterpret_cast<float*>(other + sw((s >> 1) * L + x));
          dst[s & 1] = tau6[comp6<NC>(c)];
        }
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
            const double s0 = o.s[0], s1 = o.s[1], s2 = o.s[2];
            const double pmd = (s0 + s1 + s2) / 3.0;
            const double d0 = s0 - pmd, d1 = s1 - pmd, d2 = s2 - pmd;
            const double qq = d0 * d0 + d1 * d1 + d2 * d2 +
                              2.0 * ((double)o.s[3] * o.s[3] + (double)o.s[4] * o.s[4] +
                                     (double)o.s[5] * o.s[5]);
            const double yl = (double)ph.sy + (double)ph.H * (double)o.alpha;
            vmax = fmax(vmax, fabs(sqrt(1.5 * qq) - yl) / (double)ph.sy);
          }
        } else if (a.alpha_out) {
          a.alpha_out[g] = 0.f;
        }
      }
    }
  }
  if (FINAL) {
    for (int i = 0; i < 6; ++i) {
      const double t = block_sum_d(sb[i], red);
      if (tid == 0) a.sbar_part[blockIdx.x * 6 + i] = t;
    }
    const double vm = block_max_d(vmax, red);
    if (tid == 0) a.viol_part[blockIdx.x] = vm;
    return;
  }
  // an odd line count leaves the last sequence's imaginary carrier unused: zero it
  if (S & 1)
    for (int x = tid; x < L; x += nt) other[sw((P - 1) * L + x)].y = 0.f;
  __syncthreads();
  const float2* zf = fft_block(other, zb, tw, L, P, -1);
  // the pattern's kx columns of the R rows back to the polarization lines (item order as the
  // loads: R consecutive rows of one line column)
  for (int u = tid; u < nsc; u += nt) {
    const int q = u / R, r = u - q * R;
    const int c = fdiv(q, a.dKx), j = q - c * Kx;
    const int s = r * NC + c;
    const int k = kxs[j];
    const int zb0 = (s >> 1) * L;
    const float2 zk = zf[sw(zb0 + k)], zm = zf[sw(zb0 + (k == 0 ? 0 : L - k))];
    float2 out;
    if ((s & 1) == 0) out = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    else out = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    a.T1p[(long long)q * Ny + row0 + r] = out;
  }
  __syncthreads();   // the buffers are reused by the next phase
}

// Column phase for the kx of index j (see the top of the file). full = false: only the
// inverse transform of the current coefficients (the start of a solve). Returns the FP64
// squared-increment sum of this kx to thread 0 (full only).
__device__ double p_col(const PersistArgs& a, int j, bool full, const float2* tw, float2* b0,
                        float2* b1, double* red) {
  constexpr int NC = 3;
  const int L = a.Ny, Kx = a.Kx;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int span = span_of(NC * L);
  const float2* z = nullptr;
  float2* w = b0;
  float2* scratch = b1;
  if (full) {
    // the NC columns of this kx, loads issued kL at a time before their stores
    constexpr int kL = 8;
    for (int i0 = tid; i0 < NC * L; i0 += kL * nt) {
      float2 v[kL];
#pragma unroll
      for (int u = 0; u < kL; ++u) {
        const int i = i0 + u * nt;
        if (i < NC * L) {
          const int c = fdiv(i, a.dNy), y = i - c * L;
          v[u] = __ldcg(a.T1p + (long long)(c * Kx + j) * L + y);
        }
      }
#pragma unroll
      for (int u = 0; u < kL; ++u) {
        const int i = i0 + u * nt;
        if (i < NC * L) b0[sw(i)] = v[u];
      }
    }
    __syncthreads();
    z = fft_block(b0, b1, tw, L, NC, -1);
    w = (z == b0) ? b1 : b0;
    scratch = const_cast<float2*>(z);
  }
  for (int i = tid; i < span; i += nt) w[i] = make_float2(0.f, 0.f);
  __syncthreads();
  double dsum = 0.0;   // FP64 sum of the frequencies' squared increments (each in FP32)
  const int e0 = a.jptr[j], e1 = a.jptr[j + 1];
  // the entries of this kx, kE per thread at a time: their indices, then their positions and
  // old coefficients, each group of loads issued together
  constexpr int kE = 2;
  for (int eb0 = e0 + tid; eb0 < e1; eb0 += kE * nt) {
    int2 en[kE];
    float4 n[kE];
    int pos[kE];
    float2 old[kE][NC];
#pragma unroll
    for (int u = 0; u < kE; ++u) {
      const int e = eb0 + u * nt;
      en[u] = make_int2(0, -1);
      if (e < e1) {
        en[u] = a.jent[e];
        if (full) n[u] = a.jn[e];
      }
    }
#pragma unroll
    for (int u = 0; u < kE; ++u) {
      if (en[u].y < 0) continue;
      pos[u] = a.kym[en[u].x];
      const long long base = (long long)en[u].x * NC * Kx + j;
#pragma unroll
      for (int c = 0; c < NC; ++c) old[u][c] = __ldcg(a.ER + base + (long long)c * Kx);
    }
#pragma unroll
    for (int u = 0; u < kE; ++u) {
      if (en[u].y < 0) continue;
      const long long base = (long long)en[u].x * NC * Kx + j;
      if (!full) {
#pragma unroll
        for (int c = 0; c < NC; ++c) w[sw(c * L + pos[u])] = old[u][c];
        continue;
      }
      const bool mixed0 = en[u].y == 1 && a.st->mixed;
      float2 tv[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c)
        tv[c] = (en[u].y == 0 || mixed0) ? z[sw(c * L + pos[u])] : make_float2(0.f, 0.f);
      const double* eb = a.st->ebar;
      double em[6];
      if (mixed0) {
        mixed_macro<NC>(tv, a.Nd, a.st, em);
        for (int i = 0; i < 6; ++i) a.st->ebar[i] = em[i];
        eb = em;
      }
      float er[NC], ei[NC];
      green_update<NC>(en[u].y, n[u], tv, eb, a.Nd, a.inv2mu0, a.cgam, er, ei);
      float diff = 0.f;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const float dr = er[c] - old[u][c].x, di = ei[c] - old[u][c].y;
        const float wc = (comp6<NC>(c) >= 3) ? 2.f : 1.f;   // Frobenius: shear counted twice
        diff = fmaf(n[u].w * wc, dr * dr + di * di, diff);
        const float2 nv = make_float2(er[c], ei[c]);
        a.ER[base + (long long)c * Kx] = nv;
        w[sw(c * L + pos[u])] = nv;
      }
      dsum += (double)diff;
    }
  }
  double t = 0.0;
  if (full) t = block_sum_d(dsum, red);   // barriers inside also order the scattered values
  __syncthreads();
  const float2* zi = fft_block(w, scratch, tw, L, NC, +1);
  for (int i = tid; i < NC * L; i += nt) {
    const int c = fdiv(i, a.dNy), y = i - c * L;
    a.T1[(long long)(c * Kx + j) * L + y] = zi[sw(i)];
  }
  __syncthreads();
  return t;
}

// TPB threads per block: 256 (two blocks per SM) or 512 (one block per SM), 128 registers per
// thread either way
template <bool PLASTIC, int TPB>
__global__ __launch_bounds__(TPB, 512 / TPB) void k_persist2d(const __grid_constant__ PersistArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ DevPhase phs[kMaxPhases];
  __shared__ int s_flag;
  __shared__ int s_done;
  const int tid = threadIdx.x, nt = blockDim.x;
  // the stage-major twiddle tables are read from global memory (read-only for the launch, so
  // L1-cached), which leaves shared memory to the two work buffers of two CTAs per SM
  const float2* twx = a.twx + fftc::stage_offset(a.Nx);
  const float2* twy = a.twy + fftc::stage_offset(a.Ny);
  float2* b0 = reinterpret_cast<float2*>(smem);
  float2* b1 = b0 + a.span_buf;
  int* kxs = reinterpret_cast<int*>(b1 + a.span_buf);
  for (int i = tid; i < a.Kx; i += nt) kxs[i] = a.kx[i];
  for (int i = tid; i < kMaxPhases; i += nt) phs[i] = a.law.ph[i];
  __syncthreads();
  // the decision's running values, identical in every CTA (thread 0 only: kept in shared
  // memory so that they hold no registers through the phases)
  __shared__ int s_iters;
  __shared__ double s_rmin;
  __shared__ unsigned long long s_tupd;
  if (tid == 0) {
    s_iters = a.st->iters;
    s_rmin = a.st->rmin;
  }
  // start: strain lines of the start coefficients
  for (int j = blockIdx.x; j < a.Kx; j += gridDim.x) p_col(a, j, false, twy, b0, b1, red);
  if (!grid_sync(a.bar, a.bar_limit, &s_flag)) {
    if (tid == 0) atomicExch(&a.st->timeout, 1);
    return;
  }
  if (a.trace && blockIdx.x == 0 && tid == 0) s_tupd = global_ns();
  for (int u = 0;; ++u) {
    p_row<PLASTIC, false, 4>(a, twx, b0, b1, kxs, phs, red);
    if (!grid_sync(a.bar, a.bar_limit, &s_flag)) {
      if (tid == 0) atomicExch(&a.st->timeout, 1);
      return;
    }
    __shared__ unsigned long long s_trow;
    if (a.trace && blockIdx.x == 0 && tid == 0) s_trow = global_ns();
    for (int j = blockIdx.x; j < a.Kx; j += gridDim.x) {
      const double t = p_col(a, j, true, twy, b0, b1, red);
      if (tid == 0) a.part[j] = t;
    }
    if (!grid_sync(a.bar, a.bar_limit, &s_flag)) {
      if (tid == 0) atomicExch(&a.st->timeout, 1);
      return;
    }
    // decision: the kx partials summed in a fixed order (per-thread strided sums, the block
    // tree of block_sum_d), the same in every CTA
    double s = 0.0;
    for (int i = tid; i < a.Kx; i += nt) s += __ldcg(a.part + i);
    s = block_sum_d(s, red);
    if (tid == 0) {
      // tol, enorm, inv_n2 and max_iter are set by the host before the launch
      double r = sqrt(s * a.st->inv_n2);
      if (a.st->enorm > 0.0) r /= a.st->enorm;
      const int iters = s_iters + 1;
      const double rmin = fmin(s_rmin, r);
      s_iters = iters;
      s_rmin = rmin;
      int done = 0, nonfinite = 0, diverged = 0;
      if (!isfinite(r)) {
        nonfinite = done = 1;
      } else if (r > kDivergeRatio * rmin && r > kDivergeFloor) {
        diverged = done = 1;
      } else if (r < a.st->tol || iters >= a.st->max_iter) {
        done = 1;
      }
      if (blockIdx.x == 0) {
        a.st->iters = iters;
        a.st->last_r = r;
        a.st->rmin = rmin;
        a.st->nonfinite = nonfinite;
        a.st->diverged = diverged;
        a.st->done = done;
        if (a.trace && u < a.trace_cap) {
          const unsigned long long t_col = global_ns();
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

// Final pass over the same row partition: fields, homogenised-stress partials, commit.
template <bool PLASTIC>
__global__ __launch_bounds__(512) void k_persist_final(const __grid_constant__ PersistArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double red[32];
  __shared__ DevPhase phs[kMaxPhases];
  const int tid = threadIdx.x, nt = blockDim.x;
  const float2* twx = a.twx + fftc::stage_offset(a.Nx);
  float2* b0 = reinterpret_cast<float2*>(smem);
  float2* b1 = b0 + a.span_buf;
  int* kxs = reinterpret_cast<int*>(b1 + a.span_buf);
  for (int i = tid; i < a.Kx; i += nt) kxs[i] = a.kx[i];
  for (int i = tid; i < kMaxPhases; i += nt) phs[i] = a.law.ph[i];
  __syncthreads();
  p_row<PLASTIC, true, 4>(a, twx, b0, b1, kxs, phs, red);
}

// ------------------------------------------------------------------------------------------
// host side
namespace {

// dynamic shared memory per block: the 227 KB per-block limit of sm_103a less room for the
// kernels' static shared memory
constexpr size_t kPersistSmemMax = 226 * 1024;

size_t persist_smem(const rf_ctx* c, int R) {
  const int P = (R * 3 + 1) / 2;
  const int span = std::max(span_of(P * c->nx), span_of(3 * c->ny));
  return 2 * (size_t)span * sizeof(float2) + (size_t)c->Kx * sizeof(int) + 16;
}

template <bool PL>
const void* persist_kernel(int threads) {
  return threads == 256 ? (const void*)k_persist2d<PL, 256> : (const void*)k_persist2d<PL, 512>;
}

template <bool PL>
cudaError_t launch_persist(rf_ctx* c, const PersistArgs& a, bool final_pass) {
  if (final_pass) {
    k_persist_final<PL><<<c->persist_G, c->persist_threads, c->persist_smem, c->stream>>>(a);
    return cudaGetLastError();
  }
  void* args[] = {const_cast<PersistArgs*>(&a)};
  return cudaLaunchCooperativeKernel(persist_kernel<PL>(c->persist_threads), dim3(c->persist_G),
                                     dim3(c->persist_threads), args, c->persist_smem, c->stream);
}

PersistArgs persist_args(rf_ctx* c) {
  PersistArgs a{};
  a.T1 = c->d_T1;
  a.T1p = c->d_T1p;
  a.ER = c->d_ER;
  a.phase = c->d_phase;
  a.state = c->d_state;
  a.kx = c->d_kx;
  a.twx = c->d_twx;
  a.twy = c->d_twy;
  a.jptr = c->d_jptr;
  a.jent = c->d_jent;
  a.jn = c->d_jn;
  a.kym = c->d_kym;
  a.Nx = c->nx;
  a.Ny = c->ny;
  a.Kx = c->Kx;
  a.rbase = c->rows / c->persist_G;
  a.rextra = c->rows % c->persist_G;
  const int R = a.rbase + (a.rextra > 0 ? 1 : 0);
  a.span_buf = std::max(span_of(((R * 3 + 1) / 2) * c->nx), span_of(3 * c->ny));
  a.dL = make_fastdiv((unsigned)c->nx);
  a.dKx = make_fastdiv((unsigned)std::max(1, c->Kx));
  a.dNy = make_fastdiv((unsigned)c->ny);
  a.N = c->N;
  a.invN = (float)(1.0 / (double)c->N);
  a.law = c->law;
  a.inv2mu0 = (float)(0.5 / c->mu0);
  a.cgam = (float)((c->lam0 + c->mu0) / (c->mu0 * (c->lam0 + 2.0 * c->mu0)));
  a.Nd = (double)c->N;
  a.st = c->d_status;
  a.part = c->d_part;
  a.sbar_part = c->d_sbar_part;
  a.viol_part = c->d_viol_part;
  a.bar = c->d_bar;
  a.bar_limit = 1L << 26;
  return a;
}

}  // namespace

// Chooses the grid (one or two CTAs per SM, rows spread evenly) and block size that fit
// co-resident; false if the persistent solve is not possible for this pattern.
bool persist_geometry(rf_ctx* c, int threads, int per_sm) {
  if (c->dim != 2 || !c->d_jptr) return false;
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
  const int G = std::min(c->rows, per_sm * sms);
  if (G < 1) return false;
  const int R = c->rows / G + (c->rows % G ? 1 : 0);
  const size_t smem = persist_smem(c, R);
  if (smem > kPersistSmemMax) return false;
  if (threads != 256 && threads != 512) return false;
  int occ = 0;
  const void* k = c->has_plastic ? persist_kernel<true>(threads) : persist_kernel<false>(threads);
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, threads, smem);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if ((long long)occ * sms < G) return false;
  c->persist_G = G;
  c->persist_threads = threads;
  c->persist_per_sm = per_sm;
  c->persist_smem = smem;
  return true;
}

// Barrier words and a first geometry (the autotuner may choose another); RF_ERR_INVALID if
// no geometry fits co-resident.
int persist_setup(rf_ctx* c) {
  if (int e = palloc(c, &c->d_bar, 2, "persistent solve")) return e;
  const int cand[4][2] = {{512, 2}, {256, 2}, {512, 1}, {256, 1}};
  for (const auto& cd : cand)
    if (persist_geometry(c, cd[0], cd[1])) return RF_OK;
  set_error("persistent solve: no grid of this pattern fits co-resident on the device");
  return RF_ERR_INVALID;
}

void init_attributes_persist() {
  for (const void* k : {(const void*)k_persist2d<true, 512>, (const void*)k_persist2d<true, 256>,
                        (const void*)k_persist2d<false, 512>, (const void*)k_persist2d<false, 256>})
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPersistSmemMax);
  cudaFuncSetAttribute(k_persist_final<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kPersistSmemMax);
  cudaFuncSetAttribute(k_persist_final<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)kPersistSmemMax);
  cudaGetLastError();   // a refused attribute only narrows the geometries that fit
}

// One cooperative launch: the start's inverse along y, then updates until the decision ends the
// solve (the status on the device holds tol, max_iter and the normalisation).
int launch_persist_solve(rf_ctx* c, unsigned long long* trace, int trace_cap) {
  cudaError_t e = cudaMemsetAsync(c->d_bar, 0, 2 * sizeof(unsigned), c->stream);
  if (e != cudaSuccess) return cuda_fail(e, "persistent solve");
  PersistArgs a = persist_args(c);
  a.trace = trace;
  a.trace_cap = trace_cap;
  e = c->has_plastic ? launch_persist<true>(c, a, false) : launch_persist<false>(c, a, false);
  c->launches += 1;
  return e == cudaSuccess ? RF_OK : cuda_fail(e, "persistent solve");
}

// Final pass over the same row partition (no grid barrier inside: a plain launch).
int launch_persist_final(rf_ctx* c, int commit) {
  PersistArgs a = persist_args(c);
  a.commit = commit;
  a.eps_out = c->d_eps;
  a.sig_out = c->d_sig;
  a.alpha_out = c->d_alpha;
  cudaError_t e = c->has_plastic ? launch_persist<true>(c, a, true)
                                 : launch_persist<false>(c, a, true);
  c->launches += 1;
  return e == cudaSuccess ? RF_OK : cuda_fail(e, "persistent final pass");
}

}  // namespace rfk
