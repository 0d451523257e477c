// Internal declarations of the reduced-frequency solver library (sm_103a).
//
// Data layout in device memory (see the C ABI header for conventions):
//   phase    uint8  [Nz][Ny][Nx]
//   state    float  [NS][N]     J2 internal variables, NS = 4 in 2D (ep11, ep22, ep12, alpha;
//                                ep33 = -(ep11 + ep22)), 7 in 3D (ep 11,22,33,23,13,12, alpha)
//   ER       float2 [Kz][Ky][NC][Kx]  reduced strain coefficients on the kx >= 0 half of the
//                                pattern, scattered into the dense (kz, ky, kx) rectangle of the
//                                distinct values; entries outside the pattern stay zero
//   T1, T1p  float2 [rows][NC][Kx]   per grid row (y, z): line transforms along x
//   T2       float2 [Nz][Ky][NC][Kx] (3D) line transforms along y
//   OUT      float2 [S][Kz][Ky][NC][Kx] split-K partial sums of the forward transform
// NC = 3 (11, 22, 12) in 2D plane strain, 6 (11, 22, 33, 23, 13, 12) in 3D.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/rf.h"

namespace rfk {

constexpr int kMaxPhases = 16;
constexpr int kGammaBlock = 128;   // threads per Green-operator block (one frequency each)

struct DevPhase {
  float lam, mu, sy, H;
  int plastic;
  float r3muH;   // 1 / (3 mu + H) of a plastic phase (the radial return's scaling), else 0
  int pad[2];
};

struct LawParams {
  DevPhase ph[kMaxPhases];
  float lam0, mu0;
  int has_plastic;
  int pad;
};

// per frequency of the half pattern
struct HIdx {
  int j, iy, iz;
  int kind;   // 0: regular, 1: zero frequency, 2: null operator
};

struct Status {
  int done;       // set when converged, capped, non-finite, diverged or timed out
  int iters;      // fixed-point updates of this solve
  int max_iter;
  int nonfinite;
  int timeout;    // a bounded device-side wait ran out
  int diverged;   // the measure grew past kDivergeRatio times its minimum (and kDivergeFloor)
  double tol;
  double enorm;   // Frobenius norm of ebar (0: absolute measure)
  double inv_n2;  // 1 / N^2 (Parseval)
  double last_r;
  double rmin;    // smallest measure of this solve so far
  double ebar[6]; // macroscopic strain (mixed control: the one of the last update)
  // mixed macroscopic control: component i of `target` is an average stress where
  // control[i] = 1, a strain where 0; lam0, mu0 of the reference medium in FP64
  int mixed;
  int control[6];
  int pad2;
  double target[6];
  double lam0, mu0;
};

// Divergence rule of the convergence decision: the measure exceeds both kDivergeRatio times
// its smallest value in the solve and kDivergeFloor (relative to |ebar|).
constexpr double kDivergeRatio = 1e4;
constexpr double kDivergeFloor = 1e-3;

struct DftAxisArgs {
  const float2* in;
  long long in_split_stride;
  int in_splits;
  long long in_bstride;
  float2* out;
  long long out_split_stride;
  int out_splits;
  long long out_bstride;
  int M, N, K, batch;
  const int* mvals;   // nullable: m itself; values reduced to [0, L)
  const int* kvals;   // nullable: k itself
  const float2* table;  // exp(+2 pi i t / L), t in [0, L)
  int L;
  int sign;           // +1 inverse, -1 forward
  const int* done;    // nullable early-exit flag
};

struct RowArgs {
  const float2* T;      // [rows][NC][Kx]
  float2* Tout;         // [rows][NC][Kx]
  const uint8_t* phase;
  float* state;         // [NS][N] or null
  const int* kx;        // [Kx]
  const float* fac;     // [Kx] weight / N
  const float2* table;  // exp(+2 pi i t / Nx)
  int Nx, Kx, rows, R;
  long long N;
  LawParams law;
  float* eps_out;       // final pass: [6][N] (nullable)
  float* sig_out;       // final pass: [6][N] (nullable)
  float* alpha_out;     // final pass: [N] (nullable)
  double* sbar_part;    // final pass: [gridDim.x][6]
  double* viol_part;    // final pass: [gridDim.x]
  int commit;
  const int* done;
};

struct GammaArgs {
  const float2* OUT;
  int splits;
  long long split_stride;
  float2* ER;
  const HIdx* hidx;
  const float4* hn;     // unit wave vector (x, y, z) and multiplicity in w
  long long Kh;
  int Kx, Ky, NC;
  float inv2mu0, cgam;
  const Status* st;
  Status* status;       // convergence decision written by the last block
  unsigned* counter;    // blocks finished (reset to 0 by the last block)
  double* part;         // [gridDim.x]
  const int* done;
  // while-loop graph: the last block clears the loop condition when it sets done
  cudaGraphConditionalHandle cond;
  int use_cond;
};

}  // namespace rfk

// split-precision transform along y or z: precomputed A tiles (see rf_tc.cu)
struct TcAxis {
  unsigned char* A = nullptr;
  int M = 0, K = 0, nMT = 0, nKC = 0;
};

struct rf_ctx {
  int dev = 0;
  int dim = 2, nx = 1, ny = 1, nz = 1, nc = 3, ns = 0;
  long long N = 0;
  int rows = 0;
  rf_options opt{};
  cudaStream_t stream = nullptr;
  int n_phases = 0;
  rf_phase phases[rfk::kMaxPhases];
  rfk::LawParams law{};
  double lam0 = 0, mu0 = 0;
  bool has_plastic = false;

  uint8_t* d_phase = nullptr;
  float* d_state = nullptr;

  // pattern
  bool have_pattern = false;
  long long K = 0, Kh = 0;
  int Kx = 0, Ky = 0, Kz = 0;
  std::vector<int32_t> pat;       // [K][3] as given
  std::vector<long long> map_h;   // per pattern entry: half index
  std::vector<char> map_conj;     // per pattern entry: conjugate of the half entry
  std::vector<long long> h_src;   // per half entry: a pattern entry equal to it
  int* d_kx = nullptr;   // kx values (>= 0)
  int* d_kym = nullptr;  // ky values mod Ny
  int* d_kzm = nullptr;  // kz values mod Nz
  float* d_fac = nullptr;
  rfk::HIdx* d_hidx = nullptr;
  float4* d_hn = nullptr;
  float2* d_ER = nullptr;
  float2* d_T1 = nullptr;
  float2* d_T1p = nullptr;
  float2* d_T2 = nullptr;
  float2* d_T2f = nullptr;
  float2* d_OUT = nullptr;
  int splitB = 1, splitC = 1;
  long long rect = 0;             // Kz*Ky*NC*Kx
  float2* d_twx = nullptr;
  float2* d_twy = nullptr;
  float2* d_twz = nullptr;
  double* d_part = nullptr;       // residual block partials
  unsigned* d_counter = nullptr;  // finished-block counter of the Green kernel
  int n_part = 0;
  double* d_sbar_part = nullptr;  // [row blocks][6]
  double* d_viol_part = nullptr;
  double* d_sbar = nullptr;       // [8]: sbar[6], viol, pad
  rfk::Status* d_status = nullptr;
  rfk::Status* h_status = nullptr;  // pinned
  double* h_sbar = nullptr;         // pinned [8]
  float* d_eps = nullptr;
  float* d_sig = nullptr;
  float* d_alpha = nullptr;
  bool fields_valid = false;
  int row_R = 1, row_blocks = 0;
  size_t row_smem = 0;

  long long zero_base_idx = 0;    // ER offset of the zero frequency, component 0
  std::vector<rfk::HIdx> h_hidx;  // host copy of the half-pattern indices
  float2* d_warm = nullptr;       // [Kh][6] warm-start staging

  // FFT transform mode
  int fft_R = 0, fft_blocks = 0, fft_C = 0;
  int fft_rbase = 0, fft_rextra = 0;    // row partition (see set_rows_balanced)
  int fft_row_threads = 256, fft_col_threads = 256;   // block sizes (autotuned with the tiles)
  int fft_row_warps = 0;   // > 0: row passes (not the final one) on the warp-FFT row kernel
  int fft_colw_M = 1;      // kx columns per block of the warp-FFT column phase (kColWarp)
  size_t fft_smem = 0;
  // 2D column phase: 0 forward y, Green kernel, inverse y; 1 one fused kernel per kx group
  // (kColFused); 2 forward y, then the Green operator inside the inverse y kernel
  // (kColGreenInv); 4 as 1 with a warp per line column, the transforms in registers and the
  // line coefficients in kx slabs (kColWarp, 1024 x 1024, warp-FFT row kernel); 5 the
  // persistent solve on the same passes (kColPersistW). Modes 1, 2 and 4 start a solve with one
  // inverse y of the start coefficients (3 and 5 inside their launch).
  int fft_colmode = 0;
  int fft_M = 1, fft_M_threads = 256;   // kx columns and threads per fused block
  // persistent 2D solve (column mode kColPersistent): grid, block size, dynamic shared memory,
  // grid-barrier words, per-update phase stamps of traced solves
  int persist_G = 0, persist_threads = 512, persist_per_sm = 0;
  size_t persist_smem = 0;
  unsigned* d_bar = nullptr;
  unsigned long long* d_ptrace = nullptr;
  int* d_jptr = nullptr;                // [Kx + 1] offsets of each kx's entries in d_jlist
  int* d_jlist = nullptr;               // half-pattern entries grouped by kx index
  int2* d_jent = nullptr;               // in d_jlist order: (rectangle row iy, frequency kind)
  float4* d_jn = nullptr;               // in d_jlist order: unit wave vector, multiplicity
  // last autotuned choice, reused when a new pattern has the same distinct kx, ky, kz counts
  struct Tuned {
    bool valid = false;
    int Kx = 0, Ky = 0, Kz = 0;
    int R = 0, row_threads = 0, C = 0, col_threads = 0, M = 0, M_threads = 0;
    int row_blocks_balanced = 0;
    int colmode = 0;
    int persist_per_sm = 0, persist_threads = 0;
    int row_warps = 0, colw_M = 1;
  } tuned;

  // split-precision (tensor-core) transforms along x
  unsigned char* d_phiI = nullptr;
  unsigned char* d_phiF = nullptr;
  TcAxis tc_yf, tc_yi, tc_zf, tc_zi;   // forward / inverse along y and z
  // capacities of the pattern-scoped device buffers (kept across patterns, see palloc)
  std::unordered_map<const void*, size_t> pcap;
  int* d_hk = nullptr;                 // pattern upload staging
  float* d_Tout = nullptr;        // [nXS][rows][NC][2 Kx] partial forward sums per x slice
  int* d_tc_err = nullptr;
  int tc_nXS = 0, tc_nJT = 0, tc_nJC = 0, tc_nXC = 0, tc_R = 0, tc_Qp = 0;
  unsigned tc_cols = 0;
  size_t tc_smem = 0;

  // load-path state: macroscopic strain and homogenised stress of the last solve or increment
  double prev_macro[6] = {0, 0, 0, 0, 0, 0};
  double prev_sbar[6] = {0, 0, 0, 0, 0, 0};

  // compatibility step: a context on the same grid with the full set of frequencies (created
  // by the first rf_compat, dropped when the phase map changes)
  rf_ctx* compat = nullptr;

  double last_sbar[6] = {0, 0, 0, 0, 0, 0};   // homogenised stress of the fields held now
  double* d_err = nullptr;                    // [kErrBlocks + 2] partials of rf_stress_errors

  // CUDA graphs of update chunks (replayed instead of per-kernel launches)
  struct TraceIter;
  struct GraphEntry {
    int chunk;
    bool tracing;
    cudaGraphExec_t exec;
    std::vector<int> trace_first;   // index into traces of each captured update
    long long kernels;              // kernel nodes in the graph (counted at every replay)
  };
  std::vector<GraphEntry> graphs;
  // one-launch solve: a conditional while node whose body is one update (untraced solves)
  cudaGraphExec_t while_exec = nullptr;
  cudaGraphConditionalHandle while_cond = 0;
  long long while_kernels = 0;   // kernel nodes per body
  bool while_failed = false;     // this pattern's graph could not be built: use chunks
  bool capturing_while = false;
  bool own_stream = false;
  bool capturing = false;

  // tracing: one event before each stage of an update and one after the last stage
  bool tracing = false;
  std::vector<cudaEvent_t> ev_pool;
  struct TraceIter {
    long long idx;                 // update index within the solve (-1: final pass)
    int stage[8];
    cudaEvent_t ev[9];
    int n;
  };
  std::vector<TraceIter> pending;
  std::vector<TraceIter> graph_traces;   // events owned by captured graphs
  TraceIter* cur = nullptr;
  long long launched_iters = 0;
  double stage_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long stage_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};

  // statistics
  long long launches = 0;
  int last_iters = 0;
  double last_residual = 0;
  double last_viol = 0;
};

namespace rfk {

// Division by a kernel-invariant divisor d in [1, 2^31) as a multiply-high, an add and a shift
// (round-up multiplier method of Granlund and Montgomery, 1994): with s = ceil(log2 d) and
// m = floor(2^32 (2^s - d) / d) + 1, n / d = (umulhi(n, m) + n) >> s for 0 <= n < 2^31.
struct FastDiv {
  unsigned m, s;
};

inline FastDiv make_fastdiv(unsigned d) {
  unsigned s = 0;
  while ((1ull << s) < d) ++s;
  const unsigned long long m = ((1ull << 32) * ((1ull << s) - d)) / d + 1;
  return FastDiv{(unsigned)m, s};
}

__device__ __forceinline__ int fdiv(int n, FastDiv f) {
  return (int)((__umulhi((unsigned)n, f.m) + (unsigned)n) >> f.s);
}

// Convergence decision from the block partials, in a fixed summation order. The whole block
// calls it (block size <= 1024, sh >= 32 entries): each thread sums a fixed strided subset with
// its loads issued four at a time, then warp trees and the warp sums in order.
__device__ inline void decide(const double* part, int n, Status* st, double* sh) {
  double s = 0.0;
  for (int i0 = threadIdx.x; i0 < n; i0 += 4 * blockDim.x) {
    double v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * blockDim.x;
      v[u] = i < n ? __ldcg(part + i) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) s += v[u];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) tot += sh[w];
    double r = sqrt(tot * st->inv_n2);
    if (st->enorm > 0.0) r /= st->enorm;
    st->iters += 1;
    st->last_r = r;
    st->rmin = fmin(st->rmin, r);
    if (!isfinite(r)) {
      st->nonfinite = 1;
      st->done = 1;
    } else if (r > kDivergeRatio * st->rmin && r > kDivergeFloor) {
      st->diverged = 1;
      st->done = 1;
    } else if (r < st->tol || st->iters >= st->max_iter || st->timeout) {
      st->done = 1;
    }
  }
}

// Programmatic dependent launch: the kernel may be scheduled while its predecessor in the stream
// drains; it runs its independent prologue (tables, shared-memory setup) and then calls
// grid_dep_wait() before it reads anything the predecessor writes. Every block reaches the wait
// before it exits, so completion stays transitive along the chain. Without the launch attribute
// the wait returns at once.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// kernels.cu
void set_error(const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

// Pattern-scoped device buffers live as long as their context and grow when a new pattern
// needs more room: cudaFree synchronises the device, so re-allocating a dozen buffers for every
// rf_set_pattern costs milliseconds. Buffers are released in rf_destroy.
template <class T>
inline int palloc(rf_ctx* c, T** p, size_t n, const char* what) {
  if (n == 0) n = 1;
  const size_t bytes = n * sizeof(T);
  auto it = c->pcap.find(p);
  if (*p && it != c->pcap.end() && it->second >= bytes) return RF_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  if (cudaMalloc(reinterpret_cast<void**>(p), bytes) != cudaSuccess) {
    c->pcap.erase(p);
    return cuda_fail(cudaGetLastError(), what);
  }
  c->pcap[p] = bytes;
  return RF_OK;
}
int launch_iteration(rf_ctx* c);
int launch_inverse(rf_ctx* c);
int launch_final(rf_ctx* c, int commit);
int launch_setup_tables(rf_ctx* c);
int launch_hinfo(rf_ctx* c, const int* d_hk, long long Kh);
int launch_reset_er(rf_ctx* c, const double* ebar6, double scale_old);
int launch_warm_project(rf_ctx* c, const float2* d_warm6, const double* ebar6);
int launch_phase_hist(rf_ctx* c, unsigned long long* d_hist);
int launch_scatter_full(rf_ctx* c, rf_ctx* full);
int launch_law_sweep(rf_ctx* c, const float* eps, float* tau, float* sig);
constexpr int kErrBlocks = 304;
int launch_stress_errors(rf_ctx* c, const float* sig_ref, const double* sbar,
                         const double* sbar_ref);
long long zero_base(const rf_ctx* c);
// rf_tc.cu
int tc_setup(rf_ctx* c);
int launch_tc_row(rf_ctx* c, const int* done);
// rf_fft.cu
int fft_geometry(rf_ctx* c);
int fft_autotune(rf_ctx* c);
int launch_fft_row(rf_ctx* c, const int* done, bool final_pass, int commit);
int fft_inverse_stages(rf_ctx* c, const int* done);
int fft_forward_stages(rf_ctx* c, const int* done);
int launch_fft_colphase(rf_ctx* c, const int* done);
int launch_tc_axis(rf_ctx* c, const TcAxis& ax, const float2* in, int in_splits,
                   long long in_split_stride, long long in_bstride, float2* out,
                   long long out_bstride, int N, int batch, const int* done);
int launch_fft_green_inv(rf_ctx* c, const int* done);
int launch_gather_jentries(rf_ctx* c);
constexpr int kColSeparate = 0, kColFused = 1, kColGreenInv = 2, kColPersistent = 3,
              kColWarp = 4, kColPersistW = 5;
// rf_persist.cu
bool persist_geometry(rf_ctx* c, int threads, int per_sm);
int launch_persist_solve(rf_ctx* c, unsigned long long* trace, int trace_cap);
int launch_persist_final(rf_ctx* c, int commit);
void init_attributes_persist();
int persist_setup(rf_ctx* c);
int launch_gamma_finalize(rf_ctx* c, int splits, const int* done);
void trace_begin(rf_ctx* c, long long idx);
void trace_stage(rf_ctx* c, int stage);
void trace_end(rf_ctx* c);
int trace_collect(rf_ctx* c, long long real_iters);
void trace_collect_graph(rf_ctx* c, const rf_ctx::GraphEntry& g, long long base,
                         long long real_iters);
void init_attributes_kernels();
void init_attributes_tc();
void init_attributes_fft();
void init_attributes_fftwarp();
// warp-FFT row kernel (2D, Nx = 1024, three components): applicability, shared memory of a block
// of `warps` warps, and one row pass with c->fft_row_warps warps per block
bool row_warp_ok(const rf_ctx* c);
size_t row_warp_smem(int Kx, int warps);
int launch_fft_row_warp(rf_ctx* c, const int* done);
// warp-FFT column phase (2D, 1024 x 1024, three components; column mode kColWarp; line
// coefficients in kx slabs between the row pass and the column phase) and the inverse along y
// of the held coefficients that starts a solve in that mode
bool col_warp_ok(const rf_ctx* c);
int launch_fft_colphase_warp(rf_ctx* c, const int* done);
int launch_fft_coly_init_warp(rf_ctx* c);
// the persistent solve on the warp-FFT passes (column mode kColPersistW): applicability (1024^2,
// barrier words, a co-resident grid) and one cooperative launch per solve
bool persist_warp_ok(const rf_ctx* c);
int launch_persist_warp(rf_ctx* c, unsigned long long* trace, int trace_cap);
// pattern.cu
int pattern_adapted(const rf_grid* g, const uint8_t* pm, int incl, long long k_target,
                    int32_t* out, long long cap, long long* K_out, cudaStream_t s);
int pattern_radial(const rf_grid* g, long long k_target, int32_t* out, long long cap,
                   long long* K_out, cudaStream_t s);
int pattern_adapted_noalloc(const rf_grid* g, const uint8_t* pm, int incl, long long k_target,
                            int32_t* out, long long cap, long long* K_out, cudaStream_t s);
}  // namespace rfk
