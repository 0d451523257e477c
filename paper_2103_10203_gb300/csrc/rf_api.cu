// C ABI of the reduced-frequency solver: contexts, pattern bookkeeping, solve loops.
//
// Host code here only validates inputs, builds index tables for the reduced set and drives
// kernel launches; all arithmetic of the scheme runs in the kernels of rf_kernels.cu and
// rf_pattern.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "rf_fftcore.cuh"
#include "rf_internal.cuh"

namespace rfk {

static thread_local std::string g_err;

void set_error(const std::string& m) { g_err = m; }

int cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? RF_ERR_OOM : RF_ERR_CUDA;
}

long long zero_base(const rf_ctx* c) { return c->zero_base_idx; }

}  // namespace rfk

using namespace rfk;

namespace {

std::mutex g_attr_mutex;
bool g_attr_done[64] = {false};

void init_attributes(int dev) {
  std::lock_guard<std::mutex> lock(g_attr_mutex);
  if (dev < 0 || dev >= 64 || g_attr_done[dev]) return;
  init_attributes_kernels();
  init_attributes_tc();
  init_attributes_fft();
  init_attributes_persist();
  init_attributes_fftwarp();
  g_attr_done[dev] = true;
}

struct DeviceGuard {
  int old = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&old) == cudaSuccess && old != dev) {
      cudaSetDevice(dev);
      changed = true;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(old);
  }
};

int invalid(const char* msg) {
  set_error(msg);
  return RF_ERR_INVALID;
}

int ck(cudaError_t e, const char* what) { return e == cudaSuccess ? RF_OK : cuda_fail(e, what); }

template <class T>
int dalloc(T** p, size_t n, const char* what) {
  *p = nullptr;
  if (n == 0) n = 1;
  return ck(cudaMalloc(reinterpret_cast<void**>(p), n * sizeof(T)), what);
}

template <class T>
void dfree(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

double frob6(const double* e) {
  return std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2] +
                   2.0 * (e[3] * e[3] + e[4] * e[4] + e[5] * e[5]));
}

int signed_of(int i, int n) { return i <= n / 2 ? i : i - n; }
int wrapi(int k, int n) {
  int r = k % n;
  return r < 0 ? r + n : r;
}

// reference medium from the phases present (device histogram of the phase map)
int update_reference(rf_ctx* c) {
  unsigned long long* d_hist = nullptr;
  if (int e = dalloc(&d_hist, 256, "hist")) return e;
  std::vector<unsigned long long> hist(256, 0);
  int err = ck(cudaMemsetAsync(d_hist, 0, 256 * sizeof(unsigned long long), c->stream), "memset");
  if (!err) err = launch_phase_hist(c, d_hist);
  if (!err)
    err = ck(cudaMemcpyAsync(hist.data(), d_hist, 256 * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, c->stream), "copy hist");
  if (!err) err = ck(cudaStreamSynchronize(c->stream), "sync hist");
  cudaFree(d_hist);
  if (err) return err;
  double lmin = 1e300, lmax = -1e300, mmin = 1e300, mmax = -1e300, lsum = 0, msum = 0;
  bool plastic = false;
  for (int p = 0; p < 256; ++p) {
    if (!hist[p]) continue;
    if (p >= c->n_phases) return invalid("phase map holds an id >= n_phases");
    const rf_phase& ph = c->phases[p];
    lmin = std::min(lmin, ph.lambda);
    lmax = std::max(lmax, ph.lambda);
    mmin = std::min(mmin, ph.mu);
    mmax = std::max(mmax, ph.mu);
    lsum += ph.lambda * (double)hist[p];
    msum += ph.mu * (double)hist[p];
    plastic = plastic || ph.plastic;
  }
  if (c->opt.ref_medium == RF_REF_MINMAX) {
    c->lam0 = 0.5 * (lmin + lmax);
    c->mu0 = 0.5 * (mmin + mmax);
  } else {
    c->lam0 = lsum / (double)c->N;
    c->mu0 = msum / (double)c->N;
  }
  c->law.lam0 = (float)c->lam0;
  c->law.mu0 = (float)c->mu0;
  (void)plastic;
  return RF_OK;
}

void free_graphs(rf_ctx* c) {
  for (auto& g : c->graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  if (c->while_exec) cudaGraphExecDestroy(c->while_exec);
  c->while_exec = nullptr;
  c->while_failed = false;
  for (auto& t : c->graph_traces)
    for (int i = 0; i <= t.n; ++i)
      if (t.ev[i]) cudaEventDestroy(t.ev[i]);
  c->graph_traces.clear();
}

// graph of `chunk` updates (captured once per chunk size and tracing state, then replayed)
int get_graph(rf_ctx* c, int chunk, rf_ctx::GraphEntry** out) {
  for (auto& g : c->graphs)
    if (g.chunk == chunk && g.tracing == c->tracing) {
      *out = &g;
      return RF_OK;
    }
  rf_ctx::GraphEntry g{chunk, c->tracing, nullptr, {}, 0};
  const size_t first = c->graph_traces.size();
  if (c->tracing) {
    // events are created before the capture begins
    while (c->ev_pool.size() < (size_t)chunk * 9) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) break;
      c->ev_pool.push_back(e);
    }
  }
  const long long launched = c->launched_iters;
  const long long kernels0 = c->launches;
  cudaGraph_t graph = nullptr;
  if (int e = ck(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "capture"))
    return e;
  c->capturing = true;
  int err = RF_OK;
  for (int i = 0; i < chunk && !err; ++i) err = launch_iteration(c);
  c->capturing = false;
  c->launched_iters = launched;
  g.kernels = c->launches - kernels0;   // counted when the graph is replayed
  c->launches = kernels0;
  cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
  if (!err && ce != cudaSuccess) err = cuda_fail(ce, "end capture");
  if (!err) {
    ce = cudaGraphInstantiate(&g.exec, graph, 0);
    if (ce != cudaSuccess) err = cuda_fail(ce, "instantiate graph");
  }
  if (graph) cudaGraphDestroy(graph);
  if (err) return err;
  for (size_t i = first; i < c->graph_traces.size(); ++i) g.trace_first.push_back((int)i);
  c->graphs.push_back(g);
  *out = &c->graphs.back();
  return RF_OK;
}

// One graph for a whole solve: a conditional while node whose body is kWhileBody updates; the
// Green kernel's last block clears the condition when it sets the done flag (converged, capped,
// non-finite or timed out), so the loop ends with the body in which the solve finished (updates
// after that return at once). If the graph cannot be built here, the solve falls back to
// replayed chunks of updates.
constexpr int kWhileBody = 8;

int get_while_graph(rf_ctx* c) {
  if (c->while_exec || c->while_failed) return RF_OK;
  cudaGraph_t graph = nullptr;
  auto give_up = [&]() {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    c->while_failed = true;
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
  c->while_cond = h;
  const long long launched = c->launched_iters;
  const long long kernels0 = c->launches;
  if (cudaStreamBeginCaptureToGraph(c->stream, body, nullptr, nullptr, 0,
                                    cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return give_up();
  const bool tr = c->tracing;
  c->tracing = false;
  c->capturing = true;
  c->capturing_while = true;
  int err = RF_OK;
  for (int i = 0; i < kWhileBody && !err; ++i) err = launch_iteration(c);
  c->capturing = false;
  c->capturing_while = false;
  c->tracing = tr;
  cudaGraph_t captured = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(c->stream, &captured);
  c->launched_iters = launched;
  c->while_kernels = c->launches - kernels0;
  c->launches = kernels0;
  if (err || ce != cudaSuccess) {
    set_error("");
    return give_up();
  }
  cudaGraphExec_t exec = nullptr;
  if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) return give_up();
  cudaGraphDestroy(graph);
  c->while_exec = exec;
  return RF_OK;
}

// forgets the current pattern; its device buffers stay for the next one (palloc)
void free_pattern(rf_ctx* c) {
  free_graphs(c);
  for (TcAxis* ax : {&c->tc_yf, &c->tc_yi, &c->tc_zf, &c->tc_zi}) {
    ax->M = ax->K = ax->nMT = ax->nKC = 0;
  }
  c->fft_colmode = kColSeparate;
  c->have_pattern = false;
  c->fields_valid = false;
}

void release_pattern_buffers(rf_ctx* c) {
  dfree(c->d_kx);
  dfree(c->d_kym);
  dfree(c->d_kzm);
  dfree(c->d_fac);
  dfree(c->d_hidx);
  dfree(c->d_hn);
  dfree(c->d_ER);
  dfree(c->d_T1);
  dfree(c->d_T1p);
  dfree(c->d_T2);
  dfree(c->d_T2f);
  dfree(c->d_OUT);
  dfree(c->d_part);
  dfree(c->d_counter);
  dfree(c->d_sbar_part);
  dfree(c->d_viol_part);
  dfree(c->d_warm);
  dfree(c->d_phiI);
  dfree(c->d_phiF);
  for (TcAxis* ax : {&c->tc_yf, &c->tc_yi, &c->tc_zf, &c->tc_zi}) dfree(ax->A);
  dfree(c->d_Tout);
  dfree(c->d_tc_err);
  dfree(c->d_jptr);
  dfree(c->d_jlist);
  dfree(c->d_jent);
  dfree(c->d_jn);
  dfree(c->d_hk);
  dfree(c->d_bar);
  dfree(c->d_ptrace);
  c->pcap.clear();
}

int reset_path_state(rf_ctx* c) {
  for (double& v : c->prev_macro) v = 0.0;
  for (double& v : c->prev_sbar) v = 0.0;
  if (c->d_ER)
    if (int e = ck(cudaMemsetAsync(c->d_ER, 0, sizeof(float2) * c->rect, c->stream), "memset ER"))
      return e;
  if (c->d_state)
    if (int e = ck(cudaMemsetAsync(c->d_state, 0, sizeof(float) * c->ns * c->N, c->stream),
                   "memset state"))
      return e;
  c->fields_valid = false;
  return RF_OK;
}

// Mixed control (host side of the device rule in rf_law.cuh, with <tau> = 0): the macroscopic
// strain of a homogeneous reference medium under the targets, used as the start and as the
// normalisation of the convergence measure.
void mixed_start(const rf_ctx* c, const int32_t* control, const double* target, double* E) {
  const double l = c->lam0, m = c->mu0;
  auto A = [&](int a, int b) {
    if (a < 3 && b < 3) return l + (a == b ? 2.0 * m : 0.0);
    return a == b ? 2.0 * m : 0.0;
  };
  int P[6], np = 0;
  for (int i = 0; i < 6; ++i) {
    E[i] = control[i] ? 0.0 : target[i];
    if (control[i]) P[np++] = i;
  }
  double M[6][7];
  for (int r = 0; r < np; ++r) {
    double rhs = target[P[r]];
    for (int j = 0; j < 6; ++j)
      if (!control[j]) rhs -= A(P[r], j) * E[j];
    for (int q = 0; q < np; ++q) M[r][q] = A(P[r], P[q]);
    M[r][np] = rhs;
  }
  for (int k = 0; k < np; ++k) {
    int piv = k;
    for (int r = k + 1; r < np; ++r)
      if (std::fabs(M[r][k]) > std::fabs(M[piv][k])) piv = r;
    if (piv != k)
      for (int q = 0; q <= np; ++q) std::swap(M[k][q], M[piv][q]);
    for (int r = k + 1; r < np; ++r) {
      const double f = M[r][k] / M[k][k];
      for (int q = k; q <= np; ++q) M[r][q] -= f * M[k][q];
    }
  }
  for (int k = np - 1; k >= 0; --k) {
    double v = M[k][np];
    for (int q = k + 1; q < np; ++q) v -= M[k][q] * E[P[q]];
    E[P[k]] = v / M[k][k];
  }
}

int init_status(rf_ctx* c, const double* macro, const int32_t* control = nullptr,
                const double* target = nullptr) {
  c->launched_iters = 0;
  Status& s = *c->h_status;
  s.mixed = control ? 1 : 0;
  s.pad2 = 0;
  for (int i = 0; i < 6; ++i) {
    s.control[i] = control ? control[i] : 0;
    s.target[i] = target ? target[i] : macro[i];
  }
  s.lam0 = c->lam0;
  s.mu0 = c->mu0;
  s.done = 0;
  s.iters = 0;
  s.max_iter = c->opt.max_iter;
  s.nonfinite = 0;
  s.timeout = 0;
  s.diverged = 0;
  s.tol = c->opt.tol;
  s.enorm = frob6(macro);
  s.inv_n2 = 1.0 / ((double)c->N * (double)c->N);
  s.last_r = 0.0;
  s.rmin = HUGE_VAL;
  for (int i = 0; i < 6; ++i) s.ebar[i] = macro[i];
  return ck(cudaMemcpyAsync(c->d_status, c->h_status, sizeof(Status), cudaMemcpyHostToDevice,
                            c->stream), "upload status");
}

// Persistent 2D solve: one cooperative launch runs the updates; traced solves record the phase
// stamps of every update (row phase, column phase, each up to its grid barrier).
int run_persistent(rf_ctx* c) {
  const int cap = c->tracing ? std::min(c->opt.max_iter, 8192) : 0;
  if (cap > 0)
    if (int e = palloc(c, &c->d_ptrace, 3 * (size_t)cap, "trace")) return e;
  unsigned long long* tr = cap > 0 ? c->d_ptrace : nullptr;
  if (int e = c->fft_colmode == kColPersistW ? launch_persist_warp(c, tr, cap)
                                             : launch_persist_solve(c, tr, cap))
    return e;
  if (int e = ck(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(Status), cudaMemcpyDeviceToHost,
                                 c->stream), "read status"))
    return e;
  if (int e = ck(cudaStreamSynchronize(c->stream), "persistent solve")) return e;
  c->launched_iters = c->h_status->iters;
  if (cap > 0) {
    const int n = std::min(cap, c->h_status->iters);
    std::vector<unsigned long long> t(3 * (size_t)std::max(n, 1));
    if (n > 0) {
      if (int e = ck(cudaMemcpy(t.data(), c->d_ptrace, sizeof(unsigned long long) * 3 * n,
                                cudaMemcpyDeviceToHost), "read trace"))
        return e;
      for (int u = 0; u < n; ++u) {
        c->stage_ms[2] += 1e-6 * (double)(t[3 * u + 1] - t[3 * u]);
        c->stage_ms[6] += 1e-6 * (double)(t[3 * u + 2] - t[3 * u + 1]);
        c->stage_n[2] += 1;
        c->stage_n[6] += 1;
      }
    }
  }
  return RF_OK;
}

int run_iterations(rf_ctx* c) {
  const int maxchunk = c->opt.check_every > 0 ? c->opt.check_every : 32;
  int chunk = std::min(4, maxchunk);
  const bool persistent = c->fft_colmode == kColPersistent || c->fft_colmode == kColPersistW;
  if (!persistent && c->fft_colmode != kColSeparate) {
    // these updates end with the inverse transform along y of their new coefficients, so the
    // first one needs the line transforms of the start coefficients
    const bool tr = c->tracing;
    c->tracing = false;
    const int e = c->fft_colmode == kColWarp ? launch_fft_coly_init_warp(c)
                                             : fft_inverse_stages(c, nullptr);
    c->tracing = tr;
    if (e) return e;
  }
  if (!persistent && !c->tracing) get_while_graph(c);
  if (persistent) {
    if (int e = run_persistent(c)) return e;
  } else if (!c->tracing && c->while_exec) {
    if (int e = ck(cudaGraphLaunch(c->while_exec, c->stream), "graph launch")) return e;
    if (int e = ck(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(Status),
                                   cudaMemcpyDeviceToHost, c->stream), "read status"))
      return e;
    if (int e = ck(cudaStreamSynchronize(c->stream), "iterate")) return e;
    c->launched_iters = c->h_status->iters;
    c->launches += c->while_kernels * ((c->h_status->iters + kWhileBody - 1) / kWhileBody);
  } else for (;;) {
    rf_ctx::GraphEntry* g = nullptr;
    if (int e = get_graph(c, chunk, &g)) return e;
    const long long base = c->launched_iters;
    if (int e = ck(cudaGraphLaunch(g->exec, c->stream), "graph launch")) return e;
    c->launched_iters += chunk;
    c->launches += g->kernels;
    if (int e = ck(cudaMemcpyAsync(c->h_status, c->d_status, sizeof(Status),
                                   cudaMemcpyDeviceToHost, c->stream), "read status"))
      return e;
    if (int e = ck(cudaStreamSynchronize(c->stream), "iterate")) return e;
    if (c->tracing) trace_collect_graph(c, *g, base, c->h_status->iters);
    if (c->h_status->done || c->h_status->timeout) break;
    chunk = std::min(chunk * 2, maxchunk);
  }
  c->last_iters = c->h_status->iters;
  c->last_residual = c->h_status->last_r;
  if (c->h_status->timeout) {
    set_error(persistent ? "a grid barrier of the persistent solve ran out of its wait limit"
                         : "a bounded device-side wait ran out in the tensor-core transform");
    return RF_ERR_TIMEOUT;
  }
  if (c->h_status->nonfinite) {
    set_error("convergence measure is not finite");
    return RF_ERR_NONFINITE;
  }
  if (c->h_status->diverged) {
    set_error("the fixed-point iteration diverged: the convergence measure grew past 1e4 times "
              "its smallest value (the reference medium does not bound the phases enough for "
              "the basic scheme to contract)");
    return RF_ERR_DIVERGED;
  }
  return RF_OK;
}

int finish(rf_ctx* c, int commit, double* sbar) {
  if (int e = launch_final(c, commit)) return e;
  if (int e = ck(cudaMemcpyAsync(c->h_sbar, c->d_sbar, 8 * sizeof(double),
                                 cudaMemcpyDeviceToHost, c->stream), "read sbar"))
    return e;
  if (int e = ck(cudaStreamSynchronize(c->stream), "final pass")) return e;
  trace_collect(c, 0);
  c->fields_valid = true;
  if (commit) c->last_viol = c->h_sbar[6];
  for (int i = 0; i < 6; ++i) {
    if (!std::isfinite(c->h_sbar[i])) {
      set_error("homogenised stress is not finite");
      return RF_ERR_NONFINITE;
    }
    c->last_sbar[i] = c->h_sbar[i];
    if (sbar) sbar[i] = c->h_sbar[i];
  }
  return RF_OK;
}

int check_mixed(const rf_ctx* c, const int32_t* control, const double* target) {
  for (int i = 0; i < 6; ++i) {
    if (control[i] != 0 && control[i] != 1) return invalid("mixed control: entries must be 0 or 1");
    if (!std::isfinite(target[i])) {
      set_error("mixed control: target is not finite");
      return RF_ERR_NONFINITE;
    }
  }
  if (c->dim == 2)
    for (int i = 2; i < 5; ++i)
      if (control[i] || target[i] != 0.0)
        return invalid("mixed control in 2D (plane strain): components 33, 23, 13 are strains "
                       "fixed at zero");
  return RF_OK;
}

int check_macro(const rf_ctx* c, const double* m) {
  for (int i = 0; i < 6; ++i)
    if (!std::isfinite(m[i])) {
      set_error("macroscopic strain is not finite");
      return RF_ERR_NONFINITE;
    }
  if (c->dim == 2 && (m[2] != 0.0 || m[3] != 0.0 || m[4] != 0.0))
    return invalid("2D (plane strain): macro strain components 33, 23, 13 must be zero");
  return RF_OK;
}

}  // namespace

extern "C" {

const char* rf_last_error(void) { return rfk::g_err.c_str(); }

int rf_create(rf_ctx** out, const rf_grid* grid, int32_t n_phases, const rf_phase* phases,
              const uint8_t* phase_map, const rf_options* opt, void* stream) {
  set_error("");
  if (!out || !grid || !phases || !phase_map || !opt) return invalid("rf_create: null argument");
  *out = nullptr;
  if (grid->dim != 2 && grid->dim != 3) return invalid("grid: dim must be 2 or 3");
  for (int j = 0; j < 3; ++j)
    if (grid->n[j] < 1 || grid->n[j] > 4096) return invalid("grid: sizes must be in [1, 4096]");
  if (grid->dim == 2 && grid->n[2] != 1) return invalid("grid: Nz must be 1 in 2D");
  const long long N = (long long)grid->n[0] * grid->n[1] * grid->n[2];
  if (N >= (1LL << 31)) return invalid("grid: too many voxels");
  if (n_phases < 1 || n_phases > kMaxPhases) return invalid("n_phases must be in [1, 16]");
  for (int p = 0; p < n_phases; ++p) {
    const rf_phase& ph = phases[p];
    if (!std::isfinite(ph.lambda) || !std::isfinite(ph.mu) ||
        (ph.plastic && (!std::isfinite(ph.sigma_y0) || !std::isfinite(ph.hardening)))) {
      set_error("phase moduli must be finite");
      return RF_ERR_NONFINITE;
    }
    if (!(ph.mu > 0.0) || !(ph.lambda + 2.0 * ph.mu / 3.0 > 0.0))
      return invalid("phase moduli must satisfy mu > 0 and lambda + 2 mu / 3 > 0");
    if (ph.plastic && (!(ph.sigma_y0 > 0.0) || !(ph.hardening >= 0.0) ||
                       !std::isfinite(ph.sigma_y0) || !std::isfinite(ph.hardening)))
      return invalid("plastic phase needs sigma_y0 > 0 and H >= 0");
  }
  if (!(opt->tol >= 0.0) || opt->max_iter < 1) return invalid("options: tol >= 0, max_iter >= 1");
  if (opt->green != RF_GREEN_ROTATED && opt->green != RF_GREEN_CONTINUOUS)
    return invalid("options: unknown green operator");
  if (opt->ref_medium != RF_REF_MINMAX && opt->ref_medium != RF_REF_VOLUME)
    return invalid("options: unknown reference medium rule");
  if (opt->precision != RF_PREC_FP32 && opt->precision != RF_PREC_SPLIT_BF16 &&
      opt->precision != RF_PREC_SPLIT_TF32)
    return invalid("options: unknown precision");
  if (opt->transform != RF_TRANSFORM_DFT && opt->transform != RF_TRANSFORM_FFT)
    return invalid("options: unknown transform");
  if (opt->fft_rows < 0 || opt->fft_rows > 64 || opt->fft_cols < 0 || opt->fft_cols > 64)
    return invalid("options: fft_rows and fft_cols in [0, 64]");
  if (opt->fft_row_blocks < 0) return invalid("options: fft_row_blocks >= 0");
  if (opt->fft_row_warps != -1 && opt->fft_row_warps != 0 && opt->fft_row_warps != 2 &&
      opt->fft_row_warps != 4 && opt->fft_row_warps != 8)
    return invalid("options: fft_row_warps -1, 0, 2, 4 or 8");
  if ((opt->fft_row_warps == 8) != (opt->fft_fuse == 4 || opt->fft_fuse == 5) &&
      opt->fft_row_warps != 0)
    return invalid("options: fft_row_warps 8 goes with fft_fuse 4 or 5 and only with them");
  if (opt->wait_limit < 0 || (opt->stall_test != 0 && opt->stall_test != 1))
    return invalid("options: wait_limit >= 0, stall_test 0 or 1");
  if (opt->stall_test && opt->precision == RF_PREC_FP32)
    return invalid("options: stall_test applies to the split-precision modes only");
  if (opt->fft_fuse < -1 || opt->fft_fuse > 5 || opt->fft_fuse_kx < 0 || opt->fft_fuse_kx > 16)
    return invalid("options: fft_fuse in {-1, 0, 1, 2, 3, 4, 5}, fft_fuse_kx in [0, 16]");
  if (opt->fft_fuse >= 1 && (opt->transform != RF_TRANSFORM_FFT || grid->dim != 2))
    return invalid("options: fft_fuse 1 to 5 needs the FFT transform on a 2D grid");
  if (opt->fft_fuse == 5 && (grid->n[0] != 1024 || grid->n[1] != 1024 ||
                             (opt->fft_row_warps != 0 && opt->fft_row_warps != 8)))
    return invalid("options: fft_fuse 5 needs a 1024 x 1024 grid and the warp-FFT row kernel");
  if (opt->fft_fuse == 4 && (grid->n[0] != 1024 || grid->n[1] != 1024 || opt->fft_fuse_kx > 2 ||
                             (opt->fft_row_warps != 0 && opt->fft_row_warps != 8)))
    return invalid("options: fft_fuse 4 needs a 1024 x 1024 grid, fft_fuse_kx 0, 1 or 2 and "
                   "the warp-FFT row kernel");
  if (opt->transform == RF_TRANSFORM_FFT) {
    // 2^b or 3 * 2^b (the FFT stages are radix 16, 4, 2 and one radix-3)
    auto pow2 = [](int v) {
      const int p = (v % 3 == 0) ? v / 3 : v;
      return v >= 2 && p >= 1 && (p & (p - 1)) == 0;
    };
    if (opt->precision != RF_PREC_FP32)
      return invalid("options: the FFT transform runs in FP32 precision only");
    if (!pow2(grid->n[0]) || !pow2(grid->n[1]) || (grid->dim == 3 && !pow2(grid->n[2])))
      return invalid("options: the FFT transform needs grid sizes 2^b or 3 * 2^b (>= 2)");
  }

  rf_ctx* c = new rf_ctx();
  cudaGetDevice(&c->dev);
  c->dim = grid->dim;
  c->nx = grid->n[0];
  c->ny = grid->n[1];
  c->nz = grid->n[2];
  c->N = N;
  c->rows = c->ny * c->nz;
  c->nc = c->dim == 2 ? 3 : 6;
  c->opt = *opt;
  c->stream = static_cast<cudaStream_t>(stream);
  init_attributes(c->dev);
  if (!c->stream) {
    // updates are replayed as CUDA graphs, which cannot be captured on the legacy stream
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      set_error("rf_create: cannot create a stream");
      return RF_ERR_CUDA;
    }
    c->own_stream = true;
  }
  c->n_phases = n_phases;
  bool any_plastic = false;
  for (int p = 0; p < n_phases; ++p) {
    c->phases[p] = phases[p];
    DevPhase& d = c->law.ph[p];
    d.lam = (float)phases[p].lambda;
    d.mu = (float)phases[p].mu;
    d.plastic = phases[p].plastic ? 1 : 0;
    d.sy = d.plastic ? (float)phases[p].sigma_y0 : 0.f;
    d.H = d.plastic ? (float)phases[p].hardening : 0.f;
    d.r3muH = d.plastic ? (float)(1.0 / (3.0 * phases[p].mu + phases[p].hardening)) : 0.f;
    any_plastic = any_plastic || d.plastic;
  }
  c->has_plastic = any_plastic;
  c->law.has_plastic = any_plastic;
  c->ns = any_plastic ? (c->dim == 2 ? 4 : 7) : 0;
  int err = dalloc(&c->d_phase, N, "phase map");
  if (!err && c->ns) err = dalloc(&c->d_state, (size_t)c->ns * N, "state");
  if (!err) err = dalloc(&c->d_twx, rfk::fftc::table_len(c->nx), "tables");
  if (!err) err = dalloc(&c->d_twy, rfk::fftc::table_len(c->ny), "tables");
  if (!err) err = dalloc(&c->d_twz, rfk::fftc::table_len(c->nz), "tables");
  if (!err) err = dalloc(&c->d_status, 1, "status");
  if (!err) err = dalloc(&c->d_sbar, 8, "sbar");
  if (!err) err = dalloc(&c->d_eps, 6 * (size_t)N, "fields");
  if (!err) err = dalloc(&c->d_sig, 6 * (size_t)N, "fields");
  if (!err) err = dalloc(&c->d_alpha, (size_t)N, "fields");
  if (!err) err = dalloc(&c->d_err, kErrBlocks + 2, "error partials");
  if (!err) err = ck(cudaMallocHost(&c->h_status, sizeof(Status)), "pinned");
  if (!err) err = ck(cudaMallocHost(&c->h_sbar, 8 * sizeof(double)), "pinned");
  if (!err)
    err = ck(cudaMemcpyAsync(c->d_phase, phase_map, N, cudaMemcpyHostToDevice, c->stream),
             "upload phase map");
  if (!err && c->d_state)
    err = ck(cudaMemsetAsync(c->d_state, 0, sizeof(float) * c->ns * N, c->stream), "state");
  if (!err) err = ck(cudaMemsetAsync(c->d_status, 0, sizeof(Status), c->stream), "status");
  if (!err) err = launch_setup_tables(c);
  if (!err) err = update_reference(c);
  if (err) {
    std::string keep = g_err;
    rf_destroy(c);
    g_err = keep;
    return err;
  }
  *out = c;
  return RF_OK;
}

int rf_set_phase_map(rf_ctx* c, const uint8_t* pm) {
  if (!c || !pm) return invalid("rf_set_phase_map: null argument");
  DeviceGuard dg(c->dev);
  rf_destroy(c->compat);   // the full-set context holds the old phase map
  c->compat = nullptr;
  if (int e = ck(cudaMemcpyAsync(c->d_phase, pm, c->N, cudaMemcpyHostToDevice, c->stream),
                 "upload phase map"))
    return e;
  free_graphs(c);   // the graphs hold the reference medium by value
  if (int e = update_reference(c)) return e;
  return reset_path_state(c);
}

int rf_set_phase_map_device(rf_ctx* c, const uint8_t* d_pm) {
  if (!c || !d_pm) return invalid("rf_set_phase_map_device: null argument");
  DeviceGuard dg(c->dev);
  rf_destroy(c->compat);
  c->compat = nullptr;
  if (int e = ck(cudaMemcpyAsync(c->d_phase, d_pm, c->N, cudaMemcpyDeviceToDevice, c->stream),
                 "copy phase map"))
    return e;
  free_graphs(c);
  if (int e = update_reference(c)) return e;
  return reset_path_state(c);
}

int rf_set_pattern(rf_ctx* c, const int32_t* freqs, int64_t K) {
  if (!c || !freqs) return invalid("rf_set_pattern: null argument");
  if (K < 1 || K > c->N) return invalid("rf_set_pattern: K must be in [1, N]");
  DeviceGuard dg(c->dev);
  const int n[3] = {c->nx, c->ny, c->nz};
  // signed range (-N/2, N/2]: -(N-1)/2 <= k <= N/2 with integer division
  auto in_range = [](int k, int nn) { return k >= -((nn - 1) / 2) && k <= nn / 2; };
  // frequencies as unique linear keys (offset signed indices); duplicate, conjugate and
  // position lookups go through a dense index over the key space for grids up to 4 Mi voxels,
  // else through one sorted key vector and binary searches
  auto key = [&](int kx, int ky, int kz) {
    return ((long long)(kz + (n[2] - 1) / 2) * n[1] + (ky + (n[1] - 1) / 2)) * n[0] +
           (kx + (n[0] - 1) / 2);
  };
  const bool dense = c->N <= (4LL << 20);
  std::vector<int32_t> at;      // dense: pattern index of each key, -1 if absent
  std::vector<long long> keys;  // sparse: sorted keys
  if (dense) at.assign((size_t)c->N, -1);
  else keys.resize(K);
  int zeros = 0;
  for (long long p = 0; p < K; ++p) {
    const int kx = freqs[3 * p], ky = freqs[3 * p + 1], kz = freqs[3 * p + 2];
    if (!in_range(kx, n[0]) || !in_range(ky, n[1]) || !in_range(kz, n[2]))
      return invalid("rf_set_pattern: frequency outside the signed range (-N/2, N/2]");
    if (kx == 0 && ky == 0 && kz == 0) ++zeros;
    const long long k = key(kx, ky, kz);
    if (dense) {
      if (at[k] >= 0) return invalid("rf_set_pattern: duplicate frequency");
      at[k] = (int32_t)p;
    } else {
      keys[p] = k;
    }
  }
  if (!dense) {
    std::sort(keys.begin(), keys.end());
    if (std::adjacent_find(keys.begin(), keys.end()) != keys.end())
      return invalid("rf_set_pattern: duplicate frequency");
  }
  if (zeros != 1) return invalid("rf_set_pattern: the zero frequency must be present");
  auto conj = [&](int kx, int ky, int kz) {
    return std::make_tuple(signed_of(wrapi(-kx, n[0]), n[0]), signed_of(wrapi(-ky, n[1]), n[1]),
                           signed_of(wrapi(-kz, n[2]), n[2]));
  };
  auto present = [&](long long k) {
    return dense ? at[k] >= 0 : std::binary_search(keys.begin(), keys.end(), k);
  };
  for (long long p = 0; p < K; ++p) {
    auto [cx, cy, cz] = conj(freqs[3 * p], freqs[3 * p + 1], freqs[3 * p + 2]);
    if (!present(key(cx, cy, cz)))
      return invalid("rf_set_pattern: pattern is not closed under k -> -k");
  }
  // half set: kx >= 0, sorted by (kx, ky, kz) through packed keys
  auto hkey = [&](int kx, int ky, int kz) {
    return ((long long)kx * n[1] + (ky + (n[1] - 1) / 2)) * n[2] + (kz + (n[2] - 1) / 2);
  };
  std::vector<long long> hk_sorted;
  hk_sorted.reserve(K / 2 + 2);
  for (long long p = 0; p < K; ++p)
    if (freqs[3 * p] >= 0) hk_sorted.push_back(hkey(freqs[3 * p], freqs[3 * p + 1], freqs[3 * p + 2]));
  std::sort(hk_sorted.begin(), hk_sorted.end());
  std::vector<std::tuple<int, int, int>> H(hk_sorted.size());
  for (size_t h = 0; h < hk_sorted.size(); ++h) {
    const long long v = hk_sorted[h];
    const int kz = (int)(v % n[2]) - (n[2] - 1) / 2;
    const long long r = v / n[2];
    const int ky = (int)(r % n[1]) - (n[1] - 1) / 2;
    const int kx = (int)(r / n[1]);
    H[h] = std::make_tuple(kx, ky, kz);
  }
  std::vector<int> xs, ys, zs;
  for (auto& t : H) {
    xs.push_back(std::get<0>(t));
    ys.push_back(std::get<1>(t));
    zs.push_back(std::get<2>(t));
  }
  auto uniq = [](std::vector<int>& v) {
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
  };
  uniq(xs);
  uniq(ys);
  uniq(zs);
  free_pattern(c);
  c->K = K;
  c->Kh = (long long)H.size();
  c->Kx = (int)xs.size();
  c->Ky = (int)ys.size();
  c->Kz = (int)zs.size();
  c->pat.assign(freqs, freqs + 3 * K);
  // half-set position of each frequency: the dense index now holds h, else a binary search
  if (dense)
    for (long long h = 0; h < c->Kh; ++h) {
      auto [kx, ky, kz] = H[h];
      at[key(kx, ky, kz)] = (int32_t)h;
    }
  auto hpos = [&](const std::tuple<int, int, int>& t) {
    auto [kx, ky, kz] = t;
    if (dense) return (long long)at[key(kx, ky, kz)];
    return (long long)(std::lower_bound(hk_sorted.begin(), hk_sorted.end(), hkey(kx, ky, kz)) -
                       hk_sorted.begin());
  };
  c->map_h.assign(K, 0);
  c->map_conj.assign(K, 0);
  c->h_src.assign(c->Kh, -1);
  for (long long p = 0; p < K; ++p) {
    const int kx = freqs[3 * p], ky = freqs[3 * p + 1], kz = freqs[3 * p + 2];
    if (kx >= 0) {
      c->map_h[p] = hpos(std::make_tuple(kx, ky, kz));
      c->map_conj[p] = 0;
      c->h_src[c->map_h[p]] = p;
    } else {
      c->map_h[p] = hpos(conj(kx, ky, kz));
      c->map_conj[p] = 1;
    }
  }
  auto pos = [](const std::vector<int>& v, int x) {
    return (int)(std::lower_bound(v.begin(), v.end(), x) - v.begin());
  };
  const bool even_x = (c->nx % 2 == 0);
  std::vector<int> hk(4 * c->Kh);
  c->h_hidx.assign(c->Kh, HIdx{0, 0, 0, 0});
  for (long long h = 0; h < c->Kh; ++h) {
    auto [kx, ky, kz] = H[h];
    const bool self = (kx == 0) || (even_x && kx == c->nx / 2);
    hk[4 * h] = kx;
    hk[4 * h + 1] = ky;
    hk[4 * h + 2] = kz;
    hk[4 * h + 3] = self ? 1 : 2;
    c->h_hidx[h] = HIdx{pos(xs, kx), pos(ys, ky), pos(zs, kz), 0};
  }
  std::vector<int> kym(c->Ky), kzm(c->Kz);
  std::vector<float> fac(c->Kx);
  for (int i = 0; i < c->Ky; ++i) kym[i] = wrapi(ys[i], c->ny);
  for (int i = 0; i < c->Kz; ++i) kzm[i] = wrapi(zs[i], c->nz);
  for (int j = 0; j < c->Kx; ++j) {
    const bool self = (xs[j] == 0) || (even_x && xs[j] == c->nx / 2);
    fac[j] = (float)((self ? 1.0 : 2.0) / (double)c->N);
  }
  const int NCK = c->nc * c->Kx;
  c->rect = (long long)c->Kz * c->Ky * NCK;
  c->zero_base_idx = ((long long)(pos(zs, 0) * c->Ky + pos(ys, 0)) * c->nc) * c->Kx + pos(xs, 0);
  // split-K for the forward transforms so that the grid covers the GPU
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev);
  if (c->dim == 2) {
    const long long blocks = (long long)((NCK + 63) / 64) * ((c->Ky + 31) / 32);
    c->splitB = (int)std::max(1LL, std::min<long long>((2LL * sms + blocks - 1) / blocks,
                                                        std::max(1, c->ny / 64)));
    c->splitC = 1;
  } else {
    c->splitB = 1;
    const long long blocks = (long long)((c->Ky * NCK + 63) / 64) * ((c->Kz + 31) / 32);
    c->splitC = (int)std::max(1LL, std::min<long long>((2LL * sms + blocks - 1) / blocks,
                                                        std::max(1, c->nz / 64)));
  }
  // row kernel geometry
  c->row_R = std::max(1, std::min(16, 2048 / c->nx));
  auto smem_for = [&](int R) {
    return (size_t)c->nx * sizeof(float2) + (size_t)R * NCK * sizeof(float2) +
           (size_t)c->Kx * (sizeof(int) + sizeof(float)) + (size_t)R * c->nc * c->nx * sizeof(float) +
           64;
  };
  while (c->row_R > 1 && smem_for(c->row_R) > 160 * 1024) --c->row_R;
  if (smem_for(c->row_R) > 200 * 1024) return invalid("rf_set_pattern: pattern too wide for the row kernel");
  c->row_smem = smem_for(c->row_R);
  c->row_blocks = (c->rows + c->row_R - 1) / c->row_R;
  if (c->opt.transform == RF_TRANSFORM_FFT) {
    if (int e = fft_geometry(c)) return e;
    c->splitB = c->splitC = 1;
  }
  // the split-precision modes run the y and z transforms on the tensor cores, one output slice
  if (c->opt.precision != RF_PREC_FP32) c->splitB = c->splitC = 1;
  const int part_blocks = std::max(c->row_blocks, c->rows);   // any FFT row tile (R >= 1)
  const int splits = std::max(c->splitB, c->splitC);
  int err = palloc(c, &c->d_kx, c->Kx, "pattern");
  if (!err) err = palloc(c, &c->d_kym, c->Ky, "pattern");
  if (!err) err = palloc(c, &c->d_kzm, c->Kz, "pattern");
  if (!err) err = palloc(c, &c->d_fac, c->Kx, "pattern");
  if (!err) err = palloc(c, &c->d_hidx, c->Kh, "pattern");
  if (!err) err = palloc(c, &c->d_hn, c->Kh, "pattern");
  if (!err) err = palloc(c, &c->d_ER, c->rect, "coefficients");
  if (!err) err = palloc(c, &c->d_T1, (size_t)c->rows * NCK, "line transforms");
  if (!err) err = palloc(c, &c->d_T1p, (size_t)c->rows * NCK, "line transforms");
  if (!err && c->dim == 3) err = palloc(c, &c->d_T2, (size_t)c->nz * c->Ky * NCK, "line transforms");
  if (!err && c->dim == 3) err = palloc(c, &c->d_T2f, (size_t)c->nz * c->Ky * NCK, "line transforms");
  if (!err) err = palloc(c, &c->d_OUT, (size_t)splits * c->rect, "partials");
  // block partials of the convergence measure: Green kernel blocks, or column blocks of the
  // fused modes (<= NC Kx)
  if (!err)
    err = palloc(c, &c->d_part,
                 (size_t)std::max<long long>((c->Kh + kGammaBlock - 1) / kGammaBlock,
                                             (long long)c->nc * c->Kx),
                 "partials");
  const bool fuse_ok = c->opt.transform == RF_TRANSFORM_FFT && c->dim == 2 && c->opt.fft_fuse >= 0;
  if (!err && fuse_ok) {
    // half-pattern entries grouped by kx index (counting sort) for the fused column phase
    std::vector<int> jptr(c->Kx + 1, 0), jlist(std::max<long long>(c->Kh, 1));
    for (long long h = 0; h < c->Kh; ++h) ++jptr[c->h_hidx[h].j + 1];
    for (int j = 0; j < c->Kx; ++j) jptr[j + 1] += jptr[j];
    std::vector<int> fill(jptr.begin(), jptr.end() - 1);
    for (long long h = 0; h < c->Kh; ++h) jlist[fill[c->h_hidx[h].j]++] = (int)h;
    err = palloc(c, &c->d_jptr, jptr.size(), "pattern");
    if (!err) err = palloc(c, &c->d_jlist, jlist.size(), "pattern");
    if (!err) err = palloc(c, &c->d_jent, jlist.size(), "pattern");
    if (!err) err = palloc(c, &c->d_jn, jlist.size(), "pattern");
    if (!err)
      err = ck(cudaMemcpy(c->d_jptr, jptr.data(), sizeof(int) * jptr.size(), cudaMemcpyHostToDevice),
               "up");
    if (!err)
      err = ck(cudaMemcpy(c->d_jlist, jlist.data(), sizeof(int) * jlist.size(),
                          cudaMemcpyHostToDevice),
               "up");
  }
  if (!err) err = palloc(c, &c->d_counter, 1, "counter");
  if (!err) err = ck(cudaMemsetAsync(c->d_counter, 0, sizeof(unsigned), c->stream), "memset");
  if (!err) err = palloc(c, &c->d_sbar_part, (size_t)part_blocks * 6, "partials");
  if (!err) err = palloc(c, &c->d_viol_part, (size_t)part_blocks, "partials");
  if (!err) err = palloc(c, &c->d_warm, (size_t)c->Kh * 6, "warm");
  if (!err) err = palloc(c, &c->d_hk, hk.size(), "pattern");
  int* d_hk = c->d_hk;
  if (!err) err = ck(cudaMemcpyAsync(c->d_kx, xs.data(), sizeof(int) * c->Kx, cudaMemcpyHostToDevice, c->stream), "up");
  if (!err) err = ck(cudaMemcpyAsync(c->d_kym, kym.data(), sizeof(int) * c->Ky, cudaMemcpyHostToDevice, c->stream), "up");
  if (!err) err = ck(cudaMemcpyAsync(c->d_kzm, kzm.data(), sizeof(int) * c->Kz, cudaMemcpyHostToDevice, c->stream), "up");
  if (!err) err = ck(cudaMemcpyAsync(c->d_fac, fac.data(), sizeof(float) * c->Kx, cudaMemcpyHostToDevice, c->stream), "up");
  if (!err) err = ck(cudaMemcpyAsync(c->d_hidx, c->h_hidx.data(), sizeof(HIdx) * c->Kh, cudaMemcpyHostToDevice, c->stream), "up");
  if (!err) err = ck(cudaMemcpyAsync(d_hk, hk.data(), sizeof(int) * hk.size(), cudaMemcpyHostToDevice, c->stream), "up");
  if (!err) err = launch_hinfo(c, d_hk, c->Kh);
  if (!err && c->d_jent) err = launch_gather_jentries(c);
  if (!err && fuse_ok && c->dim == 2) {
    // persistent solve: barrier words and a first geometry (needed when forced, optional for
    // the autotuner)
    const int pe = persist_setup(c);
    if (pe && c->opt.fft_fuse == 3) err = pe;
    else if (pe) set_error("");
  }
  if (!err && c->opt.precision != RF_PREC_FP32) err = tc_setup(c);
  if (!err) err = ck(cudaMemsetAsync(c->d_OUT, 0, sizeof(float2) * splits * c->rect, c->stream), "memset");
  if (!err && c->opt.transform == RF_TRANSFORM_FFT) err = fft_autotune(c);
  if (!err) err = ck(cudaStreamSynchronize(c->stream), "pattern setup");
  if (!err) {
    // frequency kinds back to the host copy (zero / null flags)
    err = ck(cudaMemcpy(c->h_hidx.data(), c->d_hidx, sizeof(HIdx) * c->Kh, cudaMemcpyDeviceToHost),
             "read kinds");
  }
  if (err) {
    free_pattern(c);
    return err;
  }
  c->have_pattern = true;
  return reset_path_state(c);
}

int rf_reset_path(rf_ctx* c) {
  if (!c) return invalid("rf_reset_path: null context");
  DeviceGuard dg(c->dev);
  return reset_path_state(c);
}

int rf_solve(rf_ctx* c, const double macro[6], const float* warm, double hom_stress[6],
             int32_t* iters, double* residual) {
  if (!c || !macro) return invalid("rf_solve: null argument");
  if (!c->have_pattern) {
    set_error("rf_solve: no pattern set");
    return RF_ERR_STATE;
  }
  if (int e = check_macro(c, macro)) return e;
  DeviceGuard dg(c->dev);
  if (int e = init_status(c, macro)) return e;
  if (warm) {
    std::vector<float2> w6((size_t)c->Kh * 6);
    for (long long h = 0; h < c->Kh; ++h) {
      const long long p = c->h_src[h];
      for (int i = 0; i < 6; ++i)
        w6[h * 6 + i] = make_float2(warm[(p * 6 + i) * 2], warm[(p * 6 + i) * 2 + 1]);
    }
    if (int e = ck(cudaMemcpyAsync(c->d_warm, w6.data(), sizeof(float2) * w6.size(),
                                   cudaMemcpyHostToDevice, c->stream), "upload warm"))
      return e;
    if (int e = ck(cudaMemsetAsync(c->d_ER, 0, sizeof(float2) * c->rect, c->stream), "memset"))
      return e;
    if (int e = launch_warm_project(c, c->d_warm, macro)) return e;
    // the staging vector must outlive the copy
    if (int e = ck(cudaStreamSynchronize(c->stream), "warm")) return e;
  } else {
    if (int e = launch_reset_er(c, macro, 0.0)) return e;
  }
  int st = run_iterations(c);
  if (st < 0) return st;
  if (int e = finish(c, 0, hom_stress)) return e;
  for (int i = 0; i < 6; ++i) {
    c->prev_macro[i] = macro[i];
    c->prev_sbar[i] = c->last_sbar[i];
  }
  if (iters) *iters = c->last_iters;
  if (residual) *residual = c->last_residual;
  return c->last_residual < c->opt.tol ? RF_OK : RF_NOT_CONVERGED;
}

int rf_solve_mixed(rf_ctx* c, const int32_t control[6], const double target[6], const float* warm,
                   double hom_stress[6], double hom_strain[6], int32_t* iters, double* residual) {
  if (!c || !control || !target) return invalid("rf_solve_mixed: null argument");
  if (!c->have_pattern) {
    set_error("rf_solve_mixed: no pattern set");
    return RF_ERR_STATE;
  }
  if (int e = check_mixed(c, control, target)) return e;
  DeviceGuard dg(c->dev);
  double E0[6];
  mixed_start(c, control, target, E0);
  if (int e = init_status(c, E0, control, target)) return e;
  if (warm) {
    std::vector<float2> w6((size_t)c->Kh * 6);
    for (long long h = 0; h < c->Kh; ++h) {
      const long long p = c->h_src[h];
      for (int i = 0; i < 6; ++i)
        w6[h * 6 + i] = make_float2(warm[(p * 6 + i) * 2], warm[(p * 6 + i) * 2 + 1]);
    }
    if (int e = ck(cudaMemcpyAsync(c->d_warm, w6.data(), sizeof(float2) * w6.size(),
                                   cudaMemcpyHostToDevice, c->stream), "upload warm"))
      return e;
    if (int e = ck(cudaMemsetAsync(c->d_ER, 0, sizeof(float2) * c->rect, c->stream), "memset"))
      return e;
    if (int e = launch_warm_project(c, c->d_warm, E0)) return e;
    if (int e = ck(cudaStreamSynchronize(c->stream), "warm")) return e;
  } else {
    if (int e = launch_reset_er(c, E0, 0.0)) return e;
  }
  int st = run_iterations(c);
  if (st < 0) return st;
  double E[6];
  for (int i = 0; i < 6; ++i) E[i] = c->h_status->ebar[i];
  if (int e = finish(c, 0, hom_stress)) return e;
  for (int i = 0; i < 6; ++i) {
    c->prev_macro[i] = E[i];
    c->prev_sbar[i] = c->last_sbar[i];
    if (hom_strain) hom_strain[i] = E[i];
  }
  if (iters) *iters = c->last_iters;
  if (residual) *residual = c->last_residual;
  return c->last_residual < c->opt.tol ? RF_OK : RF_NOT_CONVERGED;
}

int rf_solve_path_mixed(rf_ctx* c, const int32_t control[6], int32_t n_steps, const double* path,
                        double* hom_stress, double* hom_strain, int32_t* iters,
                        double* residuals) {
  if (!c || !control || !path || n_steps < 1) return invalid("rf_solve_path_mixed: invalid arguments");
  if (!c->have_pattern) {
    set_error("rf_solve_path_mixed: no pattern set");
    return RF_ERR_STATE;
  }
  for (int n = 0; n < n_steps; ++n)
    if (int e = check_mixed(c, control, path + 6 * n)) return e;
  DeviceGuard dg(c->dev);
  int status = RF_OK;
  for (int n = 0; n < n_steps; ++n) {
    const double* t = path + 6 * n;
    // start: the last converged strain plus the reference medium's response to the increment
    // of the targets (stress increments measured from the last homogenised stress)
    double incr[6], d[6], E0[6];
    for (int i = 0; i < 6; ++i) incr[i] = control[i] ? t[i] - c->prev_sbar[i] : t[i] - c->prev_macro[i];
    mixed_start(c, control, incr, d);
    mixed_start(c, control, t, E0);
    if (int e = init_status(c, E0, control, t)) return e;
    if (int e = launch_reset_er(c, d, 1.0)) return e;
    int st = run_iterations(c);
    if (st < 0) return st;
    double E[6];
    for (int i = 0; i < 6; ++i) E[i] = c->h_status->ebar[i];
    if (int e = finish(c, 1, hom_stress ? hom_stress + 6 * n : nullptr)) return e;
    for (int i = 0; i < 6; ++i) {
      c->prev_macro[i] = E[i];
      c->prev_sbar[i] = c->last_sbar[i];
      if (hom_strain) hom_strain[6 * n + i] = E[i];
    }
    if (iters) iters[n] = c->last_iters;
    if (residuals) residuals[n] = c->last_residual;
    if (!(c->last_residual < c->opt.tol)) status = RF_NOT_CONVERGED;
  }
  return status;
}

int rf_solve_path(rf_ctx* c, int32_t n_steps, const double* path, double* hom_stress,
                  int32_t* iters, double* residuals) {
  if (!c || !path || n_steps < 1) return invalid("rf_solve_path: invalid arguments");
  if (!c->have_pattern) {
    set_error("rf_solve_path: no pattern set");
    return RF_ERR_STATE;
  }
  for (int n = 0; n < n_steps; ++n)
    if (int e = check_macro(c, path + 6 * n)) return e;
  DeviceGuard dg(c->dev);
  int status = RF_OK;
  for (int n = 0; n < n_steps; ++n) {
    const double* m = path + 6 * n;
    double d[6];
    for (int i = 0; i < 6; ++i) d[i] = m[i] - c->prev_macro[i];
    if (int e = init_status(c, m)) return e;
    if (int e = launch_reset_er(c, d, 1.0)) return e;
    int st = run_iterations(c);
    if (st < 0) return st;
    if (int e = finish(c, 1, hom_stress ? hom_stress + 6 * n : nullptr)) return e;
    for (int i = 0; i < 6; ++i) {
      c->prev_macro[i] = m[i];
      c->prev_sbar[i] = c->last_sbar[i];
    }
    if (iters) iters[n] = c->last_iters;
    if (residuals) residuals[n] = c->last_residual;
    if (!(c->last_residual < c->opt.tol)) status = RF_NOT_CONVERGED;
  }
  return status;
}

int rf_get_fields(rf_ctx* c, float* strain, float* stress, float* eps_p_acc) {
  if (!c) return invalid("rf_get_fields: null context");
  if (!c->fields_valid) {
    set_error("rf_get_fields: no solve has produced fields yet");
    return RF_ERR_STATE;
  }
  DeviceGuard dg(c->dev);
  if (strain)
    if (int e = ck(cudaMemcpyAsync(strain, c->d_eps, sizeof(float) * 6 * c->N,
                                   cudaMemcpyDeviceToHost, c->stream), "copy strain"))
      return e;
  if (stress)
    if (int e = ck(cudaMemcpyAsync(stress, c->d_sig, sizeof(float) * 6 * c->N,
                                   cudaMemcpyDeviceToHost, c->stream), "copy stress"))
      return e;
  if (eps_p_acc)
    if (int e = ck(cudaMemcpyAsync(eps_p_acc, c->d_alpha, sizeof(float) * c->N,
                                   cudaMemcpyDeviceToHost, c->stream), "copy alpha"))
      return e;
  return ck(cudaStreamSynchronize(c->stream), "get fields");
}

int rf_get_reduced_strain(rf_ctx* c, float* coeffs) {
  if (!c || !coeffs) return invalid("rf_get_reduced_strain: null argument");
  if (!c->have_pattern) {
    set_error("rf_get_reduced_strain: no pattern set");
    return RF_ERR_STATE;
  }
  DeviceGuard dg(c->dev);
  std::vector<float2> er(c->rect);
  if (int e = ck(cudaMemcpyAsync(er.data(), c->d_ER, sizeof(float2) * c->rect,
                                 cudaMemcpyDeviceToHost, c->stream), "copy coefficients"))
    return e;
  if (int e = ck(cudaStreamSynchronize(c->stream), "sync")) return e;
  for (long long p = 0; p < c->K; ++p) {
    const HIdx& hi = c->h_hidx[c->map_h[p]];
    const long long base = ((long long)(hi.iz * c->Ky + hi.iy) * c->nc) * c->Kx + hi.j;
    const float sg = c->map_conj[p] ? -1.f : 1.f;
    for (int i = 0; i < 6; ++i) {
      int comp = -1;
      if (c->nc == 6) comp = i;
      else if (i == 0) comp = 0;
      else if (i == 1) comp = 1;
      else if (i == 5) comp = 2;
      float re = 0.f, im = 0.f;
      if (comp >= 0) {
        const float2 v = er[base + (long long)comp * c->Kx];
        re = v.x;
        im = sg * v.y;
      }
      coeffs[(p * 6 + i) * 2] = re;
      coeffs[(p * 6 + i) * 2 + 1] = im;
    }
  }
  return RF_OK;
}

struct StateHeader {
  uint64_t magic;
  int64_t N, rect;
  int32_t nc, ns;
  double prev_macro[6];
  double prev_sbar[6];
};

int rf_get_state(rf_ctx* c, void* buf, size_t* bytes) {
  if (!c || !bytes) return invalid("rf_get_state: null argument");
  if (!c->have_pattern) {
    set_error("rf_get_state: no pattern set");
    return RF_ERR_STATE;
  }
  const size_t need = sizeof(StateHeader) + sizeof(float2) * c->rect +
                      sizeof(float) * (size_t)c->ns * c->N;
  if (!buf) {
    *bytes = need;
    return RF_OK;
  }
  if (*bytes < need) return invalid("rf_get_state: buffer too small");
  DeviceGuard dg(c->dev);
  StateHeader h{0x52465354415446ull, c->N, c->rect, c->nc, c->ns, {0}, {0}};
  for (int i = 0; i < 6; ++i) {
    h.prev_macro[i] = c->prev_macro[i];
    h.prev_sbar[i] = c->prev_sbar[i];
  }
  char* p = static_cast<char*>(buf);
  std::memcpy(p, &h, sizeof h);
  p += sizeof h;
  if (int e = ck(cudaMemcpyAsync(p, c->d_ER, sizeof(float2) * c->rect, cudaMemcpyDeviceToHost,
                                 c->stream), "copy state"))
    return e;
  p += sizeof(float2) * c->rect;
  if (c->ns)
    if (int e = ck(cudaMemcpyAsync(p, c->d_state, sizeof(float) * c->ns * c->N,
                                   cudaMemcpyDeviceToHost, c->stream), "copy state"))
      return e;
  *bytes = need;
  return ck(cudaStreamSynchronize(c->stream), "get state");
}

int rf_set_state(rf_ctx* c, const void* buf, size_t bytes) {
  if (!c || !buf) return invalid("rf_set_state: null argument");
  if (!c->have_pattern) {
    set_error("rf_set_state: no pattern set");
    return RF_ERR_STATE;
  }
  StateHeader h;
  if (bytes < sizeof h) return invalid("rf_set_state: buffer too small");
  std::memcpy(&h, buf, sizeof h);
  const size_t need = sizeof(StateHeader) + sizeof(float2) * c->rect +
                      sizeof(float) * (size_t)c->ns * c->N;
  if (h.magic != 0x52465354415446ull || h.N != c->N || h.rect != c->rect || h.nc != c->nc ||
      h.ns != c->ns || bytes < need)
    return invalid("rf_set_state: state does not match this context");
  DeviceGuard dg(c->dev);
  const char* p = static_cast<const char*>(buf) + sizeof h;
  if (int e = ck(cudaMemcpyAsync(c->d_ER, p, sizeof(float2) * c->rect, cudaMemcpyHostToDevice,
                                 c->stream), "restore"))
    return e;
  p += sizeof(float2) * c->rect;
  if (c->ns)
    if (int e = ck(cudaMemcpyAsync(c->d_state, p, sizeof(float) * c->ns * c->N,
                                   cudaMemcpyHostToDevice, c->stream), "restore"))
      return e;
  for (int i = 0; i < 6; ++i) {
    c->prev_macro[i] = h.prev_macro[i];
    c->prev_sbar[i] = h.prev_sbar[i];
  }
  c->fields_valid = false;
  return ck(cudaStreamSynchronize(c->stream), "set state");
}

int rf_get_info(const rf_ctx* c, rf_info* info) {
  if (!c || !info) return invalid("rf_get_info: null argument");
  info->K = c->K;
  info->K_half = c->Kh;
  info->Kx = c->Kx;
  info->Ky = c->Ky;
  info->Kz = c->Kz;
  info->last_iters = c->last_iters;
  info->last_residual = c->last_residual;
  info->kernel_launches = c->launches;
  info->j2_max_violation = c->last_viol;
  info->lambda0 = c->lam0;
  info->mu0 = c->mu0;
  const bool fft = c->opt.transform == RF_TRANSFORM_FFT;
  info->fft_rows = fft ? c->fft_R : 0;
  info->fft_row_threads = fft ? c->fft_row_threads : 0;
  info->fft_cols = fft ? c->fft_C : 0;
  info->fft_col_threads = fft ? c->fft_col_threads : 0;
  info->fft_fused = c->fft_colmode;
  info->fft_fuse_kx = c->fft_colmode == kColFused ? c->fft_M
                      : (c->fft_colmode == kColWarp || c->fft_colmode == kColPersistW)
                          ? c->fft_colw_M : 0;
  info->fft_fuse_threads = c->fft_colmode == kColFused ? c->fft_M_threads : 0;
  info->fft_row_blocks = fft ? c->fft_blocks : 0;
  if (c->fft_colmode == kColPersistent) {
    info->fft_row_blocks = c->persist_G;
    info->fft_row_threads = c->persist_threads;
    info->fft_rows = (c->rows + c->persist_G - 1) / c->persist_G;
  }
  info->fft_row_warps = fft && c->fft_colmode != kColPersistent ? c->fft_row_warps : 0;
  info->reserved = 0;
  return RF_OK;
}

int rf_set_tracing(rf_ctx* c, int on) {
  if (!c) return invalid("rf_set_tracing: null context");
  c->tracing = on != 0;
  return RF_OK;
}

int rf_get_stage_times(const rf_ctx* c, double ms_total[8], int64_t counts[8]) {
  if (!c || !ms_total || !counts) return invalid("rf_get_stage_times: null argument");
  for (int i = 0; i < 8; ++i) {
    ms_total[i] = c->stage_ms[i];
    counts[i] = c->stage_n[i];
  }
  return RF_OK;
}

int rf_reset_stage_times(rf_ctx* c) {
  if (!c) return invalid("rf_reset_stage_times: null context");
  for (int i = 0; i < 8; ++i) {
    c->stage_ms[i] = 0.0;
    c->stage_n[i] = 0;
  }
  return RF_OK;
}

int rf_destroy(rf_ctx* c) {
  if (!c) return RF_OK;
  DeviceGuard dg(c->dev);
  rf_destroy(c->compat);
  c->compat = nullptr;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  trace_collect(c, 0);
  free_graphs(c);
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  c->ev_pool.clear();
  free_pattern(c);
  release_pattern_buffers(c);
  dfree(c->d_phase);
  dfree(c->d_state);
  dfree(c->d_twx);
  dfree(c->d_twy);
  dfree(c->d_twz);
  dfree(c->d_status);
  dfree(c->d_sbar);
  dfree(c->d_eps);
  dfree(c->d_sig);
  dfree(c->d_alpha);
  dfree(c->d_err);
  if (c->h_status) cudaFreeHost(c->h_status);
  if (c->h_sbar) cudaFreeHost(c->h_sbar);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return RF_OK;
}

int rf_compat(rf_ctx* c, double hom_stress[6]) {
  if (!c) return invalid("rf_compat: null context");
  if (!c->have_pattern || !c->fields_valid) {
    set_error("rf_compat: no solve has produced a reduced solution yet");
    return RF_ERR_STATE;
  }
  DeviceGuard dg(c->dev);
  if (!c->compat) {
    // the full set of frequencies on the same grid, phases and Green operator; FFT transforms
    // where the sizes allow, one update per solve
    std::vector<uint8_t> pm((size_t)c->N);
    if (int e = ck(cudaMemcpyAsync(pm.data(), c->d_phase, c->N, cudaMemcpyDeviceToHost,
                                   c->stream), "compat: phase map"))
      return e;
    if (int e = ck(cudaStreamSynchronize(c->stream), "compat: phase map")) return e;
    auto fft_ok = [](int v) {
      const int p = (v % 3 == 0) ? v / 3 : v;
      return v >= 2 && (p & (p - 1)) == 0;
    };
    rf_options o{};
    o.tol = 0.0;
    o.max_iter = 1;
    o.green = c->opt.green;
    o.ref_medium = c->opt.ref_medium;
    o.precision = RF_PREC_FP32;
    o.transform = (fft_ok(c->nx) && fft_ok(c->ny) && (c->dim == 2 || fft_ok(c->nz)))
                      ? RF_TRANSFORM_FFT : RF_TRANSFORM_DFT;
    const rf_grid g{c->dim, {c->nx, c->ny, c->nz}};
    rf_ctx* f = nullptr;
    if (int e = rf_create(&f, &g, c->n_phases, c->phases, pm.data(), &o, c->stream)) return e;
    std::vector<int32_t> full((size_t)3 * c->N);
    long long p = 0;
    for (int iz = 0; iz < c->nz; ++iz)
      for (int iy = 0; iy < c->ny; ++iy)
        for (int ix = 0; ix < c->nx; ++ix, ++p) {
          full[3 * p] = ix - (c->nx - 1) / 2;
          full[3 * p + 1] = iy - (c->ny - 1) / 2;
          full[3 * p + 2] = iz - (c->nz - 1) / 2;
        }
    if (int e = rf_set_pattern(f, full.data(), c->N)) {
      std::string keep = g_err;
      rf_destroy(f);
      g_err = keep;
      return e;
    }
    c->compat = f;
  }
  rf_ctx* f = c->compat;
  DeviceGuard dg2(f->dev);
  if (c->ns && f->ns)
    if (int e = ck(cudaMemcpyAsync(f->d_state, c->d_state, sizeof(float) * c->ns * c->N,
                                   cudaMemcpyDeviceToDevice, c->stream), "compat: state"))
      return e;
  if (int e = ck(cudaMemsetAsync(f->d_ER, 0, sizeof(float2) * f->rect, c->stream), "compat"))
    return e;
  if (int e = launch_scatter_full(c, f)) return e;
  if (int e = init_status(f, c->prev_macro)) return e;
  const int st = run_iterations(f);
  if (st < 0) return st;
  double sbar[6];
  if (int e = finish(f, 0, sbar)) return e;
  const size_t n6 = sizeof(float) * 6 * (size_t)c->N;
  if (int e = ck(cudaMemcpyAsync(c->d_eps, f->d_eps, n6, cudaMemcpyDeviceToDevice, c->stream),
                 "compat: fields"))
    return e;
  if (int e = ck(cudaMemcpyAsync(c->d_sig, f->d_sig, n6, cudaMemcpyDeviceToDevice, c->stream),
                 "compat: fields"))
    return e;
  if (int e = ck(cudaMemcpyAsync(c->d_alpha, f->d_alpha, sizeof(float) * c->N,
                                 cudaMemcpyDeviceToDevice, c->stream), "compat: fields"))
    return e;
  if (int e = ck(cudaStreamSynchronize(c->stream), "compat")) return e;
  c->launches += f->launches;
  f->launches = 0;
  for (int i = 0; i < 6; ++i) c->last_sbar[i] = sbar[i];
  if (hom_stress)
    for (int i = 0; i < 6; ++i) hom_stress[i] = sbar[i];
  return RF_OK;
}

int rf_law_sweep(rf_ctx* c, const float* d_eps, float* d_tau, float* d_sig) {
  if (!c || !d_eps || !d_tau) return invalid("rf_law_sweep: null argument");
  if (c->N % 4 != 0) return invalid("rf_law_sweep: the voxel count must be a multiple of 4");
  auto mis = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) != 0; };
  if (mis(d_eps) || mis(d_tau) || (d_sig && mis(d_sig)))
    return invalid("rf_law_sweep: field pointers must be 16-byte aligned");
  DeviceGuard dg(c->dev);
  return launch_law_sweep(c, d_eps, d_tau, d_sig);
}

int rf_stress_errors(rf_ctx* c, const rf_ctx* ref, double* Ebar, double* E) {
  if (!c || !ref || !Ebar || !E) return invalid("rf_stress_errors: null argument");
  if (c->nx != ref->nx || c->ny != ref->ny || c->nz != ref->nz || c->dev != ref->dev)
    return invalid("rf_stress_errors: contexts on different grids or devices");
  if (!c->fields_valid || !ref->fields_valid) {
    set_error("rf_stress_errors: both contexts need fields from a solve");
    return RF_ERR_STATE;
  }
  DeviceGuard dg(c->dev);
  if (ref->stream != c->stream)
    if (int e = ck(cudaStreamSynchronize(ref->stream), "stress errors")) return e;
  if (int e = launch_stress_errors(c, ref->d_sig, c->last_sbar, ref->last_sbar)) return e;
  double out[2] = {0.0, 0.0};
  if (int e = ck(cudaMemcpyAsync(out, c->d_err + kErrBlocks, sizeof out, cudaMemcpyDeviceToHost,
                                 c->stream), "stress errors"))
    return e;
  if (int e = ck(cudaStreamSynchronize(c->stream), "stress errors")) return e;
  *Ebar = out[0];
  *E = out[1];
  return RF_OK;
}

int rf_pattern_adapted(const rf_grid* grid, const uint8_t* phase_map, int32_t inclusion_phase,
                       int64_t k_target, int32_t* freqs_out, int64_t cap, int64_t* K_out,
                       void* stream) {
  set_error("");
  long long K = 0;
  int e = rfk::pattern_adapted(grid, phase_map, inclusion_phase, k_target, freqs_out, cap, &K,
                               static_cast<cudaStream_t>(stream));
  if (K_out) *K_out = K;
  return e;
}

int rf_pattern_adapted_noalloc(const rf_grid* grid, const uint8_t* phase_map,
                               int32_t inclusion_phase, int64_t k_target, int32_t* freqs_out,
                               int64_t cap, int64_t* K_out, void* stream) {
  set_error("");
  long long K = 0;
  int e = rfk::pattern_adapted_noalloc(grid, phase_map, inclusion_phase, k_target, freqs_out, cap,
                                       &K, static_cast<cudaStream_t>(stream));
  if (K_out) *K_out = K;
  return e;
}

int rf_pattern_radial(const rf_grid* grid, int64_t k_target, int32_t* freqs_out, int64_t cap,
                      int64_t* K_out, void* stream) {
  set_error("");
  long long K = 0;
  int e = rfk::pattern_radial(grid, k_target, freqs_out, cap, &K,
                              static_cast<cudaStream_t>(stream));
  if (K_out) *K_out = K;
  return e;
}

}  // extern "C"
