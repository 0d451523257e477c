/*
 * rf.h - C ABI of the reduced-frequency Lippmann-Schwinger solver for GB300 (sm_103a).
 *
 * The library solves the periodic microscopic boundary value problem of Sec. 2 (div sigma = 0,
 * sigma = sigma(eps, internal variables), eps = ebar + symmetric gradient of a periodic
 * displacement) with the reduced fixed-point scheme of Sec. 4: per iteration
 *   a) polarization stress tau = sigma(eps) - C0 : eps on every voxel,
 *   b) its DFT, evaluated only on the K frequencies of a sampling pattern,
 *   c) eps^(xi) = -Gamma0(xi) : tau^(xi) for xi != 0, eps^(0) = N ebar (Sec. 3, eq. Gamma),
 *   d) the inverse DFT from those K frequencies back to the grid,
 * until the convergence measure of Sec. 3 drops below tol. Every step runs in the library's
 * own CUDA kernels; nothing falls back to the CPU.
 *
 * Conventions
 *  - Grid: n[0] = Nx, n[1] = Ny, n[2] = Nz; Nz = 1 for dim = 2. Voxel fields are x fastest.
 *    2D problems are plane strain (eps_33 = eps_13 = eps_23 = 0; sigma_33 is an output).
 *  - Six-component tensors use the order (11, 22, 33, 23, 13, 12) with TENSOR shear
 *    components (eps_12, not gamma_12).
 *  - A frequency is an int32 triple (kx, ky, kz) in the signed range (-N_j/2, N_j/2]; the
 *    DFT is f^(k) = sum_x f(x) exp(-2 pi i sum_j k_j x_j / N_j), the inverse carries 1/N.
 *  - A pattern (the reduced set of Sec. 4) holds the zero frequency once, no duplicates, and
 *    is closed under k -> -k (mod N).
 *  - Units are the caller's; the synthetic workloads use GPa.
 *
 * Errors: every call returns an int status. 0 = RF_OK; RF_NOT_CONVERGED (1) means the
 * iteration cap was reached, outputs are written. Negative values are hard errors; outputs
 * are then unspecified. rf_last_error() returns a message for the calling thread (owned by
 * the library, valid until the thread's next call). No C++ exception crosses this ABI.
 *  RF_ERR_NONFINITE  a NaN or infinite input (modulus, macroscopic strain or stress), or a
 *                    convergence measure / homogenised stress that became non-finite on the
 *                    device (e.g. FP32 overflow).
 *  RF_ERR_DIVERGED   the convergence measure exceeded both 1e4 times its smallest value in the
 *                    solve and 1e-3: the basic scheme contracts only for a reference medium
 *                    that bounds the phases well enough (Sec. 3); RF_REF_VOLUME with a stiff
 *                    minority phase can violate that.
 *  RF_ERR_TIMEOUT    a bounded device-side wait of a tensor-core kernel ran out (see
 *                    rf_options.wait_limit); the kernels drain their copies and matrix
 *                    products in flight and release tensor memory before they return, so the
 *                    CUDA context stays usable.
 *
 * Ownership: the caller owns every pointer it passes; inputs are copied before the call
 * returns unless stated otherwise. Outputs go to caller-owned buffers of the documented size.
 * A context owns all device memory it allocates and frees it in rf_destroy.
 * Threading: a context must not be used from two threads at once.
 */
#ifndef RF_H
#define RF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RF_OK = 0,
  RF_NOT_CONVERGED = 1,
  RF_ERR_INVALID = -1,
  RF_ERR_CUDA = -2,
  RF_ERR_NONFINITE = -3,
  RF_ERR_DIVERGED = -4,
  RF_ERR_OOM = -5,
  RF_ERR_TIMEOUT = -6,
  RF_ERR_STATE = -7
};

enum { RF_GREEN_ROTATED = 0, RF_GREEN_CONTINUOUS = 1 };
enum { RF_REF_MINMAX = 0, RF_REF_VOLUME = 1 };
enum { RF_PREC_FP32 = 0, RF_PREC_SPLIT_BF16 = 1, RF_PREC_SPLIT_TF32 = 2 };
enum { RF_TRANSFORM_DFT = 0, RF_TRANSFORM_FFT = 1 };

typedef struct rf_ctx rf_ctx;

/* Grid: dim in {2, 3}; n = (Nx, Ny, Nz), each >= 1, Nz = 1 when dim = 2; Nx <= 4096,
 * Ny, Nz <= 4096, Nx*Ny*Nz < 2^31. */
typedef struct rf_grid {
  int32_t dim;
  int32_t n[3];
} rf_grid;

/* One phase (Sec. 2): isotropic linear elasticity (lambda, mu > 0); when plastic != 0 also the
 * von Mises yield function with linear isotropic hardening, initial yield stress sigma_y0 > 0
 * and hardening modulus H >= 0 (associative flow, radial return). */
typedef struct rf_phase {
  double lambda;
  double mu;
  double sigma_y0;
  double hardening;
  int32_t plastic;
  int32_t reserved;
} rf_phase;

/* Solver options.
 *  tol        convergence measure threshold (Sec. 3): RMS over voxels of the Frobenius norm of
 *             eps^(i+1) - eps^(i), divided by the Frobenius norm of ebar; iterate while >= tol.
 *  max_iter   cap on fixed-point updates per solve (>= 1).
 *  green      RF_GREEN_ROTATED: wave vector of first-order finite differences on the rotated
 *             stencil (Sec. 3); RF_GREEN_CONTINUOUS: q = 2 pi k / N (Nyquist frequencies get a
 *             zero operator).
 *  ref_medium RF_REF_MINMAX: lambda0 = (min + max)/2 and mu0 likewise over the phases present
 *             (the basic scheme of Sec. 3); RF_REF_VOLUME: volume averages.
 *  precision  RF_PREC_FP32: FP32 SIMT transforms. RF_PREC_SPLIT_BF16 / RF_PREC_SPLIT_TF32:
 *             the transforms along x run on the tensor cores (tcgen05) with operands split into
 *             hi + lo parts of BF16 or TF32, three products (hi*hi + hi*lo + lo*hi) and FP32
 *             accumulation; the law stays FP32. The residual and the homogenised stress are
 *             accumulated in FP64 in every mode. Split modes need 2 Kx <= 1152.
 *  check_every  iterations launched between host checks of the device convergence flag
 *             (0 = library default). Work after convergence is skipped on the device, so
 *             results do not depend on it.
 *  transform  RF_TRANSFORM_DFT: pruned separable DFT (only the pattern's distinct kx >= 0
 *             columns along x, its (ky, kx) rectangle along y, (kz, ky, kx) along z).
 *             RF_TRANSFORM_FFT: full FFTs along each axis restricted to the pattern (the
 *             transform the paper uses, Sec. 4); needs sizes 2^b or 3 * 2^b (Nz = 1 in 2D) and
 *             precision RF_PREC_FP32. Both compute the same restricted transform.
 *  fft_rows, fft_cols  FFT mode tiles: grid rows per row-kernel block and line columns per
 *             column-kernel block (0 = chosen by timing a few launches of each candidate when
 *             the pattern is set). Results do not depend on them.
 *  fft_fuse   2D FFT mode, how the column phase between two row passes runs: -1 three kernels
 *             (forward y, Green-operator update with the convergence decision, inverse y);
 *             1 one kernel per group of kx columns (steps b to d of Sec. 4 fused); 2 forward y,
 *             then the Green-operator update and decision inside the inverse y kernel; 3 the
 *             persistent solve: one cooperative launch per solve runs every update (row phase,
 *             grid barrier, column phase per kx, grid barrier, decision) with the grid
 *             co-resident (one or two blocks per SM); 4 (Ny = 1024) as 1 on the warp-FFT
 *             column kernel: a warp per line column, the 1024-point transforms along y in
 *             registers (four-step 32 x 32); 5 (1024 x 1024) the persistent solve on the
 *             passes of mode 4 (one cooperative launch per solve, grid barriers between the
 *             passes); 0 = chosen by timing when the pattern is set (the persistent solves only
 *             when fft_rows and fft_row_blocks are 0; modes 4 and 5 on 1024 x 1024 grids). Must
 *             be 0 or -1 in 3D. All give the same update up to the order of FP32 and FP64
 *             summation.
 *  fft_fuse_kx  kx columns per block of the fused kernel (0 = chosen by timing; 1..16; 1 or 2
 *             in mode 4; mode 5 uses 2).
 *  fft_row_blocks  FFT mode: run the row kernel on this many blocks with the grid rows spread
 *             evenly (blocks differ by at most one row; clamped to the row count), instead of
 *             tiles of fft_rows; 0 = fft_rows or the autotuner (which also times such
 *             partitions over whole multiples of the SM count).
 *  wait_limit  split-precision modes: polls of every bounded mbarrier wait in the tensor-core
 *             kernels before the wait gives up and the solve returns RF_ERR_TIMEOUT (0 = the
 *             library default, 2^26 polls); >= 0.
 *  stall_test  split-precision modes, for testing the timeout path: when 1, every tensor-core
 *             kernel first waits on a barrier that nothing completes, so the bounded wait runs
 *             out after wait_limit polls and the solve returns RF_ERR_TIMEOUT. 0 otherwise.
 *  fft_row_warps  2D FFT mode with Nx = 1024 and plane strain: the row passes between column
 *             phases (not the final pass) may run on the warp-FFT row kernel, a warp pair per
 *             grid row with the 1024-point transforms in registers (four-step 32 x 32). 0 = the
 *             autotuner compares it with the shared-memory row kernel (only when fft_rows and
 *             fft_row_blocks are 0); 2 or 4 = always, with that many warps (one or two rows) per
 *             block; 8 = four rows per block on row-group slabs, the form that goes with
 *             fft_fuse 4 and 5 (and only with them; 0 there means 8); -1 = never. Ignored
 *             where it does not apply; the same update either way up to FP32 rounding order.
 *  batch_resident  rf_batch only, FFT transforms: when every RVE is square with a side of 64,
 *             96, 128, 192 or 256, a solve may run as one RVE-resident launch (a block holds
 *             an RVE for all of its updates and its final pass, RVEs taken largest first from a
 *             queue; no step waits for other RVEs) instead of sweeps of every RVE per update.
 *             0 = the faster of the two by timing a short solve each way at creation; 1 =
 *             always where the batch qualifies; -1 = never. The same update and convergence
 *             rules either way (up to FP32 rounding order). Ignored by rf_create. */
typedef struct rf_options {
  double tol;
  int32_t max_iter;
  int32_t green;
  int32_t ref_medium;
  int32_t precision;
  int32_t check_every;
  int32_t transform;
  int32_t fft_rows;
  int32_t fft_cols;
  int32_t fft_fuse;
  int32_t fft_fuse_kx;
  int32_t fft_row_blocks;
  int64_t wait_limit;
  int32_t stall_test;
  int32_t fft_row_warps;
  int32_t batch_resident;
} rf_options;

/* Run statistics of the last solve on a context. */
typedef struct rf_info {
  int64_t K;              /* pattern size */
  int64_t K_half;         /* frequencies held on the device (kx >= 0 half of the pattern) */
  int32_t Kx, Ky, Kz;     /* distinct kx >= 0, ky, kz values of that half */
  int32_t last_iters;     /* fixed-point updates of the last solve */
  double last_residual;   /* convergence measure after the last update */
  int64_t kernel_launches;/* kernels this context has launched so far */
  double j2_max_violation;/* FP64 check of the last commit: max |sigma_eq - (sy + H a)| / sy */
  double lambda0, mu0;    /* reference medium in use */
  int32_t fft_rows;       /* FFT mode: rows per row-kernel block (set or autotuned), else 0 */
  int32_t fft_row_threads;/* FFT mode: threads per row-kernel block, else 0 */
  int32_t fft_cols;       /* FFT mode: columns per column-kernel block, else 0 */
  int32_t fft_col_threads;/* FFT mode: threads per column-kernel block, else 0 */
  int32_t fft_fused;      /* column-phase mode in use (see fft_fuse): 0 to 5 */
  int32_t fft_fuse_kx;    /* kx columns per fused block, else 0 */
  int32_t fft_fuse_threads;/* threads per fused block, else 0 */
  int32_t fft_row_blocks; /* FFT mode: row-kernel blocks (fft_rows is the largest block's row
                           * count; blocks may hold one row fewer to balance the SMs), else 0;
                           * the persistent solve's grid (and fft_row_threads its block size) */
  int32_t fft_row_warps;  /* warps per block of the warp-FFT row kernel in use, else 0 */
  int32_t reserved;
} rf_info;

/* Create a solver context for one microstructure.
 *  phase_map: HOST uint8 [Nz][Ny][Nx], entries < n_phases (1 <= n_phases <= 16); copied.
 *  stream: a cudaStream_t (or NULL for the legacy default stream) on which all work of this
 *  context is enqueued. The device is the current CUDA device at creation.
 *  Errors: RF_ERR_INVALID for bad sizes, phases or ids; RF_ERR_OOM; RF_ERR_CUDA. */
int rf_create(rf_ctx** ctx, const rf_grid* grid, int32_t n_phases, const rf_phase* phases,
              const uint8_t* phase_map, const rf_options* opt, void* stream);

/* Replace the phase map (same grid) from HOST memory, or from DEVICE memory (same device,
 * readable on the context's stream). The reference medium is recomputed; the internal
 * variables and the load-path state are reset. */
int rf_set_phase_map(rf_ctx* ctx, const uint8_t* phase_map);
int rf_set_phase_map_device(rf_ctx* ctx, const uint8_t* d_phase_map);

/* Set the reduced set of frequencies (Sec. 4), HOST int32 [K][3] (kx, ky, kz); copied.
 * Must satisfy the pattern rules above (checked: RF_ERR_INVALID). Resets the load-path state. */
int rf_set_pattern(rf_ctx* ctx, const int32_t* freqs, int64_t K);

/* One solve at macroscopic strain macro[6] with the internal variables held fixed (they are
 * not committed). warm: nullable HOST float [K][6][2] (re, im) start coefficients in the
 * pattern's order, projected onto compatible strains before use; NULL = uniform start
 * eps = ebar. Outputs (each nullable): homogenised stress [6] (volume average, FP64
 * accumulation), iteration count, final convergence measure.
 * Returns RF_OK, RF_NOT_CONVERGED, or an error (RF_ERR_NONFINITE if the measure is not finite). */
int rf_solve(rf_ctx* ctx, const double macro[6], const float* warm, double hom_stress[6],
             int32_t* iters, double* residual);

/* Load path: n_steps macroscopic strains path[n_steps][6] applied as increments from the
 * context's current state (after rf_create / rf_set_pattern / rf_reset_path: zero strain, zero
 * internal variables). Each increment starts from eps_(n-1) + (ebar_n - ebar_(n-1)), iterates
 * with the internal variables frozen, then commits them from the return map at the converged
 * strain. Outputs (nullable): hom_stress [n_steps][6], iters [n_steps], residuals [n_steps].
 * Returns RF_OK, or RF_NOT_CONVERGED if any increment hit max_iter (the path continues). */
int rf_solve_path(rf_ctx* ctx, int32_t n_steps, const double* path, double* hom_stress,
                  int32_t* iters, double* residuals);

/* Mixed macroscopic control, as an FE-FFT coupling prescribes it at a Gauss point (Sec. 1):
 * for each component i of the six (order 11,22,33,23,13,12, tensor shear), control[i] = 0
 * prescribes the macroscopic strain ebar_i = target[i], control[i] = 1 the average stress
 * <sigma>_i = target[i]. In 2D (plane strain) components 33, 23, 13 must be strain-controlled
 * with target 0. Every update sets the zero frequency to N E, where E takes the prescribed
 * strains and solves (C0 : E)_i = target_i - <tau>_i for the stress-controlled components,
 * <tau> = tau^(0) / N (the averaged Lippmann-Schwinger equation <sigma> = C0 : <eps> + <tau>),
 * in FP64 on the device. The start is E0 (the same rule with <tau> = 0), and the convergence
 * measure is normalised by |E0| instead of |ebar|; otherwise as rf_solve.
 * hom_strain (nullable) receives E of the last update (the macroscopic strain reached).
 * rf_solve_path_mixed: path[n_steps][6] of targets with one control for all increments; each
 * increment starts from the last converged strain plus the reference medium's response (the
 * rule above with <tau> = 0) to the increment of the targets, stress increments measured from
 * the last homogenised stress (from the zero state: E0); commits as rf_solve_path; hom_stress
 * and hom_strain are [n_steps][6].
 * Errors: RF_ERR_INVALID (control not 0/1, 2D out-of-plane components), RF_ERR_NONFINITE. */
int rf_solve_mixed(rf_ctx* ctx, const int32_t control[6], const double target[6],
                   const float* warm, double hom_stress[6], double hom_strain[6], int32_t* iters,
                   double* residual);
int rf_solve_path_mixed(rf_ctx* ctx, const int32_t control[6], int32_t n_steps,
                        const double* path, double* hom_stress, double* hom_strain,
                        int32_t* iters, double* residuals);

/* Reset the load-path state (strain and internal variables) to zero. */
int rf_reset_path(rf_ctx* ctx);

/* Fields of the last solve, HOST float buffers (nullable) of [6][N] (strain, stress; order
 * 11,22,33,23,13,12) and [N] (accumulated plastic strain after the last commit). */
int rf_get_fields(rf_ctx* ctx, float* strain, float* stress, float* eps_p_acc);

/* Reduced strain coefficients of the last solve: HOST float [K][6][2] in the pattern's order. */
int rf_get_reduced_strain(rf_ctx* ctx, float* coeffs);

/* Checkpoint of the load-path state (strain coefficients, internal variables, last macro
 * strain). Call with buf = NULL to get the size in *bytes. rf_set_state restores a buffer
 * produced by rf_get_state on a context with the same grid, phases and pattern. */
int rf_get_state(rf_ctx* ctx, void* buf, size_t* bytes);
int rf_set_state(rf_ctx* ctx, const void* buf, size_t bytes);

int rf_get_info(const rf_ctx* ctx, rf_info* info);

/* Per-stage device-time accounting. With tracing on, every stage launch of every fixed-point
 * update is bracketed by CUDA events on the context's stream; the elapsed times of updates
 * that did work (not the ones skipped after convergence) are accumulated per stage.
 * Stages: 0 inverse transform along z, 1 inverse along y, 2 row kernel (transforms along x,
 * constitutive law, polarization), 3 forward along y, 4 forward along z, 5 Green-operator
 * update with the convergence decision (with fft_fuse 2 it includes the inverse along y),
 * 6 fused column phase (fft_fuse 1: stages 3, 5 and 1 in one kernel), 7 final pass (fields,
 * homogenised stress, commit).
 * rf_get_stage_times fills ms_total[8] (milliseconds) and counts[8] (launches timed). */
int rf_set_tracing(rf_ctx* ctx, int on);
int rf_get_stage_times(const rf_ctx* ctx, double ms_total[8], int64_t counts[8]);
int rf_reset_stage_times(rf_ctx* ctx);

/* Compatibility step (Sec. 5.1, also applied in Sec. 5.2 and 5.3): the Lippmann-Schwinger
 * equation solved once on the full set of frequencies from the fields of the last reduced solve.
 * Reading: one update of the basic scheme with every frequency of the grid, starting from the
 * reduced strain field (its coefficients on the pattern; all other frequencies zero):
 *   tau = sigma(eps) - C0 : eps, eps_c^(xi) = -Gamma0(xi) : tau^(xi) for xi != 0,
 *   eps_c^(0) = N ebar (ebar of the last solve or increment), 0 at null frequencies,
 * then sigma_c = sigma(eps_c), with the internal variables the context holds (after
 * rf_solve_path: those committed for its last increment; nothing is committed here).
 * The context's fields (rf_get_fields) are replaced by eps_c, sigma_c; hom_stress (nullable)
 * receives the volume average of sigma_c. The reduced coefficients and the load-path state are
 * unchanged. The first call builds a second context on the same grid with the full set of
 * frequencies (FFT transforms when the sides are 2^b or 3 * 2^b, else the pruned DFT) and keeps
 * it until the phase map changes or the context is destroyed.
 * Errors: RF_ERR_STATE if no solve has produced fields yet; RF_ERR_OOM; RF_ERR_NONFINITE. */
int rf_compat(rf_ctx* ctx, double hom_stress[6]);

/* Constitutive sweep on its own (step a of Sec. 4, unfused): for every voxel,
 * tau = sigma(eps) - C0 : eps with the context's phase map, phases, reference medium and internal
 * variables (held fixed), from strain planes in DEVICE memory.
 *  d_eps: DEVICE float [NC][N] (NC = 3 in 2D: 11, 22, 12; 6 in 3D: 11, 22, 33, 23, 13, 12),
 *  d_tau: DEVICE float [NC][N] output, d_sig: nullable DEVICE float [NC][N] stress output.
 *  N must be a multiple of 4 and the pointers 16-byte aligned (16-byte loads and stores).
 * Asynchronous: enqueued on the context's stream. The fused solver runs the same law inside its
 * row kernels; this entry point exists to measure and use the sweep by itself. */
int rf_law_sweep(rf_ctx* ctx, const float* d_eps, float* d_tau, float* d_sig);

/* Error measures of Sec. 5 between the fields a context holds now (after a solve or
 * rf_compat) and those of a reference context on the same grid and device (typically a solve
 * with the full set of frequencies):
 *   Ebar = |sbar - sbar_ref| / |sbar_ref|,
 *   E    = (1/N) sum_x |sigma(x) - sigma_ref(x)| / |sigma_ref(x)|,
 * Frobenius norms with both shear entries counted; voxels where |sigma_ref| = 0 add nothing.
 * Computed on the device in FP64 on ctx's stream (ref's stream is synchronised first).
 * Errors: RF_ERR_INVALID for different grids or devices; RF_ERR_STATE without fields. */
int rf_stress_errors(rf_ctx* ctx, const rf_ctx* ref, double* Ebar, double* E);

/* Destroy a context and free its device memory. NULL is accepted. */
int rf_destroy(rf_ctx* ctx);

/* Geometrically adapted sampling pattern (Sec. 4.2, 3D as in Sec. 5.3): the step function
 * g = [phase == inclusion_phase] is transformed (FP64), amplitudes |g^| are quantised to
 * round(|g^| / |g^(0)| * 2^30); pairs (k, -k) are ranked by (larger amplitude, smaller |k|^2,
 * smaller signed linear index) and added whole until >= k_target frequencies are held.
 *  phase_map: HOST uint8 [Nz][Ny][Nx]. freqs_out: HOST int32 [cap][3], sorted by signed linear
 *  index (z slowest, x fastest; index = ((kz+hz)Ny + ky+hy)Nx + kx+hx, h_j = (N_j-1)/2).
 *  *K_out receives the pattern size (k_target or k_target + 1); RF_ERR_INVALID if it exceeds cap.
 *  stream: cudaStream_t or NULL. Runs on the current device; allocates and frees scratch. */
int rf_pattern_adapted(const rf_grid* grid, const uint8_t* phase_map, int32_t inclusion_phase,
                       int64_t k_target, int32_t* freqs_out, int64_t cap, int64_t* K_out,
                       void* stream);

/* Same result as rf_pattern_adapted, for grids of at most 65536 voxels, without allocating.
 * No counterpart in the paper: this exists for callers that cannot allocate device memory.
 * rf_pattern_adapted calls cudaMalloc/cudaFree for its scratch, and cudaFree synchronises the
 * whole device; a caller that shares the GPU with streams it must not stall, or whose device
 * memory belongs to another framework's pool allocator, cannot make those calls. This entry
 * point uses a fixed scratch array (about 4.5 MB) that lives in the library's static device
 * memory on every GPU that loads the library, until the process exits; it calls no
 * cudaMalloc, cudaFree, cudaMallocHost or other allocating routine.
 *  - The first call on a device looks up that array's device address (once per device, with
 *    the device current); make that first call before any stream capture begins.
 *  - Grids with more than 65536 voxels are rejected with RF_ERR_INVALID and a message.
 *  - All calls share the one array: calls whose GPU work overlaps (different streams or host
 *    threads at the same time) race and corrupt each other's results. Serialise them.
 *  - Arguments, output order and errors are those of rf_pattern_adapted; the call returns
 *    when the result is in freqs_out. */
int rf_pattern_adapted_noalloc(const rf_grid* grid, const uint8_t* phase_map,
                               int32_t inclusion_phase, int64_t k_target, int32_t* freqs_out,
                               int64_t cap, int64_t* K_out, void* stream);

/* Fixed radial sampling pattern (Sec. 4.1), 2D only. The paper shows it only as a figure;
 * this library's reading: L equiangular lines through the origin at angles pi l / L, each
 * rasterised by unit steps along its dominant axis with the other coordinate rounded half away
 * from zero; the smallest L whose union holds >= k_target frequencies; trimmed by keeping
 * pairs of smaller |k|^2 first (ties: signed linear index). Output as rf_pattern_adapted. */
int rf_pattern_radial(const rf_grid* grid, int64_t k_target, int32_t* freqs_out, int64_t cap,
                      int64_t* K_out, void* stream);

/* ---- Batched solve: many independent 2D RVEs (e.g. the Gauss points of an FE-FFT macro model,
 * Sec. 1), each with its own grid (sides 2..1024, any size), phase map, adapted pattern and
 * macroscopic strain, solved together on one GPU. Every update of all unconverged RVEs is a fixed
 * sequence of persistent kernels walking (RVE, tile) work lists; RVEs leave the work as they
 * converge, and a whole solve is one CUDA graph launch (a conditional while node over a few
 * updates, ended on the device once every RVE is done). Elastic phases only, plane strain, FP32
 * transforms (precision RF_PREC_FP32):
 *   options.transform = RF_TRANSFORM_FFT: FFTs along x and y, restricted to each pattern, for
 *     RVEs whose sides are 2^b or 3 * 2^b; the pruned DFT for the other sides;
 *   options.transform = RF_TRANSFORM_DFT: the pruned separable DFT for every RVE.
 * FP64 convergence measure and homogenised stress; the same convergence measure and rules
 * (converged, capped, non-finite, diverged) as rf_solve, per RVE.
 *  rf_batch_create: grids[n_rve]; phase_maps[n_rve] HOST uint8 pointers; phases shared by all
 *  RVEs; patterns[n_rve] HOST int32 [K[r]][3] pointers (rules of rf_set_pattern, kz = 0); all
 *  inputs are copied. Chooses the rows per row work item for each size class of RVE (largest
 *  side <= 64, <= 96, <= 128, <= 192, larger), whether the y transforms run as warp-FFT column
 *  items, and the persistent grid size by timing updates of the whole batch (autotuner).
 *  With options.transform = RF_TRANSFORM_FFT, options.fft_row_warps = -1 keeps every row and
 *  column item on the shared-memory FFTs, > 0 puts every row and column of 64, 96, 128, 192 or
 *  256 voxels on the warp-FFT items, 0 lets the autotuner choose. stream as in rf_create.
 *  rf_batch_solve: macro [n_rve][6]; warm nullable, else warm[r] nullable HOST float
 *  [K[r]][6][2] start coefficients (projected as in rf_solve); outputs (each nullable):
 *  hom_stress [n_rve][6], iters [n_rve], residuals [n_rve], status [n_rve] (RF_OK,
 *  RF_NOT_CONVERGED, RF_ERR_NONFINITE or RF_ERR_DIVERGED per RVE). Returns RF_OK when every
 *  RVE converged, RF_NOT_CONVERGED otherwise, or a hard error (RF_ERR_NONFINITE for a
 *  non-finite macroscopic strain).
 *  rf_batch_info: kernels launched so far (graph replays included), the rows per row item
 *  chosen for each of the five size classes (rows_per_item: int32 [5], nullable: 1, 2, 4 or 8
 *  for shared-memory FFT or DFT items; 85, 53, 42, 26 or 21 for the warp-FFT row items of rows
 *  of 64, 96, 128, 192 or 256 voxels, which transform 32 / P packed line pairs of L = 32 P
 *  points per warp in registers), persistent grid size. */
typedef struct rf_batch rf_batch;
int rf_batch_create(rf_batch** batch, int32_t n_rve, const rf_grid* grids,
                    const uint8_t* const* phase_maps, int32_t n_phases, const rf_phase* phases,
                    const int32_t* const* patterns, const int64_t* K, const rf_options* opt,
                    void* stream);
int rf_batch_solve(rf_batch* batch, const double* macro, const float* const* warm,
                   double* hom_stress, int32_t* iters, double* residuals, int32_t* status);
int rf_batch_info(const rf_batch* batch, int64_t* kernel_launches, int32_t* rows_per_item,
                  int32_t* grid);
/* rf_batch_mode: *resident = 1 when the batch's solves run RVE-resident (options.batch_resident),
 * else 0. */
int rf_batch_mode(const rf_batch* batch, int32_t* resident);
int rf_batch_destroy(rf_batch* batch);

/* Message of the last error on the calling thread ("" if none). */
const char* rf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* RF_H */
