/*
 * rf_mlp.h - C ABI of the learned warm start for the batched reduced-frequency solver
 * (sm_103a).
 *
 * The fixed-point scheme of Sec. 4 converges from any start; the plain start is eps = ebar
 * (only the zero frequency set). A better start shortens the iteration, and the converged
 * result is unchanged because the convergence measure of Sec. 3 still decides when to stop.
 * This header adds a small network, trained on solutions the solver itself produced, that
 * predicts the reduced strain coefficients of an RVE from its phase-indicator coefficients
 * and its macroscopic strain.
 *
 * Slots. The slots of an RVE are the frequencies of the kx >= 0 half of its pattern (the half
 * the solver stores, in the solver's order); rf_batch_slots gives their count and per-RVE
 * offsets. gamma(k) = g^(k) / N is the DFT of the inclusion indicator g (Sec. 4.2) divided by
 * the voxel count N, a = kx / Nx, b = ky / Ny, rho = sqrt(a^2 + b^2).
 *
 * Network input: 48 descriptors per RVE (volume fraction; square root of the power sum of
 * gamma over the nonzero pattern frequencies in 24 radial bins i = min(23, floor(96 rho)),
 * decided in FP64; four bands of six bins with the power-weighted means of cos 2t, sin 2t,
 * cos 4t, sin 4t, t the angle of (a, b); the square root of the total power; zeros).
 * Network: h1 = GELU(x W1 + b1), h2 = GELU(h1 W2 + b2), o = h2 W3 + b3 (48 -> H -> H -> 243),
 * GELU(z) = z Phi(z) with the standard normal CDF Phi; W row-major [in][out].
 * Head: o[(c*3 + d)*27 + n] expands a real transfer T_cd(k) = sum_n o[...] phi_n(k) over the
 * basis phi_n = r_i(rho) h_j(t), n = 9 i + j, r = (1, 4 rho, 16 rho^2),
 * h = (1, cos 2t, sin 2t, cos 4t, sin 4t, cos 6t, sin 6t, cos 8t, sin 8t); the prediction is
 * p_c(k) = sum_d T_cd(k) gamma(k) e_d for c, d in (11, 22, 12), e = (ebar_11, ebar_22,
 * ebar_12) / |ebar| (Frobenius norm). It has the structure of the scheme's first update (Sec. 4
 * step c on the plain start): linear in gamma and in ebar, conjugate-symmetric.
 * Targets: t_c(k) = eps^_c(k) / (N |ebar|) of converged solutions. Loss: mean over the six real
 * parts of (p - t)^2 over the pattern's nonzero, non-null frequencies (slot weights count k and
 * -k), minimised with Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 *
 * GEMMs run on the tensor cores with FP32 accumulation: BF16 operands for inference
 * (RF_MLP_BF16), TF32 operands for training (RF_MLP_TF32); weights, activations and optimiser
 * state are FP32 in device memory.
 *
 * Pointers named d_* are DEVICE pointers (16-byte aligned, caller-owned, not retained after
 * the call returns); all others are host pointers. A minibatch is B consecutive RVEs whose
 * slots d_offsets[0] .. d_offsets[B] (device int64, B + 1 entries) index into d_slots and the
 * per-slot arrays. Calls are asynchronous on the network's stream unless they return data to
 * the host. Errors as in rf.h.
 */
#ifndef RF_MLP_H
#define RF_MLP_H

#include "rf.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { RF_MLP_BF16 = 0, RF_MLP_TF32 = 1 };
enum { RF_MLP_IN = 48, RF_MLP_BASIS = 27, RF_MLP_OUT = 243 };

/* One slot. weight: 0 for the zero frequency and null frequencies of the Green operator,
 * 1 for a frequency whose conjugate is its own slot, 2 when the slot stands for k and -k. */
typedef struct rf_slot {
  float g_re, g_im;   /* gamma(k) */
  float a, b;         /* kx / Nx, ky / Ny */
  float weight;
  float inv_n;        /* 1 / N of the slot's RVE */
  int32_t rve;        /* rve_base + index of the RVE in its batch */
  int32_t kind;       /* 0 regular, 1 zero frequency, 2 null */
} rf_slot;

typedef struct rf_mlp rf_mlp;

typedef struct rf_mlp_dims {
  int32_t n_in;       /* 48 */
  int32_t n_hidden;   /* H */
  int32_t n_out;      /* 243 */
  int32_t max_batch;
  int64_t n_params;   /* 48*H + H + H*H + H + H*243 + 243 */
  int64_t adam_steps;
} rf_mlp_dims;

/* n_hidden a multiple of 16 in [16, 4096], max_batch in [1, 65536]. Parameters start at zero
 * (set them with rf_mlp_set_params). stream: cudaStream_t or NULL (own stream). */
int rf_mlp_create(rf_mlp** net, int32_t n_hidden, int32_t max_batch, void* stream);
int rf_mlp_get_dims(const rf_mlp* net, rf_mlp_dims* dims);

/* Parameters / gradients as one host float array of n_params: W1, b1, W2, b2, W3, b3 in that
 * order, each row-major. set_params also clears the Adam moments and step count. */
int rf_mlp_set_params(rf_mlp* net, const float* params);
int rf_mlp_get_params(const rf_mlp* net, float* params);
int rf_mlp_get_grads(const rf_mlp* net, float* grads);

/* Raw network output o for B <= max_batch descriptor rows: d_x [B][48] -> d_out [B][243]. */
int rf_mlp_forward(rf_mlp* net, int32_t B, const float* d_x, float* d_out, int32_t precision);

/* Targets and unit directions of B RVEs: d_macro [B][6] (double), d_coeffs [slots][3][2]
 * (eps^ components 11, 22, 12 at the slots, as rf_batch_reduced_strain writes them) ->
 * d_t [slots][6], d_e [B][3]. */
int rf_mlp_targets(rf_mlp* net, int32_t B, const double* d_macro, const rf_slot* d_slots,
                   const int64_t* d_offsets, const float* d_coeffs, float* d_t, float* d_e);

/* Loss and gradients (TF32 tensor-core GEMMs) of one minibatch of B <= max_batch RVEs.
 * loss (host, nullable) receives the mean squared error (the call then waits for the stream).
 * Gradients stay on the device until rf_mlp_get_grads. */
int rf_mlp_loss_grad(rf_mlp* net, int32_t B, const float* d_x, const float* d_e,
                     const rf_slot* d_slots, const int64_t* d_offsets, const float* d_t,
                     double* loss);
/* One Adam step with the gradients of the last rf_mlp_loss_grad, learning rate lr > 0. */
int rf_mlp_adam(rf_mlp* net, float lr);
/* rf_mlp_loss_grad followed by rf_mlp_adam. */
int rf_mlp_train_step(rf_mlp* net, int32_t B, const float* d_x, const float* d_e,
                      const rf_slot* d_slots, const int64_t* d_offsets, const float* d_t,
                      float lr, double* loss);

/* Warm start of B RVEs (BF16 inference, any B): d_warm [slots][3][2] = N |ebar| p at regular
 * slots, 0 at the others (components 11, 22, 12). */
int rf_mlp_predict_warm(rf_mlp* net, int32_t B, const float* d_x, const double* d_macro,
                        const rf_slot* d_slots, const int64_t* d_offsets, float* d_warm);

/* Kernels launched by this network so far. */
int rf_mlp_launches(const rf_mlp* net, int64_t* launches);
int rf_mlp_destroy(rf_mlp* net);

/* Batch hooks (rf_batch of rf.h), all on the batch's stream:
 *  rf_batch_slots: total slot count and offsets [n_rve + 1] (nullable) of each RVE's slots.
 *  rf_batch_descriptors: d_x [n_rve][48] and d_slots [slots] of every RVE from the batch's
 *    phase maps and patterns (g = indicator of inclusion_phase); slot.rve = rve_base + r.
 *  rf_batch_reduced_strain: coefficients of the last solve at the slots, d_coeffs
 *    [slots][3][2] (components 11, 22, 12, real and imaginary parts).
 *  rf_batch_solve_warm: rf_batch_solve from DEVICE start coefficients d_warm [slots][3][2]
 *    (as rf_mlp_predict_warm writes them), projected onto compatible strains before the first
 *    update (zero frequency set to N ebar); outputs as rf_batch_solve. */
int rf_batch_slots(const rf_batch* batch, int64_t* n_slots, int64_t* offsets);
int rf_batch_descriptors(rf_batch* batch, int32_t inclusion_phase, int32_t rve_base, float* d_x,
                         rf_slot* d_slots);
int rf_batch_reduced_strain(rf_batch* batch, float* d_coeffs);
int rf_batch_solve_warm(rf_batch* batch, const double* macro, const float* d_warm,
                        double* hom_stress, int32_t* iters, double* residuals, int32_t* status);

#ifdef __cplusplus
}
#endif

#endif /* RF_MLP_H */
