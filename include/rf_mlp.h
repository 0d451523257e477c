/*
 * rf_mlp.h - C ABI of the learned warm start for the reduced-frequency solver (sm_103a).
 *
 * The fixed-point scheme of Sec. 4 converges from any start; the plain start is eps = ebar
 * (only the zero frequency set). A better start shortens the iteration, and the converged
 * result is unchanged because the convergence measure of Sec. 3 still decides when to stop.
 * This header adds a small network that predicts the reduced strain coefficients of an RVE
 * from its geometry and macroscopic strain, trained on solutions the solver itself produced.
 *
 * Network (all arithmetic in the library's kernels):
 *  - input x [4 S]: per slot s < S (the s-th frequency of the RVE's pattern, pattern order)
 *    Re g^(k_s) / N, Im g^(k_s) / N, kx_s / Nx, ky_s / Ny, g the indicator of the inclusion
 *    phase (Sec. 4: the same transform that defines the adapted pattern); missing slots 0.
 *  - h1 = GELU(x W1 + b1), h2 = GELU(h1 W2 + b2), o = h2 W3 + b3, GELU(z) = z Phi(z) with the
 *    standard normal CDF Phi; W1 [4S][H], W2 [H][H], W3 [H][18 S] row-major.
 *  - head: o holds per slot s, strain component c in (11, 22, 12), direction d in
 *    (11, 22, 12) and real/imaginary part r the coefficient o[((s*3 + c)*3 + d)*2 + r]; the
 *    prediction is p[(s*3 + c)*2 + r] = sum_d o[...] e_d with the unit direction
 *    e = (ebar_11, ebar_22, ebar_12) / |ebar| (|ebar| the Frobenius norm). The prediction is
 *    therefore exactly linear in ebar, as the elastic fixed point is.
 *  - targets: t[(s*3 + c)*2 + r] = eps^_c(k_s) / (N |ebar|) from converged coefficients.
 *  - loss: mean of (p - t)^2 over the valid entries (slots s < valid[b]), minimised with Adam
 *    (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 *
 * GEMMs run on the tensor cores with FP32 accumulation: BF16 operands for inference
 * (RF_MLP_BF16), TF32 operands for training (RF_MLP_TF32); weights, activations and optimiser
 * state are FP32 in device memory.
 *
 * Pointers named d_* are DEVICE pointers (16-byte aligned, caller-owned, not retained after
 * the call returns); all others are host pointers. Calls are asynchronous on the network's
 * stream unless they return data to the host. Errors as in rf.h.
 */
#ifndef RF_MLP_H
#define RF_MLP_H

#include "rf.h"

#ifdef __cplusplus
extern "C" {
#endif

enum { RF_MLP_BF16 = 0, RF_MLP_TF32 = 1 };

typedef struct rf_mlp rf_mlp;

typedef struct rf_mlp_dims {
  int32_t n_slots;    /* S */
  int32_t n_in;       /* 4 S */
  int32_t n_hidden;   /* H */
  int32_t n_out;      /* 18 S */
  int32_t max_batch;
  int32_t pad;
  int64_t n_params;   /* 4S*H + H + H*H + H + H*18S + 18S */
  int64_t adam_steps;
} rf_mlp_dims;

/* n_slots >= 1, n_hidden a multiple of 16 in [16, 4096], max_batch in [1, 65536]. Parameters
 * start at zero (set them with rf_mlp_set_params). stream: cudaStream_t or NULL (own stream). */
int rf_mlp_create(rf_mlp** net, int32_t n_slots, int32_t n_hidden, int32_t max_batch,
                  void* stream);
int rf_mlp_get_dims(const rf_mlp* net, rf_mlp_dims* dims);

/* Parameters / gradients as one host float array of n_params: W1, b1, W2, b2, W3, b3 in that
 * order, each row-major. set_params also clears the Adam moments and step count. */
int rf_mlp_set_params(rf_mlp* net, const float* params);
int rf_mlp_get_params(const rf_mlp* net, float* params);
int rf_mlp_get_grads(const rf_mlp* net, float* grads);

/* Raw network output o for B <= max_batch inputs: d_x [B][4S] -> d_out [B][18S]. */
int rf_mlp_forward(rf_mlp* net, int32_t B, const float* d_x, float* d_out, int32_t precision);

/* Training targets from solver coefficients: d_coeffs [B][S][6][2] (the layout of
 * rf_batch_reduced_strain), d_macro [B][6] (double), d_nvox [B] (double, N of each RVE) ->
 * d_t [B][6S] and the unit directions d_e [B][3]. */
int rf_mlp_targets(rf_mlp* net, int32_t B, const float* d_coeffs, const double* d_macro,
                   const double* d_nvox, float* d_t, float* d_e);

/* Loss and gradients (TF32 tensor-core GEMMs) of one batch; d_valid [B] int32 valid slots per
 * sample (each clamped to [0, S]). loss (host, nullable) receives the mean squared error (the
 * call then waits for the stream). Gradients stay on the device until rf_mlp_get_grads. */
int rf_mlp_loss_grad(rf_mlp* net, int32_t B, const float* d_x, const float* d_t,
                     const float* d_e, const int32_t* d_valid, double* loss);
/* One Adam step with the gradients of the last rf_mlp_loss_grad, learning rate lr > 0. */
int rf_mlp_adam(rf_mlp* net, float lr);
/* rf_mlp_loss_grad followed by rf_mlp_adam. */
int rf_mlp_train_step(rf_mlp* net, int32_t B, const float* d_x, const float* d_t,
                      const float* d_e, const int32_t* d_valid, float lr, double* loss);

/* Warm start (BF16 inference): d_x [B][4S], d_macro [B][6] (double), d_nvox [B] (double) ->
 * d_coeffs [B][S][6][2] start coefficients N |ebar| p in the rf_batch_reduced_strain layout
 * (components 33, 23, 13 zero). */
int rf_mlp_predict_warm(rf_mlp* net, int32_t B, const float* d_x, const double* d_macro,
                        const double* d_nvox, float* d_coeffs);

/* Kernels launched by this network so far. */
int rf_mlp_launches(const rf_mlp* net, int64_t* launches);
int rf_mlp_destroy(rf_mlp* net);

/* Batch hooks (rf_batch of rf.h), all on the batch's stream:
 *  rf_batch_features: network inputs of every RVE, d_x [n_rve][4 n_slots], from the batch's
 *    phase maps and patterns (g = indicator of inclusion_phase); d_valid [n_rve] (nullable)
 *    receives min(K, n_slots) per RVE.
 *  rf_batch_reduced_strain: converged coefficients of the last solve in pattern order,
 *    d_coeffs [n_rve][n_slots][6][2] (slots >= K zero), as rf_get_reduced_strain.
 *  rf_batch_solve_warm: rf_batch_solve with DEVICE start coefficients d_warm
 *    [n_rve][n_slots][6][2] in pattern order (as produced by rf_mlp_predict_warm; frequencies
 *    of slot >= n_slots start at zero), projected onto compatible strains before the first
 *    update; outputs as rf_batch_solve. */
int rf_batch_features(rf_batch* batch, int32_t inclusion_phase, int32_t n_slots, float* d_x,
                      int32_t* d_valid);
int rf_batch_reduced_strain(rf_batch* batch, int32_t n_slots, float* d_coeffs);
int rf_batch_solve_warm(rf_batch* batch, const double* macro, const float* d_warm,
                        int32_t n_slots, double* hom_stress, int32_t* iters, double* residuals,
                        int32_t* status);

#ifdef __cplusplus
}
#endif

#endif /* RF_MLP_H */
