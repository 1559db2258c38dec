/*
 * fockdiag_mlp.h -- the learned proposal model of the library.
 *
 * A multilayer perceptron FK_MLP_IN -> 256 -> 256 -> 256 -> FK_MLP_OUT with
 * BF16 weights and activations, FP32 accumulation on the tensor cores, SiLU
 * hidden activations, an MSE loss and Adam on FP32 master weights.  It maps
 * 15 circuit parameters (3 squeezings, 3 displacements, 9 interferometer
 * angles) to 2 scores of the state the circuit heralds (log success
 * probability and fidelity to a target); proposals are verified by the
 * exact recurrence.  The paper does not define this model: it leaves the
 * ansatz, cost function and target state outside its scope (Sec. 1), and
 * this model serves the gradient-based circuit optimisation of Sec. 2.5.
 *
 * Parameters are packed FP32 [W1 b1 W2 b2 W3 b3 W4 b4], each W row-major
 * [out][in].  All pointers are device pointers; calls are stream-ordered.
 */
#ifndef FOCKDIAG_MLP_H
#define FOCKDIAG_MLP_H

#include <stddef.h>
#include <stdint.h>

#include "fockdiag.h"

#ifdef __cplusplus
extern "C" {
#endif

#define FK_MLP_IN 15
#define FK_MLP_HIDDEN 256
#define FK_MLP_OUT 2

/* Bytes of the model state (master weights, Adam moments, BF16 copies), of
 * the workspace for `batch` samples, and the number of parameters. */
int fk_mlp_sizes(int batch, size_t *state_bytes, size_t *ws_bytes, int64_t *n_params);

/* Sets the master weights from d_params (packed FP32), clears the Adam
 * moments and refreshes the BF16 copies.  d_state 256-byte aligned. */
int fk_mlp_load(void *d_state, const float *d_params, void *stream);

/* d_y [batch][2] = model(d_x [batch][15]). */
int fk_mlp_forward(const void *d_state, int batch, const float *d_x, float *d_y, void *d_ws,
                   size_t ws_bytes, void *stream);

/* Gradient of sum_bj d_gy[b][j] * y[b][j] with respect to the packed
 * parameters (FP32, written to d_gparams) at inputs d_x. */
int fk_mlp_backward(const void *d_state, int batch, const float *d_x, const float *d_gy,
                    float *d_gparams, void *d_ws, size_t ws_bytes, void *stream);

/* One Adam step (step >= 1) on the loss mean_bj (y - target)^2 over the
 * batch; d_loss (1 float, may be NULL) receives the loss before the step. */
int fk_mlp_train_step(void *d_state, int batch, const float *d_x, const float *d_target,
                      float lr, float beta1, float beta2, float eps, int step, float *d_loss,
                      void *d_ws, size_t ws_bytes, void *stream);

/*
 * Scores of heralded states, the labels the model learns and the objective
 * the proposals are refined on.  For circuit i, rho = the [NU][NU] block at
 * element offset d_offsets[i] of d_rho (a fock_conditional_dm output: the
 * unnormalised state of the undetected mode for the heralding pattern):
 *   d_P[i] = Tr rho (the heralding probability, Sec. 3.2),
 *   d_F[i] = <t|rho|t> / Tr rho, t = d_target [NU] normalised,
 * and, if d_grad_rho is not NULL, the gradient of J = F + lambda ln P with
 * respect to rho (PyTorch convention), written at the same offsets:
 *   (t_k conj(t_l) - F delta_kl + lambda delta_kl) / P.
 */
int fk_herald_scores(int batch, const fk_c128 *d_rho, const int64_t *d_offsets, int NU,
                     const fk_c128 *d_target, double lambda, double *d_P, double *d_F,
                     fk_c128 *d_grad_rho, void *stream);

/*
 * The tensor-core GEMM the 256-wide layers of the model run on (exposed for
 * its own tests; the paper has no counterpart): d_C [M][N] fp32 =
 * d_A [M][K] d_B [N][K]^T, both operands bf16 row-major (K contiguous), on
 * the fifth-generation tensor cores (tcgen05.mma, fp32 accumulation in
 * tensor memory, operand tiles loaded by TMA).  N must be a multiple of 256
 * and K of 8 (TMA row strides are multiples of 16 bytes); base pointers
 * 16-byte aligned.  ksplit > 1 splits K over CTAs into d_partials
 * [ceil(K / k_slice)][M][N] fp32 (at most ksplit slices) summed in a fixed
 * order into d_C.  d_status (device int, may be NULL) becomes FK_ETIMEOUT if
 * a wait inside the kernel ran out (the kernel then returns without
 * writing).  FK_EINVAL for bad sizes, FK_ECUDA for a failed launch.
 */
int fk_tc_gemm_bf16(int M, int N, int K, const void *d_A, const void *d_B, float *d_C,
                    float *d_partials, int ksplit, int *d_status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FOCKDIAG_MLP_H */
