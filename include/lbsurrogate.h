/*
 * lbsurrogate — learned warm start for the spheroid lattice Boltzmann runs of
 * lbsph.h, on NVIDIA GB300 (sm_103a).  Part of liblbsph.so.
 *
 * The paper computes the drag of a spheroid by running the LB method to steady
 * state (Sec. III: Oberbeck drag, drift, Jeffery orbits).  This part learns
 * that map: a small multilayer perceptron predicts the spheroid's 6x6
 * resistance tensor R (force/torque = R (U, Omega), Eq. Fsplit-Eq. Tsplit at
 * steady state with the drag of the whole flow) from its aspect ratio, size,
 * viscosity, confinement and orientation.  It is trained on resistance
 * tensors that the LB method itself produces, and its prediction warm-starts a
 * run: particle velocities (U, Omega) = R^-1 (F_ext, T_ext) plus the periodic
 * steady flow of the particles' forces in the lattice fluid as the initial
 * fluid (lbsph.h, lb_stokes_field / lb_init_fluid), so that fewer steps reach
 * steady state.
 *
 * Network (fixed shape): x[8] -> 256 -> 256 -> 21, ReLU between layers, inputs
 * padded to 16 and outputs to 32 for the tensor-core tiles.  The 21 outputs
 * are a lower-triangular 6x6 L (row-major lower triangle; diagonal through
 * softplus) and the prediction is the dimensionless tensor R^ = L L^T.
 * Every matrix product runs on the 5th-generation tensor cores (tcgen05.mma,
 * BF16 operands in shared memory, FP32 accumulators in tensor memory); the
 * loss, the backward pass and the Adam update are CUDA kernels of this
 * library.  Master weights are FP32; the products read BF16 copies.
 *
 * Conventions as in lbsph.h: lb_status returns, caller-owned buffers, device
 * pointers where stated, asynchronous on the given stream (NULL = legacy
 * default stream) unless stated.
 */
#ifndef LBSURROGATE_H
#define LBSURROGATE_H

#include <stddef.h>
#include <stdint.h>

#include "lbsph.h"

#ifdef __cplusplus
extern "C" {
#endif

#define LB_MLP_IN 8        /* features per sample                         */
#define LB_MLP_IN_PAD 16   /* padded input width (zeros beyond 8)          */
#define LB_MLP_HID 256     /* hidden width                                */
#define LB_MLP_OUT 21      /* lower triangle of L                         */
#define LB_MLP_OUT_PAD 32  /* padded output width                         */
#define LB_MLP_MAX_BATCH 65536

/* Parameter block, FP32, in this order (row-major, [out][in]):
 * W1[256][16], b1[256], W2[256][256], b2[256], W3[32][256], b3[32];
 * rows 21..31 of W3 and entries 21..31 of b3 are kept at zero, and so are
 * columns 8..15 of W1. */
#define LB_MLP_NPARAM (256 * 16 + 256 + 256 * 256 + 256 + 32 * 256 + 32)

typedef struct lb_mlp lb_mlp;

/* C = act(A B^T + bias), a BF16 x BF16 -> FP32 product on the tensor cores
 * (tcgen05.mma, kind::f16, FP32 accumulate in tensor memory), exposed for
 * tests and tools.  A(m, k) = A[m*a_sm + k*a_sk] (M x K), B(n, k) = B[n*b_sn +
 * k*b_sk] (N x K), BF16 as uint16 bit patterns, device memory.  bias (FP32,
 * [N], device) may be NULL; relu != 0 applies max(0, .).  C32 (FP32) and/or C16
 * (BF16) receive C(m, n) at [m*c_sm + n*c_sn]; either may be NULL.  M, N, K >= 1.
 * Errors: LB_EINVAL, LB_ECUDA, LB_ETIMEOUT (a tensor-core completion wait gave
 * up; detected at the next synchronising call of lb_mlp or lb_gemm_status). */
lb_status lb_gemm_bf16(const uint16_t* A, int64_t a_sm, int64_t a_sk, const uint16_t* B, int64_t b_sn,
                       int64_t b_sk, int32_t M, int32_t N, int32_t K, const float* bias, int32_t relu, float* C32,
                       uint16_t* C16, int64_t c_sm, int64_t c_sn, void* stream);

/* Waits for the device and returns LB_ETIMEOUT if any tensor-core wait of
 * lb_gemm_bf16 gave up since the last call (and clears the flag). */
lb_status lb_gemm_status(void);

/* Creates a network on `device` with all parameters zero and an Adam state
 * (beta1 0.9, beta2 0.999, eps 1e-8) for batches of up to max_batch samples. */
lb_status lb_mlp_create(int32_t device, int32_t max_batch, lb_mlp** out);
lb_status lb_mlp_destroy(lb_mlp* m);

/* Copies LB_MLP_NPARAM FP32 parameters from / to host memory (layout above);
 * set resets the Adam moments and step count.  Synchronous. */
lb_status lb_mlp_set_params(lb_mlp* m, const float* host);
lb_status lb_mlp_get_params(lb_mlp* m, float* host);

/* Forward pass for n samples.  x: device FP32 [n][8] features.  Writes, when
 * not NULL, y_dev (device FP32 [n][21], raw outputs) and R_dev (device FP32
 * [n][36], the predicted dimensionless R^ = L L^T, row-major). */
lb_status lb_mlp_forward(lb_mlp* m, const float* x_dev, int32_t n, float* y_dev, float* R_dev, void* stream);

/* Loss and gradients for n samples with targets Rt_dev (device FP32 [n][36]):
 * loss = (1/n) sum_s (1/36) sum_ij (R^_sij - Rt_sij)^2.  Writes the loss to
 * loss_dev (device FP32 [1]) and, when grad_dev is not NULL, the gradient of
 * every parameter (device FP32, LB_MLP_NPARAM, layout above). */
lb_status lb_mlp_loss_grad(lb_mlp* m, const float* x_dev, const float* Rt_dev, int32_t n, float* loss_dev,
                           float* grad_dev, void* stream);

/* One Adam step (learning rate lr) on the loss of lb_mlp_loss_grad for this
 * batch; loss_dev (may be NULL) receives the loss before the step. */
lb_status lb_mlp_train_step(lb_mlp* m, const float* x_dev, const float* Rt_dev, int32_t n, float lr,
                            float* loss_dev, void* stream);

/* Solves R^ (u) = (f) for n samples on the device, R^ symmetric positive
 * definite (Cholesky, FP64): R_dev FP32 [n][36], f_dev FP64 [n][6], u_dev FP64
 * [n][6].  Used for the warm-start velocities U, Omega = R^-1 (F_ext, T_ext). */
lb_status lb_spd_solve6(const float* R_dev, const double* f_dev, double* u_dev, int32_t n, void* stream);

/* Inverts n symmetric positive definite 6x6 matrices (FP64, device [n][36]) in
 * place and symmetrises the result: measured mobilities -> resistance targets. */
lb_status lb_spd_invert6(double* M_dev, int32_t n, void* stream);

/* Network inputs from geometry, per sample geom_dev[n][8] (FP64, device) =
 * (a, b, nu, L, e_x, e_y, e_z, rho0): long and short semi-axes, kinematic
 * viscosity, box edge (for several particles in one box: the edge of the volume
 * per particle), unit long axis e (e and -e give the same features: the sign is
 * taken so that e_z >= 0), fluid density.  x_dev[n][8] (FP32, device) =
 * (a/b - 2, b - 3, 10 (nu - 1/6), 10 b/L - 1, e, 1). */
lb_status lb_mlp_features(const double* geom_dev, int32_t n, float* x_dev, void* stream);

/* Training targets from measured mobilities: M_dev[n][36] (FP64, device; column
 * j = (U, Omega) at steady state per unit (F, T) along j) -> Rhat_dev[n][36]
 * (FP32) = (D M D)^-1, symmetrised, with D = diag(s_t I3, s_r I3), s_t^2 =
 * 6 pi mu b, s_r^2 = 8 pi mu b^3, mu = rho0 nu: the dimensionless resistance
 * tensor R^ = D^-1 R D^-1, the identity for a radius-b sphere in free space. */
lb_status lb_resistance_targets(const double* M_dev, const double* geom_dev, int32_t n, float* Rhat_dev,
                                void* stream);

/* Warm-start velocities: UW_dev[n][6] = (U, Omega) = R^-1 (F, T) with R =
 * D R^ D from a predicted Rhat_dev[n][36] (FP32) and FT_dev[n][6] = (F_ext,
 * T_ext) (FP64).  Cholesky in FP64 on the device. */
lb_status lb_warm_velocities(const float* Rhat_dev, const double* geom_dev, const double* FT_dev, int32_t n,
                             double* UW_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif
