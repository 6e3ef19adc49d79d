/*
 * mp_net — learned initial guess for the pressure solve: a small 3D U-Net
 * that maps the level set and the right-hand side to a pressure estimate,
 * run and trained with hand-written BF16 tensor-core (tcgen05) implicit-GEMM
 * convolution kernels, FP32 accumulation.
 *
 * The paper (arXiv 2312.11740) has no learned component; it names the
 * multigrid pressure solve (Grid_solvePoisson, Section 3) that this guess
 * feeds.  The network follows the stated reading: 4 levels with 16, 32, 64,
 * 64 channels, two 3x3x3 convolutions + ReLU per level, 2x2x2 average
 * pooling down, nearest upsampling + concatenation with the encoder output
 * up, a 1x1x1 head.  Inputs (two channels, zero-padded to 16):
 *   f0 = clip(phi / (4h), -1, 1),  f1 = bt / s,  s = rms(bt),
 * with bt the h^2-scaled, mean-free right-hand side.  Output q: the shape
 * of the pressure (trained on targets normalised to unit rms); the solver
 * fits its scale (energy-optimal alpha = (q.bt)/(q.A q)).
 *
 * Layouts: activations (nz, ny, nx, C) BF16, channels fastest; 3x3x3
 * weights [Cout][27][Cin], tap t = 9 dz + 3 dy + dx with offset
 * (dz-1, dy-1, dx-1); zero padding outside the grid.  Every dimension must
 * be a multiple of 32 (four levels of 8 x 4 x 4 voxel bricks).
 * Errors and streams follow include/mp_poisson.h.
 */
#ifndef MP_NET_H
#define MP_NET_H

#include <stddef.h>

#include "mp_poisson.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mp_net *mp_net_handle;

/*
 * Defines: no paper passage (the paper has no learned component); the 3x3x3 convolution
 * layer of the learned initial guess for Grid_solvePoisson (Section 3).
 *
 * Single 3x3x3 convolution (zero padding), for tests and building blocks.
 * y[v, co] = bias[co] + sum_{t, ci} x[v + off_t, ci] w[co, t, ci], ReLU if
 * relu != 0.  The input is the channel concatenation of xa (ca channels,
 * at half resolution when up_a != 0, read through nearest-neighbour
 * upsampling) and xb (cb channels, full resolution; NULL with cb = 0).
 * ca, cb, cout: multiples of 16, cout in {16, 32, 48, 64, 96, 128}.
 * w: [cout][27][ca+cb] BF16; bias: cout FP32 or NULL.  Output y (BF16)
 * or, when y32 is not NULL, FP32 into y32 instead.  All device pointers,
 * 16-byte aligned.  Grid dims multiples of 8 (x) and 4 (y, z).
 */
mp_status mp_conv3d_fwd(int nx, int ny, int nz, const void *xa, int ca, int up_a, const void *xb,
                        int cb, const void *w, const float *bias, int cout, int relu, void *y,
                        float *y32, void *stream);

/*
 * Defines: no paper passage (the paper has no learned component); the weight gradient
 * of the convolution, for training the network on the GPU.
 *
 * Weight gradient of mp_conv3d_fwd: dw[co, t, ci] = sum_v x[v + off_t, ci] g[v, co],
 * x as in mp_conv3d_fwd (concatenation of xa/xb), g (BF16, cout channels).
 * dw: FP32 [cout][27][ca+cb], overwritten.  Deterministic (fixed-order
 * split-K reduction).
 */
mp_status mp_conv3d_wgrad(int nx, int ny, int nz, const void *xa, int ca, int up_a,
                          const void *xb, int cb, const void *g, int cout, float *dw,
                          void *stream);

/* Defines: no paper passage (the paper has no learned component); the 4-level U-Net.
 * Create a network for an nx x ny x nz grid (multiples of 32).  All device
 * memory it needs is allocated here.  Parameters start at zero: set them
 * with mp_net_set_params (the caller draws the initial values). */
mp_status mp_net_create(mp_net_handle *out, int nx, int ny, int nz, void *stream);

/* Defines: no paper passage (the paper has no learned component); handle query.
 * Grid of the network. */
mp_status mp_net_dims(mp_net_handle net, int *nx, int *ny, int *nz);

/* Defines: no paper passage (the paper has no learned component); handle query.
 * Number of FP32 parameters (all conv weights and biases, then the head). */
size_t mp_net_param_count(mp_net_handle net);

/* Defines: no paper passage (the paper has no learned component); measurement.
 * Kernels the network has launched on inference paths (features, forward,
 * pressure) since creation. */
unsigned long long mp_net_launches(mp_net_handle net);

/* Defines: no paper passage (the paper has no learned component); parameter transfer.
 * Copy the FP32 master parameters in or out (device pointers, param_count
 * floats); setting them also refreshes the BF16 copies the kernels use. */
mp_status mp_net_set_params(mp_net_handle net, const float *params_dev);
mp_status mp_net_get_params(mp_net_handle net, float *params_dev);

/* Defines: no paper passage (the paper has no learned component); the network input,
 * the level set phi (Section 2, Fig. 2 caption sign) and the right-hand side.
 * Input features from phi (FP64) and the mean-free right-hand side b
 * (FP64) with bt = b_scale * b the h^2-scaled one (b_scale = h^2 for the
 * unscaled b of mp_poisson_rhs, 1 for the solver's scaled b): writes the
 * network input (16-channel BF16, internal buffer) and returns
 * s = rms(bt) (host).  h: cell size. */
mp_status mp_net_features(mp_net_handle net, const double *phi_dev, const double *b_dev, double h,
                          double b_scale, double *s_out);

/* Defines: no paper passage (the paper has no learned component); the input of a network
 * run on a grid half as fine as the solver's.
 * mp_net_features for fields on a grid `factor` (1 or 2) times finer than the
 * network's in every dimension (phi, b: device FP64 on that grid; h its cell
 * size): with factor 2 the features are formed from the means of the 8
 * children of every network cell (cell size 2h). */
mp_status mp_net_features_at(mp_net_handle net, int factor, const double *phi_dev,
                             const double *b_dev, double h, double b_scale, double *s_out);

/* Defines: no paper passage (the paper has no learned component); the initial guess
 * interpolated from the network's grid onto the solver's.
 * mp_net_pressure onto a grid `factor` (1 or 2) times finer: with factor 2,
 * p = s (q - mean q) interpolated trilinearly (cell-centred weights 3/4 and
 * 1/4 per axis; periodic axes wrap, wall axes clamp). p_dev: device FP64 on
 * the fine grid. */
mp_status mp_net_pressure_at(mp_net_handle net, int factor, const mp_bc bc[3], double s,
                             double *p_dev);

/* Defines: no paper passage (the paper has no learned component); input transfer.
 * The two used input channels (f0, f1) as a compact BF16 array (N*2), out
 * of or into the network input; set_input2 zero-fills the other 14. */
mp_status mp_net_get_input2(mp_net_handle net, void *x2_dev);
mp_status mp_net_set_input2(mp_net_handle net, const void *x2_dev);

/* Defines: no paper passage (the paper has no learned component); inference.
 * Forward pass on the current input features; q_dev: FP32 output (N). */
mp_status mp_net_forward(mp_net_handle net, float *q_dev);

/* Defines: no paper passage (the paper has no learned component); training on the GPU
 * on solutions the plain solver produces.
 * One training step on (features already set by mp_net_features or
 * mp_net_set_input, target q_target_dev FP32 N): forward, gauge-free MSE
 * loss, backward through every layer, Adam (lr, beta1 0.9, beta2 0.999,
 * eps 1e-8, bias correction with step >= 1).  loss_out (host) gets the
 * loss before the update. */
mp_status mp_net_train_step(mp_net_handle net, const float *q_target_dev, float lr, int step,
                            double *loss_out);

/* Defines: no paper passage (the paper has no learned component); training
 * checkpoint and resume.
 * Adam's first and second moment estimates (device FP32, param_count each):
 * get copies them out, set restores them (call after mp_net_set_params,
 * which zeroes them).  With the parameters, the step count and the sample
 * order they make a checkpoint from which training resumes exactly. */
mp_status mp_net_get_adam(mp_net_handle net, float *m_dev, float *v_dev);
mp_status mp_net_set_adam(mp_net_handle net, const float *m_dev, const float *v_dev);

/*
 * Defines: no paper passage (the paper has no learned component); the training loss;
 * the energy norm uses the ghost-fluid operator of the solve (varDens,
 * Section 3).
 *
 * Loss of mp_net_train_step.  kind 0: gauge-free mean squared error against
 * the target (default).  kind 1: energy norm,
 *   L = 1 - (q.A t)^2 / ((q.A q)(t.A t)),
 * the squared relative A-norm error of the best multiple of q, i.e. of the
 * guess the solver forms with its energy-optimal scale.  A is the
 * (positive semidefinite) variable-coefficient Laplacian whose ghost-fluid
 * face coefficients come from the phi channel of the current input
 * (f0 = phi / 4h is unclipped wherever a face crosses the interface), with
 * densities rho_l, rho_g and boundary conditions bc (as mp_poisson_setup).
 */
mp_status mp_net_set_loss(mp_net_handle net, int kind, double rho_l, double rho_g,
                          const mp_bc bc[3]);

/* Defines: no paper passage (the paper has no learned component); the loss gradient
 * that training feeds to the backward pass.
 * Forward pass on the current input and the loss of mp_net_train_step
 * (mp_net_set_loss) against q_target_dev (FP32, N) with its gradient with
 * respect to the network output q, without the backward pass or an update:
 * gq_dev (device FP32 N, may be NULL) gets dL/dq, loss_out (host, may be
 * NULL) the loss.  The gradient is the one mp_net_train_step feeds to the
 * backward pass, for tests and for callers who form their own updates. */
mp_status mp_net_loss_grad(mp_net_handle net, const float *q_target_dev, float *gq_dev,
                           double *loss_out);

/* Defines: no paper passage (the paper has no learned component); training on a
 * loss formed outside the network (the deflated energy of mp_poisson_deflated_energy).
 * One Adam step (as mp_net_train_step) from the gradient gq_dev = dL/dq (device FP32,
 * N) of the network output for the current input: forward, backward from gq_dev,
 * update. */
mp_status mp_net_train_step_grad(mp_net_handle net, const float *gq_dev, float lr, int step);

/* Defines: no paper passage (the paper has no learned component); input transfer.
 * Set the 16-channel BF16 input directly (device pointer, N*16 bf16). */
mp_status mp_net_set_input(mp_net_handle net, const void *x16_dev);

/* Defines: no paper passage (the paper has no learned component); the backward pass.
 * Gradients of sum(q * gq) w.r.t. all parameters for the current input
 * (no update): grad_dev gets param_count floats.  For tests. */
mp_status mp_net_backward(mp_net_handle net, const float *gq_dev, float *grad_dev);

/* Defines: no paper passage (the paper has no learned component); the initial guess on
 * the network's own grid.
 * Pressure shape from the last forward pass: p = s (q - mean q) (device,
 * N f64). */
mp_status mp_net_pressure(mp_net_handle net, double s, double *p_dev);

/* Defines: no paper passage (the paper has no learned component); the training target
 * from a pressure the plain solver produced.
 * Training target from a pressure field: q = (p - mean p) / rms(p - mean p)
 * (p: device N f64; q: device N f32). */
mp_status mp_net_make_target(mp_net_handle net, const double *p_dev, float *q_dev);

/* Defines: no paper passage (the paper has no learned component); configuration.
 * Stream for the network's work (cudaStream_t; NULL = legacy default). */
mp_status mp_net_set_stream(mp_net_handle net, void *stream);

/* Defines: no paper passage (test support for the error path of the bounded
 * waits).  Test only: the next n convolution launches of this process treat
 * the first wait of every CTA on its shared-memory staging barrier as timed
 * out.  That wait comes before any tensor-core instruction; the CTA then
 * waits (bounded, as always) for the copies it has already started,
 * releases its tensor memory and returns, and the call that launched it
 * returns MP_ERR_TIMEOUT.  Handles stay usable.  n = 0 cancels. */
mp_status mp_net_test_wait_timeout(int n);

/* Defines: no paper passage (the paper has no learned component); resource release. */
void mp_net_destroy(mp_net_handle net);

/* Defines: no paper passage (the paper has no learned component); the learned initial
 * guess of the multigrid solve (Grid_solvePoisson, Section 3), with the
 * residual check that falls back to the zero guess.
 * Use `net` (or NULL to detach) for initial_guess = 2 in mp_poisson_solve.
 * The network grid equals the solver grid, or is half of it in every
 * dimension (the guess is then formed on the coarser grid from restricted
 * features and interpolated, see mp_net_features_at / mp_net_pressure_at).
 * The solve builds the features from phi and b, runs the network, takes
 * p0 = alpha (q - mean q) with the energy-optimal alpha = (q.bt)/(q.A q),
 * and keeps it according to mp_opts.net_check (default: only if
 * ||b - A p0|| < ||b||; mp_stats.used_net, mp_stats.net_relres); otherwise
 * it starts from zero. */
mp_status mp_poisson_set_net(mp_handle hd, mp_net_handle net);

#ifdef __cplusplus
}
#endif

#endif /* MP_NET_H */
