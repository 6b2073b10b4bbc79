/*
 * mmx_residual.h -- C ABI of the learned residual correction of the
 * extrapolated demag field (part of libmmx).
 *
 * The paper's method (Sec. II, Eq. 6) replaces the demag field at the RK
 * sub-steps by a polynomial extrapolation of the non-self field G = H_d +
 * N00 M from the last p+1 exact evaluations.  It has no learned component;
 * this extension trains a small convolutional net to predict the
 * extrapolation's error from the stage state, so that G_ext + Ms r is a
 * corrected non-self field.  The net:
 *   - input x: 6 channels (m, G_ext / Ms) on the mesh, FP32, layout
 *     [6][nz][ny][nx] (x fastest);
 *   - output r: 3 channels, (G - G_ext) / Ms, FP32, layout [3][nz][ny][nx];
 *   - four 3x3x3 cross-correlation layers with zero padding, 6 -> 32 -> 32
 *     -> 32 -> 3 channels, a bias per output channel, ReLU after the first
 *     three; tap t = (tz*3 + ty)*3 + tx reads (z+tz-1, y+ty-1, x+tx-1);
 *   - BF16 operands rounded to nearest even (the input, every weight, and
 *     each hidden layer's output after its ReLU) on the tensor cores with
 *     FP32 accumulation; biases FP32; the output is not rounded;
 *   - parameters: MMX_RNET_PARAMS FP32 values, per layer W[27][cout][cin]
 *     then b[cout];
 *   - training: loss = mean over cells and channels of (r - target)^2,
 *     gradients through the rounded weights and stored activations
 *     (roundings as identity), Adam with beta1 0.9, beta2 0.999, eps 1e-8
 *     and bias-corrected moments on the FP32 master parameters.
 *
 * Ownership and errors follow mmx.h: every pointer passed in stays owned by
 * the caller; the net owns its device buffers (parameters, Adam moments,
 * activations for up to max_cells cells) and frees them in
 * mmx_rnet_destroy; work is enqueued on the stream given at create; calls
 * return MMX_OK or a negative MMX_ERR_* code, with the text from
 * mmx_rnet_last_error.  Any mesh size nx, ny, nz >= 1 with nx*ny*nz <=
 * max_cells is accepted.
 */
#ifndef MMX_RESIDUAL_H
#define MMX_RESIDUAL_H

#include "mmx.h"

#ifdef __cplusplus
extern "C" {
#endif

#define MMX_RNET_PARAMS 63171

typedef struct mmx_rnet mmx_rnet;

/* Allocates a net for meshes of up to max_cells cells, parameters zero.
 * MMX_ERR_ARG for max_cells < 1 or > 2^26; MMX_ERR_OOM. */
int mmx_rnet_create(long long max_cells, void *cuda_stream, mmx_rnet **out);

/* Copies MMX_RNET_PARAMS FP32 values from / to host memory and resets the
 * Adam moments and step count (set only).  Synchronises the stream. */
int mmx_rnet_set_params(mmx_rnet *net, const float *params_host);
int mmx_rnet_get_params(mmx_rnet *net, float *params_host);

/* r = net(x): x_dev and r_dev are device FP32 arrays of 6 and 3 channels on
 * an nx*ny*nz mesh (layouts above); r_dev may be NULL (the output stays in
 * the net's own buffer, readable with mmx_rnet_get_activation). */
int mmx_rnet_forward(mmx_rnet *net, int nx, int ny, int nz, const float *x_dev, float *r_dev);

/* One Adam step at learning rate lr on the pair (x_dev, target_dev), both
 * device FP32 ([6][cells] and [3][cells]); *loss_out (may be NULL) receives
 * the loss before the update, which synchronises the stream. */
int mmx_rnet_train_step(mmx_rnet *net, int nx, int ny, int nz, const float *x_dev, const float *target_dev,
                        float lr, double *loss_out);

/* Gradient of the last train step (MMX_RNET_PARAMS FP32 values) to host
 * memory.  Synchronises the stream. */
int mmx_rnet_get_grads(mmx_rnet *net, float *grads_host);

/* Copies what the last forward or train step left in the net to host
 * memory: for layer 0..3 the BF16 input of that layer, channels last
 * [cells][16] for layer 0 (channels 6..15 zero) and [cells][32] for 1..3, as
 * raw 16-bit patterns; for layer 4 the FP32 output r [3][cells].  bytes
 * must equal that size.  Synchronises the stream. */
int mmx_rnet_get_activation(mmx_rnet *net, int layer, void *dst_host, size_t bytes);

const char *mmx_rnet_last_error(const mmx_rnet *net);
void mmx_rnet_destroy(mmx_rnet *net);

/* Training pair of the net from a context's exact demag (Eq. 2) and Eq. 6's
 * extrapolation, at time t for state m:
 *   x = (m, G_ext / Ms),  target = (G(m) - G_ext) / Ms,
 *   G_ext = sum_i L_i(t) G(m_i), L_i the Lagrange basis on the p+1 node
 *   times t_nodes (tau = t - t_nodes[p] in FP64, on the host).
 * m_nodes_dev: device array [p+1][3][nz][ny][nx] of the context's element
 * type (the states at t_nodes); m_dev: [3][nz][ny][nx]; x_dev, target_dev:
 * device FP32 [6][cells] and [3][cells].  The sums run in the context's
 * precision.  0 <= p <= 5; node times distinct.  Uses the context's demag
 * scratch buffer, not the integrator state. */
int mmx_residual_sample(mmx_ctx *ctx, int p, const void *m_nodes_dev, const double *t_nodes, const void *m_dev,
                        double t, float *x_dev, float *target_dev);

/* Attaches net to an FP32 context that extrapolates (extrap_order >= 0), or
 * detaches it (net = NULL).  While attached, every extrapolated stage k >= 2
 * of an attempt (Eq. 4-6) uses the non-self field G_ext + Ms r with r =
 * net(Y_k, G_ext / Ms) instead of G_ext; stage 1 and the priming steps keep
 * the exact evaluation.  Exact demag (Eq. 2) is the fallback: an attempt
 * whose error estimate (Eq. 3-5) exceeds e_max is retried, with the step the
 * controller proposes, with exact demag at every stage; and with a periodic
 * check configured (mmx_set_residual_check) every check_every accepted
 * steps one attempt runs with exact demag at every stage and compares the
 * net's corrected field with the exact one at stage 2 — while the last check
 * exceeds its tolerance, every attempt runs with exact demag.  The choice is
 * made on the device by the controller (conditional graph nodes; no host
 * round trip).  The net's parameters are read at each use (train it between
 * runs if wanted); it must outlive the attachment, including any batch
 * built while it is attached, and must not be used by another context's run
 * at the same time.  Attaching resets the check state (the net counts as
 * passing).  MMX_ERR_ARG for an FP64 context, extrap_order < 0 or a net
 * created for fewer cells than the mesh; MMX_ERR_OOM when the check's
 * scratch field (3 x cells FP32) cannot be allocated.  Synchronises the
 * context's stream and drops its captured attempt graphs (rebuilt at the
 * next run). */
int mmx_set_residual(mmx_ctx *ctx, mmx_rnet *net);

/* The periodic exact check of an attached net: every `every` accepted steps
 * (0: never) one attempt runs with exact demag at every stage, and the net's
 * corrected field at its stage 2 must satisfy max|G_net - G| <= tol max|G|
 * (max over cells and components); otherwise the following attempts run
 * with exact demag until a later check passes.  No counterpart in the
 * paper (the learned residual is this library's addition).  Defaults: 0 and
 * 0.  MMX_ERR_ARG for every < 0 or tol not finite and >= 0.  Synchronises
 * the stream and drops the captured attempt graphs. */
int mmx_set_residual_check(mmx_ctx *ctx, int every, double tol);

/* Counters of the learned residual's fallback since the context was created:
 * out4[0] attempts with the net rejected by the error estimate (each retried
 * with exact demag), out4[1] periodic checks run, out4[2] checks that
 * exceeded their tolerance, out4[3] 1 while the net passes (its last check
 * within tolerance).  Synchronises the stream. */
int mmx_residual_stats(mmx_ctx *ctx, long long *out4);

#ifdef __cplusplus
}
#endif

#endif
