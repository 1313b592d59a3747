/*
 * exx_guess.h -- C ABI of the learned CG warm start (a 3D U-Net).
 *
 * The paper starts every pair solve from an initial guess and names better
 * guesses as a way to cut CG iterations (Sec. III.C Step IV; conclusions);
 * it does not use a network. This library adds one: a 3D U-Net that maps the
 * pair density rho_ij on a cube of S^3 grid points centred on the pair's grid
 * point g_ij to a guess of v_ij on the same cube. The solver's
 * warm_start = 2 option (exx.h) runs it before the CG, which still decides
 * the result (the stop rule is relative to ||b||, so a poor guess costs
 * iterations, never accuracy).
 *
 * Network: 4 levels of widths 16/32/64/128, two 3x3x3 convolutions with ReLU
 * per level (zero padding), 2x2x2 average pooling down, nearest up-sampling
 * and channel concatenation with the level's skip tensor up, a 1x1x1 head.
 * Activations and weights BF16 (channels last), accumulation FP32; all
 * 3x3x3 convolutions after the input layer run on the tcgen05 tensor cores.
 *
 * Sample layout (every array FP32, C order):
 *   input  [batch][S][S][S][3]: channel 0 = rho(o) / s on the PE ball and 0
 *          elsewhere; channel 1 = the multipole boundary values: outside the
 *          PE ball, the expansion of Eq. me (moments of Eq. mepole of rho / s
 *          over the ball points in the cube, l <= l_max, in FP32) divided by
 *          delta^2, and 0 on the ball; channel 2 = 1 on the PE ball
 *          (|o|^2 <= R_PE^2) and 0 elsewhere; cube voxel (z, y, x) is the
 *          offset o = (z, y, x) - S/2 (axes in the orbital-array order); s =
 *          max |rho| on the ball.
 *   target / output [batch][S][S][S]: v(o) / (s delta^2), delta^2 the
 *          geometric mean of the squared spacings.
 * Loss: sum over the batch of (output - target)^2 on ball voxels, divided by
 * batch * S^3.
 *
 * Parameters: exx_guess_param_count() FP32 values, layers in the order
 *   in(3->16) c0b(16->16) c1a(16->32) c1b(32->32) c2a(32->64) c2b(64->64)
 *   c3a(64->128) c3b(128->128) u2a(192->64) u2b(64->64) u1a(96->32)
 *   u1b(32->32) u0a(48->16) u0b(16->16) head(16->1)
 * each as W[27][cin][cout] (tap = 9 dz + 3 dy + dx over offsets -1..1 in the
 * z, y, x order above) then bias[cout]; the head is w[16] then b[1]. A model
 * blob for exx_load_guess_model is four int32 {0x47585845, 2, S, count}
 * followed by the count parameters.
 *
 * Errors: every function returns an exx_status; exx_last_error(NULL)
 * describes the last failure of a function in this header.
 */
#ifndef EXX_GB300_GUESS_H
#define EXX_GB300_GUESS_H

#include <stddef.h>
#include "exx.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct exx_guess exx_guess;

/* Number of FP32 parameters of the network. */
size_t exx_guess_param_count(void);

/*
 * Creates a network for cubes of side S (a multiple of 8, 16 <= S <= 64) and
 * up to batch_max samples per call (1..1024); parameters start at zero.
 * Device memory is about batch_max * S^3 * 1.2 kB. EXX_EINVAL on bad sizes,
 * EXX_ENOMEM / EXX_ECUDA on allocation failure.
 */
exx_status exx_guess_create(exx_guess **out, int S, int batch_max);

/* Host FP32 parameter vector in and out (n must equal the parameter count). */
exx_status exx_guess_set_params(exx_guess *g, const float *params, size_t n);
exx_status exx_guess_get_params(exx_guess *g, float *params, size_t n);

/*
 * Inference. input: device [batch][S^3][3]; output: device [batch][S^3].
 * stream: cudaStream_t (NULL = legacy default); the call is stream-ordered
 * and synchronises only to read the tensor-core time-out flag.
 */
exx_status exx_guess_forward(exx_guess *g, const float *input, float *output, int batch, void *stream);

/*
 * Forward and backward pass: loss (host, may be NULL) and the gradient of the
 * loss with respect to every parameter (host [count], may be NULL).
 */
exx_status exx_guess_gradient(exx_guess *g, const float *input, const float *target, int batch, float *loss,
                              float *grad, void *stream);

/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on one batch; loss before the step. */
exx_status exx_guess_train_step(exx_guess *g, const float *input, const float *target, int batch, float lr,
                                float *loss, void *stream);

void exx_guess_destroy(exx_guess *g);

/*
 * Training samples from a solved call: after exx_compute on ctx with
 * warm_start = 1 (which keeps every pair's converged v on its PE ball), writes
 * for the first min(count, cap) pairs of that call's list the network input
 * and target on a cube of side S (even, 8..128) as laid out above.
 *   orbitals  device, the same array the call used (EXX_EINVAL otherwise)
 *   input     device [cap][S^3][3]; target device [cap][S^3]
 *   count     host, receives the call's pair count
 * Synchronises the context's work and the given stream. Errors are reported
 * through exx_last_error(ctx).
 */
exx_status exx_export_samples(exx_ctx *ctx, const double *orbitals, int S, float *input, float *target, int cap,
                              int *count, void *stream);

/*
 * One 3x3x3 convolution (zero padding) on the tensor-core path, for tests.
 *   x     device BF16 [batch][D][H][W][cin], channels last
 *   w     device FP32 [27][cin][cout] (tap order as above)
 *   bias  device FP32 [cout] or NULL
 *   mask  device BF16 [batch][D][H][W][cout] or NULL
 *   y     device BF16 [batch][D][H][W][cout]
 *   mode  0: y = conv + bias; 1: y = ReLU(conv + bias);
 *         2: data gradient: y has cin channels, x has cout:
 *            y[v][ci] = sum_tap sum_co x[v - (tap offset)][co] w[tap][ci][co],
 *            times (mask[v][ci] > 0) when mask is given (mask then has cin channels)
 * cin, cout multiples of 16 in [16, 256]. Allocates and frees a packed copy
 * of w; synchronises the stream.
 */
exx_status exx_unet_conv3d(const void *x, const float *w, const float *bias, const void *mask, void *y, int batch,
                           int D, int H, int W, int cin, int cout, int mode, void *stream);

#ifdef __cplusplus
}
#endif

#endif
