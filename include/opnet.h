/*
 * opnet.h - C ABI of the learned warm start for the orthogonality-preserving
 * eigensolver (opevo.h).
 *
 * The paper (arXiv 2511.06788) evolves any orthonormal U^0 to the lowest-p
 * eigenspace, and converges from any start whose energy lies below the
 * excited-state level (the basin condition of §3).  This extension maps the
 * potential V to a starting block by a small convolutional network:
 *
 *   Y = net(V)  (n x p)  ->  op_init / op_init_device orthonormalises Y once
 *   (Cholesky-QR, FP64)  ->  the plain scheme (op_step / op_solve).
 *
 * The scheme is unchanged; its own steps decide the result.
 *
 * Network: a 3-level U-Net on an N^3 grid, N % 4 == 0.  Tensors are
 * channels-last [grid point][channel], with the point ordering of opevo.h.
 *
 *   layer  input                  taps  Cin      Cout  grid
 *   0 e0a  x0 = [V/6, x^, y^, z^]  27   4        c0    N
 *   1 e0   e0a                     27   c0       c0    N
 *   2 e1a  pool(e0)                27   c0       c1    N/2
 *   3 e1   e1a                     27   c1       c1    N/2
 *   4 b2a  pool(e1)                27   c1       c2    N/4
 *   5 b2   b2a                     27   c2       c2    N/4
 *   6 d1a  [up(b2), e1]            27   c2 + c1  c1    N/2
 *   7 d1   d1a                     27   c1       c1    N/2
 *   8 d0a  [up(d1), e0]            27   c1 + c0  c1    N
 *   9 d0   d0a                     27   c1       c1    N
 *  10 out  d0                      1    c1       p     N
 *
 * - x^ = 2 (x - lo) / (hi - lo) - 1 is the box coordinate of the point.
 * - Layers 0-9 apply silu(z) = z / (1 + e^-z) to a 3x3x3 zero-padded
 *   cross-correlation plus bias; tap t = (dz+1)*9 + (dy+1)*3 + (dx+1) reads
 *   the point (x+dx, y+dy, z+dz).
 * - pool is the 2x2x2 mean; up is nearest-neighbour x2; [a, b] concatenates
 *   channels.
 * - Layer 10 is linear.
 * - Parameters are one flat FP32 vector: per layer, W (taps x Cin x Cout,
 *   row-major) then b (Cout).
 *
 * Training loss (rotation- and scale-invariant), for a converged block U*
 * with orthonormal columns.  With G = Y^T Y, P = U*^T Y, b = tr G and
 * Gh = p G / b:
 *
 *   L = (1 - ||P||_F^2 / b) + gamma ||Gh - I||_F^2 / p^2
 *
 * The first term is the share of ||Y||^2 outside span U*.  The second makes
 * the columns orthogonal and of equal norm.  L = 0 exactly when Y = c U* Q with
 * Q orthogonal.
 *
 * Parameters are updated by Adam (Kingma and Ba, 2015), FP32 master weights.
 *
 * Conventions: as opevo.h.  The forward convolutions and the data gradients of layers
 * with at most 128 input channels run on the tensor cores with BF16 operands and FP32
 * accumulation (opnet_set_conv selects FP32 CUDA cores); the rest is FP32 with FP32
 * accumulation inside a layer; the loss's p x p algebra is FP64.  Device pointers are
 * 16-byte aligned and caller-owned.  Calls are ordered on the network's stream and
 * return after it has been synchronised, except where stated.
 */
#ifndef OPNET_H
#define OPNET_H

#include "opevo.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct opnet opnet;

typedef struct {
  int N;                 /* grid points per axis; N % 4 == 0, 4 <= N <= 512      */
  double lo[3], hi[3];   /* the box (only the features use it)                  */
  int p;                 /* output columns; p % 8 == 0, 8 <= p <= 128              */
  int width[3];          /* channels c0, c1, c2 of the three levels, each 1..128  */
  void *stream;          /* cudaStream_t for all of this network's work (NULL: legacy) */
} opnet_config;

/* Allocate a network and all of its device buffers for one grid size.  The
 * parameters are zero until opnet_set_params. */
op_status opnet_create(opnet **net, const opnet_config *cfg);

/* Number of FP32 parameters, or -1 for a NULL net. */
long long opnet_param_count(const opnet *net);

/* Shape of layer i (0..10, table above); OP_ERR_ARG past the last layer. */
op_status opnet_layer(const opnet *net, int i, int *taps, int *cin, int *cout);

/* Copy `count` (= opnet_param_count) parameters from / to host memory.  Setting
 * resets the Adam moments and step counter. */
op_status opnet_set_params(opnet *net, const float *theta_host, long long count);
op_status opnet_get_params(opnet *net, float *theta_host, long long count);

/* Arithmetic of the forward convolutions (the 11 layers of every forward pass, in
 * inference and in training):
 *   OPNET_CONV_BF16_TC  tcgen05 tensor cores, BF16 operands (activations and weights
 *                       rounded to nearest), FP32 accumulation; the default;
 *   OPNET_CONV_FP32     FP32 CUDA cores, FP32 accumulation.
 * In training, the data gradients of the layers (opnet_conv_dgrad's arithmetic) follow the
 * same choice for layers with at most 128 input channels, and run on the FP32 CUDA cores
 * otherwise; the weight gradients and the rest of the backward pass are FP32 either way.
 * OP_ERR_ARG for a NULL net or another kind. */
typedef enum { OPNET_CONV_FP32 = 0, OPNET_CONV_BF16_TC = 1 } opnet_conv_kind;
op_status opnet_set_conv(opnet *net, int kind);

/* One convolution layer on its own (the network's kernels, for kernel-level checks):
 * Z = conv(X, W) + bias and A = silu(Z), X [N^3][cin], W [taps * cin][cout] (row-major,
 * the parameter layout above), bias [cout] or NULL, Z and A [N^3][cout] (either may be
 * NULL), all FP32 device arrays; taps 27 (3x3x3, zero padded) or 1; 1 <= cout <= 128,
 * cin <= 512, N <= 512; X 16-byte aligned.  `kind` as opnet_set_conv.  Allocates and
 * frees a small scratch and synchronises `stream` (cudaStream_t, may be NULL). */
op_status opnet_conv(int kind, const float *X, int N, int taps, int cin, int cout,
                     const float *W, const float *bias, float *Z, float *A, void *stream);

/* The data gradient of that layer (the network's backward kernels, for kernel-level
 * checks): dX = d loss / d X for dZ = d loss / d Z, i.e. the adjoint of the correlation,
 *   dX[m][ci] = sum_t sum_co dZ[m - off_t][co] W[t cin + ci][co]   (zero outside the grid),
 * computed as the forward convolution of dZ with the tap-reversed, transposed weights.
 * dZ [N^3][cout] (16-byte aligned), W [taps * cin][cout], dX [N^3][cin], FP32 device
 * arrays; taps 27 or 1; cin, cout <= 512, N <= 512.  OPNET_CONV_BF16_TC: on the tensor
 * cores (BF16 dZ and W, FP32 accumulation) when cin <= 128, else as OPNET_CONV_FP32 (FP32
 * CUDA cores).  Allocates and frees a small scratch and synchronises `stream`. */
op_status opnet_conv_dgrad(int kind, const float *dZ, int N, int taps, int cin, int cout,
                           const float *W, float *dX, void *stream);

/* Y = net(V): V is N^3 FP64 values (device), Y is N^3 x p FP32 (device, ld = p). */
op_status opnet_forward(opnet *net, const double *V_dev, float *Y_dev);

/* The warm start: Y = net(V) written as an N^3 x p FP64 block (device, ld = p),
 * ready for op_init_device, which orthonormalises it (Cholesky-QR). */
op_status opnet_infer(opnet *net, const double *V_dev, double *U0_dev);

/* Loss at the current parameters for the target Ustar (N^3 x p FP32 device,
 * ld = p, orthonormal columns).  Also the full gradient, when grad_host (count
 * floats, host) is not NULL. */
op_status opnet_loss_grad(opnet *net, const double *V_dev, const float *Ustar_dev, double gamma,
                          double *loss, float *grad_host, long long count);

/* One Adam step (step size lr, beta1, beta2, eps) on the loss for (V, Ustar); *loss
 * receives the loss before the step. */
op_status opnet_train_step(opnet *net, const double *V_dev, const float *Ustar_dev,
                           double gamma, double lr, double beta1, double beta2, double eps,
                           double *loss);

void opnet_destroy(opnet *net);

#ifdef __cplusplus
}
#endif

#endif /* OPNET_H */
