/*
 * bfs_cno.h -- C ABI of the learned initial guess for bfs_solve: a small
 * convolutional neural operator on the nodal grid, trained on solutions the
 * solver itself produces.  An addition to the method: Newton's method
 * (Sec. 3.2) needs a starting iterate, and the paper starts from a flat free
 * surface (the uniform stream; Fig. 3) or from a solution of a nearby problem.
 * A network guess is used only through Newton, which must still reach the
 * same residual tolerance; nothing here changes what a converged solution is.
 *
 * Network: four dilated 3x3 convolutions (dilations 1, 3, 9, 27; channel
 * widths 16 -> 32 -> 32 -> 32 -> 16, of which 4 inputs and 3 outputs are
 * used), SiLU between layers, zero padding at the grid edge.  Weights and
 * activations are BF16 on the tensor cores with FP32 accumulation; master
 * weights and Adam moments are FP32.
 *
 * Conventions are those of bfs.h (status codes, device/host pointers, caller-
 * owned buffers, streams, one host thread per handle), and:
 *   - Images are on the nodal grid of a mesh: H = M rows (y), W = N columns (x).
 *   - x (features): device FP32, [Bt][H][W][4], channels
 *       0: (beta + 1) / 0.3   (bottom height above the flat bed)
 *       1: (F - 0.95) / 0.45  (Froude number, the same in every pixel)
 *       2, 3: x and y of the node, scaled to [-1, 1] over the mesh.
 *   - Outputs and targets: channels zeta, phi - x, psi - x at each node
 *     (phi and psi the velocity potential on the free surface and bottom,
 *     Sec. 2.2), divided by the per-channel output scales.
 *   - Parameters: FP32 vector of bfs_cno_num_params() values holding, layer
 *     by layer, the weights [cout][tap][cin] (tap = 3 ky + kx) then the
 *     cout biases.
 */
#ifndef BFS_CNO_H
#define BFS_CNO_H

#include "bfs.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bfs_cno bfs_cno;

/* Number of FP32 parameters of the network. */
int bfs_cno_num_params(void);

/* Create a network for H x W images and batches of up to Bmax images.  Its
   device memory (parameters, gradient, Adam moments, activations for Bmax
   images) is owned by the handle and freed by bfs_cno_destroy.  Parameters
   start at zero; set them with bfs_cno_set_params.  BFS_EINVAL for H < 3,
   W < 3, Bmax < 1 or out == NULL; BFS_ENOMEM when an allocation fails (*out is
   then NULL and the message is in bfs_cno_last_error(NULL)). */
int bfs_cno_create(int H, int W, int Bmax, bfs_cno **out);
void bfs_cno_destroy(bfs_cno *net);
const char *bfs_cno_last_error(const bfs_cno *net);

/* Load parameters (host FP32, bfs_cno_num_params values) and the three output
   scales (host FP32; NULL = 1, 1, 1); resets the Adam moments and step.
   Synchronous. */
int bfs_cno_set_params(bfs_cno *net, const float *params, const float *out_scale);

/* Copy the FP32 master parameters to params (host, bfs_cno_num_params
   values).  Synchronous. */
int bfs_cno_get_params(bfs_cno *net, float *params);

/* y = network(x) for Bt images.  x: device [Bt][H][W][4]; y: device FP32
   [Bt][H][W][16], channels 0..2 the scaled outputs, the rest unused.
   Asynchronous.  BFS_EINVAL unless 1 <= Bt <= Bmax. */
int bfs_cno_forward(bfs_cno *net, const float *x, int Bt, float *y, void *stream);

/* Gradient of the mean squared error between the outputs for x and target
   (device FP32 [Bt][H][W][3], scaled outputs) with respect to every
   parameter, into grad_host (host, bfs_cno_num_params values; may be NULL)
   and the loss into *loss_host (may be NULL).  Synchronous. */
int bfs_cno_gradient(bfs_cno *net, const float *x, const float *target, int Bt, float *grad_host,
                     float *loss_host, void *stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
   mean squared error of (x, target), laid out as for bfs_cno_gradient.
   Asynchronous; the loss before the step stays on the device for
   bfs_cno_read_loss. */
int bfs_cno_train_step(bfs_cno *net, const float *x, const float *target, int Bt, float lr, void *stream);

/* Loss of the last bfs_cno_gradient or bfs_cno_train_step into *loss_host.
   Synchronises stream. */
int bfs_cno_read_loss(bfs_cno *net, float *loss_host, void *stream);

/* Initial guess for ctx: the network on one image x (device [1][M][N][4] for
   ctx's mesh) -> nodal zeta, phi, psi -> unknown vector u (device FP64,
   length bfs_n_unknowns(ctx), the layout of bfs.h): q(x1, y_j) from the first
   node of each row, q_x by centred second-order differences (one-sided at the
   row ends).  Asynchronous.  BFS_EINVAL when the network's grid is not ctx's
   N x M nodes. */
int bfs_cno_guess(bfs_cno *net, bfs_ctx *ctx, const float *x, double *u, void *stream);

/* The learned start of a solve: u = the network's guess from the features x
   (device, as for bfs_cno_guess), then bfs_solve from it; the guess is
   accepted only through Newton to the solver's tolerance, and when that solve
   fails (BFS_ENOCONV, BFS_ELINESEARCH, BFS_EBREAKDOWN, BFS_ENAN, BFS_ETIMEOUT)
   u is reset to the uniform stream and solved again -- the method without the
   network.  u: device vector of bfs_n_unknowns(ctx).  st (optional) receives
   the counts and time of both solves summed, *used_fallback (optional) 1 if
   the uniform stream was needed.  Returns the final solve's status.
   Synchronous. */
int bfs_cno_solve(bfs_cno *net, bfs_ctx *ctx, const float *x, double *u, bfs_stats *st, int *used_fallback,
                  void *stream);

/* bfs_cno_solve on HOST buffers: the features x_host (M*N*4 floats, as for
   bfs_cno_guess) are copied to the device, the solution copied back into
   u_host (bfs_n_unknowns(ctx) doubles); both copies inside the call.
   Synchronous. */
int bfs_cno_solve_host(bfs_cno *net, bfs_ctx *ctx, const float *x_host, double *u_host, bfs_stats *st,
                       int *used_fallback, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* BFS_CNO_H */
