/*
 * h2nn -- kernels of the learned preconditioner: a small 3-D convolutional
 * network on the voxel grid that maps a residual to a correction, used as the
 * right preconditioner of flexible GMRES around the H^2 product. The paper
 * solves with an unpreconditioned BiCGStab (Sec. V); the network is the
 * learned-preconditioner pattern built around the same product (Sec. IV.B).
 *
 * Tensors are channel-last on a Dx x Dy x Dz voxel grid (voxel index
 * v = ix + Dx (iy + Dy iz)): a batch of B samples is [B][V][C], V = Dx Dy Dz.
 * Convolutions are 3x3x3, stride 1, zero padding 1, weights [Cout][27][Cin]
 * (tap t = dx + 3 (dy + 3 dz), neighbour offset (dx-1, dy-1, dz-1)), bias
 * [Cout]. Channel counts are 8, 16 or 32 (pad with zero channels).
 * bf16 tensors are passed as uint16 storage.
 * All pointers are DEVICE pointers owned by the caller; `stream` is a
 * cudaStream_t passed as void*; every call is asynchronous and returns
 * H2_ERR_ARG for unsupported shapes and H2_ERR_CUDA when a launch fails.
 */
#ifndef LIBH2_H2NN_H
#define LIBH2_H2NN_H

#include <stdint.h>

#include "h2.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Forward convolution (implicit GEMM on the tcgen05 tensor cores: M = 128
 * voxels per tile, N = Cout, K = 27 taps x Cin, bf16 products, FP32
 * accumulation in tensor memory):
 *   z[b][v][co] = bias[co] + sum_{t,ci} w[co][t][ci] in[b][v + off(t)][ci]
 *   out = ReLU(z) when relu != 0, else z.
 * in, w: bf16; bias: f32 or NULL; out_bf16 (bf16) and/or out_f32 (f32) may
 * each be NULL.
 */
h2_status h2nn_conv3d_fwd(const void *in, const void *w, const float *bias, void *out_bf16, float *out_f32,
                          int32_t B, int32_t Dx, int32_t Dy, int32_t Dz, int32_t Cin, int32_t Cout,
                          int32_t relu, void *stream);

/*
 * Weights of the data gradient: wt[ci][t][co] = w[co][26 - t][ci] (bf16), so
 * that the gradient with respect to the input of a convolution is
 * h2nn_conv3d_fwd(dz, wt, NULL, ...) with Cin and Cout exchanged.
 */
h2_status h2nn_flip_weights(const void *w, void *wt, int32_t Cin, int32_t Cout, void *stream);

/*
 * Weight and bias gradients: dw[co][t][ci] (+)= sum_{b,v} dz[b][v][co] in[b][v + off(t)][ci],
 * db[co] (+)= sum_{b,v} dz[b][v][co]. dz: f32 [B][V][Cout]; in: bf16;
 * dw, db: f32 (db may be NULL). accumulate = 0 overwrites, 1 adds.
 * dw on the tcgen05 tensor cores: M = (tap, ci) pairs, N = Cout, K = voxels;
 * in is bf16 (exact), dz is split into bf16 hi + lo and both products are
 * accumulated in FP32 (about 16 significant bits per term); db on CUDA cores.
 */
h2_status h2nn_conv3d_bwd_weight(const float *dz, const void *in, float *dw, float *db, int32_t B, int32_t Dx,
                                 int32_t Dy, int32_t Dz, int32_t Cin, int32_t Cout, int32_t accumulate,
                                 void *stream);

/* H2_ERR_TIMEOUT if a bounded wait inside a tensor-core convolution ran out
   since the last call (that launch skipped its output), else H2_OK;
   synchronises the device and clears the flag. */
h2_status h2nn_device_status(void);

/* dz = dy * (y > 0) (ReLU backward from the layer's output y), count entries;
   dy f32, y bf16, dz f32 (dz may alias dy). */
h2_status h2nn_relu_bwd(const float *dy, const void *y, float *dz, int64_t count, void *stream);

/* out = in converted to bf16 (count entries). */
h2_status h2nn_f32_to_bf16(const float *in, void *out, int64_t count, void *stream);

/*
 * Mean-square loss and its gradient against a target:
 *   loss_parts[b] = sum_{v,c<Cu} (out - target)^2 / sum (target)^2 per sample b,
 *   grad = d(mean_b loss_parts[b]) / d(out) with the denominators held fixed,
 *   zero on the padding channels c >= Cu.
 * out, target, grad: f32 [B][V][C]; loss_parts: f32 [2B] (entries B..2B-1 are
 * scratch; on return they hold the per-sample sums of target^2).
 */
h2_status h2nn_mse(const float *out, const float *target, float *grad, float *loss_parts, int32_t B, int64_t V,
                   int32_t C, int32_t Cu, void *stream);

/*
 * Adam step on FP32 master parameters p with gradient g and moments m, v
 * (Kingma & Ba): p -= lr * mhat / (sqrt(vhat) + eps); also writes the bf16
 * copy p_bf16 (may be NULL). step counts from 1.
 */
h2_status h2nn_adam(float *p, const float *g, float *m, float *v, void *p_bf16, int64_t count, float lr,
                    float beta1, float beta2, float eps, int32_t step, void *stream);

/*
 * Residual vector <-> network channels. The vector holds 3 complex unknowns per
 * voxel in tree order (unknown 3 p + c is component c of the voxel at tree
 * position p); grid_of[p] is that voxel's grid index.
 * pack: chan[b][v][0..5] = scale_b * (Re, Im) of components x, y, z of vector
 * b at voxel v, chan[b][v][6] = aux[v] (may be NULL: 0), chan[b][v][7] = 0;
 * chan is bf16 with C = 8 channels. vec: c128 [B][3 nv] (column stride ldv).
 * unpack: vec[b][unknown] = scale_b * (chan[b][v][2c] + i chan[b][v][2c+1])
 * from f32 channels [B][V][C] (C >= 6). scale: f64 [B] (NULL: 1).
 */
h2_status h2nn_pack(const void *vec, int64_t ldv, const int32_t *grid_of, const float *aux, const double *scale,
                    void *chan, int32_t B, int32_t nv, int64_t V, void *stream);
h2_status h2nn_unpack(const float *chan, int32_t C, const int32_t *grid_of, const double *scale, void *vec,
                      int64_t ldv, int32_t B, int32_t nv, int64_t V, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LIBH2_H2NN_H */
