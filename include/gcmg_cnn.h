/* Learned initial guess for the multigrid solve: C ABI of the network in
 * libgcmg.so.  The paper has no learned part; this network (six 3x3
 * convolution layers, channels 4 -> 32 -> 32 -> 32 -> 32 -> 32 -> 2, ReLU
 * after the first five, dilation d_l per layer) maps the problem data of a
 * 2D domain -- level set phi, h^2 f, boundary data g and a boundary-type mask
 * on the grid -- to an approximation of the solution that the V-cycle then
 * starts from; the V-cycle's FP64 defect decides convergence, so the network
 * never changes the converged result.  Operands are BF16 with FP32
 * accumulation on the tcgen05 tensor cores; training (forward, backward,
 * Adam) runs on the same kernels.
 *
 * Memory: every pointer named *_dev is caller-owned device memory, borrowed
 * for the call; *_host pointers are host memory.  Images are FP32, NCHW:
 * input [batch][4][H][W], output [batch][2][H][W].  Parameters are one FP32
 * vector: per layer the weights [C_out][C_in][3][3] followed by the biases
 * [C_out] (gcmg_cnn_num_params() values in all).  All work runs on the
 * stream given at creation; every call returns after it has completed.
 * Errors: GCMG_E_ARG (bad argument), GCMG_E_OOM, GCMG_E_CUDA, and
 * GCMG_E_TIMEOUT when a bounded tensor-core wait runs out (the context stays
 * usable). */
#ifndef GCMG_CNN_H
#define GCMG_CNN_H

#include <stdint.h>

#include "gcmg.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gcmg_cnn gcmg_cnn;

/* Number of FP32 parameters of the network. */
int64_t gcmg_cnn_num_params(void);

/* A network for batches of `batch` images of H x W pixels; dilations[6]
 * (each in [1, 96]; NULL: 1, 3, 9, 27, 81, 1).  Parameters start at zero. */
gcmg_status gcmg_cnn_create(int batch, int H, int W, const int *dilations, void *stream, gcmg_cnn **out);
void gcmg_cnn_destroy(gcmg_cnn *net);
const char *gcmg_cnn_last_error(const gcmg_cnn *net);

/* Sets (and resets the optimiser state) / reads the parameter vector. */
gcmg_status gcmg_cnn_set_params(gcmg_cnn *net, const float *params_host, int64_t count);
gcmg_status gcmg_cnn_get_params(gcmg_cnn *net, float *params_host, int64_t count);

/* out_dev[batch][2][H][W] = network(in_dev[batch][4][H][W]). */
gcmg_status gcmg_cnn_forward(gcmg_cnn *net, const float *in_dev, float *out_dev);

/* The BF16 activation entering layer `layer` (0: the input, 4 channels;
 * 1..5: 32 channels) of the last forward pass, as FP32 [batch][C][H][W]. */
gcmg_status gcmg_cnn_activation(gcmg_cnn *net, int layer, float *dst_dev);

/* Parameter gradients (the layout of the parameter vector) of a loss whose
 * derivative with respect to the last forward pass's output is dout_dev
 * [batch][2][H][W]. */
gcmg_status gcmg_cnn_backward(gcmg_cnn *net, const float *dout_dev, float *grad_dev);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on the
 * batch's loss (target, mask: [batch][2][H][W])
 *   L = sum(m_0 (out_0 - target_0)^2) / mask_count
 *     + lap_weight sum_{m_1 = 1} s^2 / lap_count,
 * where e = (out_0 - target_0) m_0 is the error of channel 0 and
 * s = e_N + e_S + e_E + e_W - 4 e (h^2 times its 5-point Laplacian) is taken
 * at the pixels whose mask channel 1 is 1 (and not on the image edge): the
 * second term weighs the error by the residual it leaves.  lap_weight = 0
 * drops it; output channel 1 is not trained.  loss_host receives L before
 * the step. */
gcmg_status gcmg_cnn_train_step(gcmg_cnn *net, const float *in_dev, const float *target_dev, const float *mask_dev,
                                float mask_count, float lap_weight, float lap_count, float lr, double *loss_host);

#ifdef __cplusplus
}
#endif

#endif
