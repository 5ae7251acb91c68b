/*
 * archer_denoise.h -- C ABI of the EPID-image denoiser (a learned denoiser of
 * low-count Monte Carlo EPID images, the extension the paper names as future
 * work in Sec. 5).  Built into the same library as archer_epid.h and sharing
 * its status codes.
 *
 * The network is a stated reading of that one-line proposal: a 2D U-Net with
 * `levels` levels of base_channels * 2^l channels.  Encoder level l: two 3x3
 * convolutions (zero padding) with bias and ReLU, 2x2 max pooling between
 * levels; decoder level l: nearest-neighbour 2x upsampling of the level below,
 * concatenated (upsampled channels first) with the encoder output of level l,
 * two 3x3 convolutions with ReLU; output: a 1x1 convolution to one channel.
 * Loss: mean squared error; optimiser: Adam (Kingma and Ba 2015, Algorithm 1,
 * beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected).
 *
 * Numerics: activations, weights as MMA operands and propagated gradients are
 * bfloat16; every convolution accumulates in float32 on the tensor cores
 * (tcgen05, TMEM accumulators); master weights, weight gradients and the Adam
 * moments are float32; the loss is reduced in float64.
 *
 * Parameter vector (float32, the order of dn_get_params / dn_set_params):
 * for each convolution in the order enc0a, enc0b, enc1a, enc1b, ...,
 * enc{L-1}b, dec{L-2}a, dec{L-2}b, ..., dec0a, dec0b, out: its weights
 * [Co][k][k][Ci] then its biases [Co]; Ci of dec{l}a is the concatenation
 * (upsampled channels, then skip channels).
 *
 * Tensors of the primitive calls are NHWC bfloat16 device arrays passed as
 * uint16_t*; channel counts must be multiples of 8 (pad with zeros).
 * Conventions as in archer_epid.h: plain pointers, caller-owned buffers,
 * mc_status results, work ordered on `stream`.
 */
#ifndef ARCHER_DENOISE_H
#define ARCHER_DENOISE_H

#include <stddef.h>
#include <stdint.h>

#include "archer_epid.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dn_ctx dn_ctx;

typedef struct dn_config {
    int height, width;        /* image size; multiples of 2^(levels-1) */
    int batch;                /* images per step */
    int levels;               /* U-Net levels, 2..5 (4) */
    int base_channels;        /* channels of level 0: 32 (a multiple of 32; 32 * 2^(levels-1) <= 256) */
    int in_channels;          /* input planes, 1..8 (1): the noisy image, then auxiliary maps */
    uint64_t seed;            /* He-normal initialisation of the weights (biases 0) */
} dn_config;

void dn_config_default(dn_config* cfg);

/* Allocates the network, its activations, gradients and optimiser state on
 * `device` and initialises the weights. */
mc_status dn_create(const dn_config* cfg, int device, dn_ctx** out);
mc_status dn_destroy(dn_ctx* ctx);
const char* dn_last_error(const dn_ctx* ctx);

/* Number of float32 parameters. */
mc_status dn_param_count(const dn_ctx* ctx, size_t* n);
/* Host float32 arrays of dn_param_count elements.  dn_set_params resets the
 * Adam moments and step count. */
mc_status dn_set_params(dn_ctx* ctx, const float* params, size_t n);
mc_status dn_get_params(dn_ctx* ctx, float* params, size_t n);
/* Gradient of the loss of the last dn_train_step, before its update. */
mc_status dn_get_grads(dn_ctx* ctx, float* grads, size_t n);

/* Inference: input is device float32 [batch][in_channels][height][width]
 * (plane 0 the noisy image, planes 1.. auxiliary maps), output device float32
 * [batch][height][width].  The network sees plane 0 * in_scale and the other
 * planes as given, each rounded to bfloat16; the output is the network's
 * bfloat16 output * out_scale. */
mc_status dn_forward(dn_ctx* ctx, const float* input, float in_scale, float* output, float out_scale,
                     void* stream);

/* One optimisation step on a batch: input as for dn_forward, target device
 * float32 [batch][height][width]; forward, MSE loss against target * in_scale, backward, Adam with learning rate lr.  loss (host, may be
 * NULL) receives the batch loss; it synchronizes the stream when given. */
mc_status dn_train_step(dn_ctx* ctx, const float* input, const float* target, float in_scale, float lr,
                        double* loss, void* stream);

/* Reads the network output of the last forward pass (bf16 values as float32,
 * unscaled) into a device float32 [batch][height][width] array. */
mc_status dn_get_output(dn_ctx* ctx, float* out, void* stream);

/* ---- primitives (device NHWC bfloat16 tensors, for testing and reuse) ----
 * Convolution, k = 1 or 3, input = concatenation of x0 (c0 channels) and x1
 * (c1 channels, x1 = NULL for none), weight float32 [co][k][k][c0+c1] (device),
 * bias float32 [co] (device) or NULL:
 *   y[n,i,j,o] = act(bias[o] + sum w[o,dy,dx,c] x[n, i+dy-k/2, j+dx-k/2, c]),
 * act = ReLU if relu else identity; y has y_stride channels per pixel
 * (only the first co are written). */
mc_status dn_conv2d_forward(const uint16_t* x0, int c0, const uint16_t* x1, int c1, int batch, int height,
                            int width, const float* weight, const float* bias, int k, int co, int relu, uint16_t* y,
                            int y_stride, void* stream);

/* Input gradient: dx_s = dL/dx_s for both parts of the input, given
 * dz = dL/d(pre-activation output) with dz_stride channels per pixel (co
 * used); where mask_s is not NULL the result is zeroed where mask_s <= 0 (the
 * ReLU of the layer that produced x_s). */
mc_status dn_conv2d_backward_data(const uint16_t* dz, int dz_stride, int co, int batch, int height, int width,
                                  const float* weight, int k, uint16_t* dx0, int c0, const uint16_t* mask0,
                                  uint16_t* dx1, int c1, const uint16_t* mask1, void* stream);

/* Weight and bias gradients, ADDED to dw [co][k][k][c0+c1] and db [co]
 * (float32 device; db may be NULL). */
mc_status dn_conv2d_backward_weights(const uint16_t* dz, int dz_stride, int co, const uint16_t* x0, int c0,
                                     const uint16_t* x1, int c1, int batch, int height, int width, int k, float* dw,
                                     float* db, void* stream);

/* 2x2 max pooling of x [batch][height][width][c] (height, width even) and
 * its backward: dx = the gradient dy [batch][height/2][width/2][c] routed to
 * the first maximum of each window in the order (0,0), (0,1), (1,0), (1,1),
 * plus `add` [batch][height][width][c] if not NULL. */
mc_status dn_maxpool2(const uint16_t* x, uint16_t* y, int batch, int height, int width, int c, void* stream);
mc_status dn_maxpool2_backward(const uint16_t* x, const uint16_t* dy, const uint16_t* add, uint16_t* dx, int batch,
                               int height, int width, int c, void* stream);
/* Nearest 2x upsampling of x [batch][height][width][c] into
 * y [batch][2 height][2 width][c], and its backward: dx [batch][height][width][c]
 * = the sum of the four children of dy. */
mc_status dn_upsample2(const uint16_t* x, uint16_t* y, int batch, int height, int width, int c, void* stream);
mc_status dn_upsample2_backward(const uint16_t* dy, uint16_t* dx, int batch, int height, int width, int c,
                                void* stream);

#ifdef __cplusplus
}
#endif

#endif /* ARCHER_DENOISE_H */
