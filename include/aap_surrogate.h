/*
 * aap_surrogate.h -- C ABI of the learned coarse-grained surrogate.
 *
 * The particle library (aap.h) coarse-grains a state into fields on an
 * nbx x nby grid: density rho, polarisation density (sum cos theta,
 * sum sin theta) per unit area (aap_coarse_grain).  The surrogate advances
 * such fields 10 particle steps per application,
 *     F(t + 10) = F(t) + Net(F(t), eta),
 * with Net four 3x3 convolutions with circular padding (4 -> 32 -> 32 -> 32
 * -> 3 channels, the 4th input channel the noise strength eta), ReLU between
 * layers.  Weights and activations are BF16, every contraction accumulates
 * in FP32; the master weights and the Adam moments are FP32.  The network is
 * trained on fields that the particle simulation produces, by the library's
 * own forward and backward kernels.  The paper has no learned component; the
 * particle method stays the reference for the surrogate's error in p and in
 * the density structure factor.
 *
 * Conventions as in aap.h: int status (AAP_OK or a negative AAP_E* code),
 * message from aap_sur_last_error(); device pointers are caller-owned (e.g.
 * torch tensors' data_ptr()); all work runs on the stream given at creation;
 * only calls that return host data synchronise.  Field buffers hold
 * batch x 3 x nby x nbx FP32 values (plane-major, x fastest), the layout of
 * aap_coarse_grain.
 */
#ifndef AAP_SURROGATE_H
#define AAP_SURROGATE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct aap_sur_params {
    int32_t  nbx, nby;      /* field grid: multiples of 16, <= 4096                 */
    int32_t  max_batch;     /* largest batch of a train or predict call (1..4096)  */
    int32_t  conserve;      /* bit 0: one application keeps each sample's mean
                               density (the particle number), bit 1: its mean
                               polarisation; the network's residual is projected
                               to zero grid mean in those channels (training
                               included).  0 = free (default)                   */
    double   rho0;          /* mean density: fields are scaled by 1/rho0           */
    double   eta_center;    /* the eta channel is (eta - eta_center) / eta_scale   */
    double   eta_scale;
    double   lr, beta1, beta2, eps;   /* Adam                                   */
    uint64_t seed;          /* initial weights                                   */
} aap_sur_params;

typedef struct aap_sur aap_sur;

const char *aap_sur_last_error(void);

/* Defaults: 128 x 128 fields, batch 32, rho0 = 2, eta channel centred at 0.4
 * with scale 0.1, Adam lr 1e-3, betas (0.9, 0.999), eps 1e-8, seed 1. */
void aap_sur_params_default(aap_sur_params *p);

/* Create a network with He-uniform initial weights (the last layer scaled by
 * 0.1 so that the map starts near the identity) and allocate its buffers for
 * max_batch samples.  Errors: AAP_EINVAL, AAP_ENOMEM, AAP_ECUDA. */
int aap_sur_create(const aap_sur_params *p, void *stream, aap_sur **out);

int aap_sur_destroy(aap_sur *s);

/* Number of FP32 parameters (weights [co][tap][ci] and biases of the four
 * layers, channel-padded: 16 -> 32, 32 -> 32, 32 -> 32, 32 -> 8). */
int aap_sur_param_count(aap_sur *s, int64_t *count);

/* Copy the FP32 master parameters to / from host memory (set_params also
 * resets the Adam state).  count must equal aap_sur_param_count.  Sync. */
int aap_sur_get_params(aap_sur *s, float *host, int64_t count);
int aap_sur_set_params(aap_sur *s, const float *host, int64_t count);

/* FP32 gradient of the loss of the last train step (same layout).  Sync. */
int aap_sur_get_grads(aap_sur *s, float *host, int64_t count);

/* Apply the network `applications` times (10 particle steps each) to `batch`
 * field samples dev_in with per-sample noise strengths dev_eta (device,
 * batch floats); the result goes to dev_out (may alias dev_in).  The call's
 * kernels are captured once as a CUDA graph on a private stream and replayed
 * on the handle's stream while dev_in, dev_eta, dev_out, batch and
 * applications stay the same (the weights are read when it runs, so training
 * in between is seen). */
int aap_sur_predict(aap_sur *s, const float *dev_in, const float *dev_eta, int32_t batch, int32_t applications,
                    float *dev_out);

/* One Adam step on the mean squared error between one application to dev_in
 * and dev_target (normalised fields, the 3 channels averaged).  loss_out
 * (host, may be NULL) receives the loss before the step; then the call
 * synchronises. */
int aap_sur_train_step(aap_sur *s, const float *dev_in, const float *dev_target, const float *dev_eta,
                       int32_t batch, double *loss_out);

/* ---- the convolution kernels alone (tests, tools) -------------------------
 * BF16 tensors are passed as raw 16-bit words, NHWC (channels fastest).
 * Circular padding; batch >= 1; h and w multiples of 16 (a tensor-core tile
 * is 16 rows x 8 columns). */

/* y[b,y,x,co] = bias[co] + sum_{tap,ci} wt[tap][co][ci] x[b,(y+dy-1)%h,(x+dx-1)%w,ci]
 * (tap = 3 dy + dx), ReLU if relu != 0.  (cin, cout) in
 * {(16,32), (32,32), (32,8), (16,8)}. */
int aap_conv3x3_forward(const uint16_t *x, int32_t batch, int32_t h, int32_t w, int32_t cin, int32_t cout,
                        const uint16_t *wt, const float *bias, int32_t relu, uint16_t *y, void *stream);

/* Data gradient: dx[b,q,ci] = sum_{tap',co} wt_t[tap'][ci][co] dy[b,q+tap'-1,co]
 * where wt_t[tap'][ci][co] = w[co][8-tap'][ci] (flipped, transposed), set to 0
 * where mask[b,q,ci] <= 0 (the ReLU of the layer input).  (cout, cin) in
 * {(32,32), (16,32)}: cout is the channel count of dy. */
int aap_conv3x3_backward_data(const uint16_t *dy, int32_t batch, int32_t h, int32_t w, int32_t cin, int32_t cout,
                              const uint16_t *wt_t, const uint16_t *mask, uint16_t *dx, void *stream);

/* Weight and bias gradients: dw[co][tap][ci] = sum_{b,p} dy[b,p,co] x[b,p+tap-1,ci],
 * db[co] = sum_{b,p} dy[b,p,co] (FP32), dy holding dy_stride channels per
 * pixel of which the first cout are used.  part: device scratch of
 * part_floats >= (h / r) * batch * (cout*9*cin + cout) floats, r = 4 if h % 4
 * == 0 else 2 or 1.  Deterministic (fixed reduction order).  (cin, cout) in
 * {(32,32), (16,32), (32,8)}. */
int aap_conv3x3_backward_weight(const uint16_t *x, const uint16_t *dy, int32_t dy_stride, int32_t batch, int32_t h,
                                int32_t w, int32_t cin, int32_t cout, float *part, int64_t part_floats, float *dw,
                                float *db, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* AAP_SURROGATE_H */
