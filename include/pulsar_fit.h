/*
 * pulsar_fit.h: the optimisation loop around the renderer (Sec. 3.4,
 * "End-to-end Optimization", and the scene fit of Sec. 5): an image loss
 * against target views and its gradient dL/dF, and Adam (Kingma & Ba, the
 * optimiser the paper uses in every experiment) over the sphere parameters.
 *
 * One step of a fit over V views of one sphere set is:
 *   pulsar_render_batched         V scenes sharing the sphere arrays
 *   pulsar_image_loss             L = scale * sum over views and pixels, G = dL/dF
 *   pulsar_render_bwd_batched     PULSAR_FLAG_ACCUMULATE, every view adding into
 *                                 one set of gradient buffers
 *   pulsar_adam_step              updates the parameters and zeroes the gradients
 * All calls are asynchronous on the given stream and allocate nothing, so the
 * step can be captured in a CUDA graph and replayed.
 */
#ifndef PULSAR_FIT_H
#define PULSAR_FIT_H

#include "pulsar.h"

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PULSAR_LOSS_L2 = 0,   /* sum (F - T)^2, dL/dF = 2 (F - T) (the fit of Sec. 5 with an L2 loss) */
  PULSAR_LOSS_L1 = 1    /* sum |F - T|, dL/dF = sign(F - T), 0 where F = T (Sec. 3.4) */
};

/* Device floats pulsar_image_loss needs as scratch (per-CTA partial sums). */
#define PULSAR_LOSS_SCRATCH_FLOATS 1024

/* Image loss of n values (any layout: the images of all views, flattened),
 * multiplied by `scale` (1 for a sum, 1/n for a mean):
 *   image     device, n floats F
 *   target    device, n floats T
 *   grad      device, n floats, receives scale * dL/dF; may be NULL
 *   loss      device, one float, receives the loss; may be NULL
 *   scratch   device, PULSAR_LOSS_SCRATCH_FLOATS floats
 * The sum is taken in a fixed order (per-CTA partials, then one CTA), so the
 * loss is the same on every run.  PULSAR_ERR_INVALID_ARG for an unknown kind,
 * n < 0, or a NULL image, target or scratch when n > 0. */
pulsar_status pulsar_image_loss(int kind, const float* image, const float* target, int64_t n,
                                float scale, float* grad, float* loss, float* scratch,
                                void* stream);

/* One parameter tensor of an Adam step.  Device pointers, n floats each. */
typedef struct {
  float* param;        /* theta, updated in place */
  float* grad;         /* g; set to 0 after use when zero_grad is set */
  float* m;            /* first-moment estimate, 0 before the first step */
  float* v;            /* second-moment estimate, 0 before the first step */
  int64_t n;
  float lo, hi;        /* theta is clamped to [lo, hi] after the update (box-projected
                          Adam; -inf / +inf for none) */
} pulsar_adam_tensor;

typedef struct {
  float lr;            /* step size alpha */
  float beta1, beta2;  /* moment decay rates, in [0, 1) */
  float eps;           /* added to sqrt(v_hat) */
  int32_t zero_grad;   /* nonzero: write 0 into each gradient after reading it, ready for
                          the next backward with PULSAR_FLAG_ACCUMULATE */
} pulsar_adam_hyper;

/* Step counter of an Adam optimiser: device memory, 16 bytes, all zero before
 * the first step.  pulsar_adam_step advances t on the device, so a captured
 * step replays with the right bias correction. */
typedef struct {
  int32_t t;              /* steps taken */
  float step_size;        /* lr / (1 - beta1^t) for the current step */
  float inv_sqrt_bc2;     /* 1 / sqrt(1 - beta2^t) for the current step */
  int32_t reserved;
} pulsar_adam_state;

#define PULSAR_ADAM_MAX_TENSORS 8

/* One Adam step (Kingma & Ba, Algorithm 1) over up to PULSAR_ADAM_MAX_TENSORS
 * tensors: t += 1; m = beta1 m + (1 - beta1) g; v = beta2 v + (1 - beta2) g^2;
 * theta -= lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps);
 * theta = min(max(theta, lo), hi).
 *   tensors   host array of n_tensors descriptors, read during the call
 *   state     device, the optimiser's step counter
 * PULSAR_ERR_INVALID_ARG for n_tensors outside [1, PULSAR_ADAM_MAX_TENSORS], a
 * NULL pointer, n < 0, lo > hi, lr < 0, beta1 or beta2 outside [0, 1), or
 * eps < 0. */
pulsar_status pulsar_adam_step(int n_tensors, const pulsar_adam_tensor* tensors,
                               const pulsar_adam_hyper* hyper, pulsar_adam_state* state,
                               void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PULSAR_FIT_H */
