/*
 * gk_tail.h - C ABI of the learned Green-Kubo tail extrapolator.
 *
 * A small fully connected network predicts the converged viscosity and
 * thermal conductivity of a run from the first readout points of its
 * on-the-fly stress and heat-flux autocorrelations (arXiv 2503.07526
 * Sec. 2.2 Eq. (cor) and Appendix D Algorithm 2 for the readout, Sec. 2.3
 * Eqs. (visc), (therm) for the Green-Kubo targets).  The paper has no learned
 * component: the network, its features and its training are this library's
 * own extension, defined below.
 *
 * Network: x (n_in) -> [z = h W^T + b, h = tanh(z)] x depth -> y = h W^T + b
 * (n_out).  Weights live in FP32 (the master copy that Adam updates); every
 * product runs on the tensor cores with bfloat16 operands and FP32
 * accumulation.  Rounding to bfloat16 happens at exactly these points: the
 * standardised inputs, the weight copies, every stored activation (which
 * also feeds tanh' = 1 - h^2), the output gradient dY and every
 * pre-activation gradient dZ.  Loss: mean over rows and outputs of the
 * squared error of the standardised targets.  Training: Adam with bias
 * correction and decoupled weight decay on the weight matrices.
 *
 * Conventions are those of otf_md.h: int status (MD_OK or MD_E*), message in
 * md_last_error(), host (MD_MEM_HOST) or device (MD_MEM_DEVICE) arrays
 * selected by a mem flag, inputs copied, handles owned by the library, all
 * GPU work on the stream given at creation; calls that return host results
 * synchronise it.  Matrices are row-major.
 */
#ifndef GK_TAIL_H
#define GK_TAIL_H

#include <stdint.h>

#include "otf_md.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlp_params {
  int32_t n_in;        /* input features, 1..240 */
  int32_t width;       /* hidden width: 128 */
  int32_t depth;       /* hidden layers, 1..6 */
  int32_t n_out;       /* outputs, 1..16 */
  int32_t batch;       /* training rows per step: a multiple of 128, at most 4096 */
  float lr, beta1, beta2, eps, weight_decay; /* Adam */
  uint64_t seed;       /* Glorot-uniform weights (SplitMix64), zero biases */
} mlp_params;

typedef struct mlp_handle_s mlp_handle;

/* Creates a network on the current device.  Returns MD_EINVAL for sizes out
 * of range. */
OTF_API int mlp_create(const mlp_params *p, void *cuda_stream, mlp_handle **out);

/* Number of FP32 parameters in the flat order used by mlp_get_params /
 * mlp_set_params: for each layer in order, W [out][in] then b [out]. */
OTF_API int mlp_param_count(const mlp_handle *h, int64_t *count);
OTF_API int mlp_get_params(mlp_handle *h, float *flat, int64_t count, int32_t mem);
/* Sets the master weights and restarts Adam (moments zero, step count 0). */
OTF_API int mlp_set_params(mlp_handle *h, const float *flat, int64_t count, int32_t mem);

/* Feature and target standardisation, host arrays: the network sees
 * (x - x_mean) / x_std and is trained on (t - y_mean) / y_std; mlp_forward
 * returns y * y_std + y_mean.  Identity (0, 1) after mlp_create. */
OTF_API int mlp_set_scaler(mlp_handle *h, const float *x_mean, const float *x_std, const float *y_mean,
                           const float *y_std);
/* Sets the scaler to the mean and standard deviation (population, FP64) of
 * the rows of X [rows][n_in] and T [rows][n_out] (host arrays); a zero
 * standard deviation becomes 1. */
OTF_API int mlp_fit_scaler(mlp_handle *h, const float *X, const float *T, int64_t rows);

/* Y [rows][n_out] = network(X [rows][n_in]); any rows >= 1. */
OTF_API int mlp_forward(mlp_handle *h, const float *X, int64_t rows, float *Y, int32_t mem);

/* One forward and backward pass on exactly `batch` rows: returns the loss and
 * keeps the gradients for mlp_adam_step; grad (nullable) receives them in the
 * flat parameter order. */
OTF_API int mlp_loss_grad(mlp_handle *h, const float *X, const float *T, int64_t rows, double *loss,
                          float *grad, int32_t mem);

/* One Adam step with the given gradients (flat order, count = parameter
 * count), or with those of the last mlp_loss_grad when grad is NULL. */
OTF_API int mlp_adam_step(mlp_handle *h, const float *grad, int32_t mem);

/* Mini-batch training for `epochs` passes over X [rows][n_in], T [rows][n_out]
 * (host or device).  Epoch e visits the rows in the order order[e][0..rows)
 * (int64, host; NULL: a SplitMix64 shuffle seeded by shuffle_seed) in
 * consecutive batches; the last incomplete batch is dropped.  The whole
 * pass runs on the device; loss_per_epoch (host, nullable, [epochs]) gets the
 * mean batch loss of each epoch. */
OTF_API int mlp_train(mlp_handle *h, const float *X, const float *T, int64_t rows, int32_t epochs,
                      const int64_t *order, uint64_t shuffle_seed, double *loss_per_epoch, int32_t mem);

/* Limit, in nanoseconds of wall time, of the pipeline waits of the layered
 * tensor-core kernel (a TMA panel landing, a stage's products done) used by
 * mlp_loss_grad, mlp_train and the layered forward pass (the paper has no
 * counterpart; default 2e9).  A wait that runs out stops its CTA cleanly
 * (the copies and products it issued are still waited for, up to 2 s) and
 * the call returns MD_ETIMEOUT with the handle still usable.  0 gives up at
 * once on any wait not already complete, which is how the timeout path is
 * tested.  MD_EINVAL for a null handle or ns < 0. */
OTF_API int mlp_set_wait_limit(mlp_handle *h, int64_t ns);

OTF_API void mlp_free(mlp_handle *h);

/* Features of nruns runs for the learned tail, host arrays: c_sigma and c_q
 * [nruns][ld] hold each run's shear-stress autocorrelation (mean of xy, xz,
 * yz) and heat-flux autocorrelation (mean of x, y, z) on the multiple-tau
 * readout grid (Algorithm 2), of which the first 64 points are used (ld >= 64).
 * Row r of out [nruns][132] is: c_sigma/c_sigma[0] at the 64 points,
 * log(V C_sigma(0) / T), c_q/c_q[0] at the 64 points, log(V C_q(0) / T^2),
 * T, density.  MD_EINVAL if a lag-0 value or V or T is not positive. */
OTF_API int gk_tail_features(const double *c_sigma, const double *c_q, int64_t ld, int64_t nruns,
                             const double *volume, const double *temperature, const double *density,
                             float *out);

/* Where the learned tail is used (a project extension; the paper has no
 * counterpart).  The network is trusted inside the temperature-density box
 * of its training runs, and only where a run is short enough that its own
 * Green-Kubo integral is expected to be less accurate than the network: the
 * own integral's rms relative error is modelled as short_coeff / sqrt(steps)
 * (it falls with the run length and, for the integral of one global flux,
 * not with the number of atoms), the network's as net_error, its rms
 * relative error on validation runs.  Index 0: viscosity, 1: conductivity. */
typedef struct {
  double T_min, T_max, rho_min, rho_max; /* the training runs' temperature and density box */
  double net_error[2];                   /* the network's rms relative error on validation runs */
  double short_coeff[2];                 /* own integral: rms relative error x sqrt(correlated steps) */
} gk_tail_rule;

/* The box of n runs' temperatures and densities (host arrays) into rule.
 * MD_EINVAL for a null argument or n < 1. */
OTF_API int gk_tail_box(const double *temperature, const double *density, int64_t n, gk_tail_rule *rule);

/* sqrt(mean_r (((a_r - b_r) / b_r)^2 w_r)) over n host values, w = NULL
 * meaning all weights 1: the network's validation error (w = NULL), or, with
 * a = the short runs' integrals, b = the long runs' and w = the short runs'
 * correlated steps, short_coeff.  MD_EINVAL for a null argument, n < 1 or a
 * zero b_r. */
OTF_API int gk_tail_rms_rel(const double *a, const double *b, const double *w, int64_t n, double *out);

/* Per run r and output k (host arrays; net, own, out, used [nruns][2]):
 * out = net where (T_r, rho_r) lies in the rule's box and
 * short_coeff[k] / sqrt(steps_r) > net_error[k], else own; used (nullable)
 * records the choice.  MD_EINVAL for a null argument or steps_r <= 0. */
OTF_API int gk_tail_choose(const gk_tail_rule *rule, const double *temperature, const double *density,
                           const double *steps, const double *net, const double *own, int64_t nruns, double *out,
                           int32_t *used);

/* Reads `rows` rows of a correlator at once: row i is the mean of groups
 * g0 + i*avg .. g0 + i*avg + avg - 1 on the Algorithm 2 readout grid.
 * times [npts] and values [rows][cap] (host); *n = points per row.
 * MD_ECAP if cap < *n. */
OTF_API int corr_read_rows(corr_handle *c, int64_t g0, int64_t rows, int64_t avg, double *times,
                           double *values, int64_t cap, int64_t *n);

#ifdef __cplusplus
}
#endif

#endif /* GK_TAIL_H */
