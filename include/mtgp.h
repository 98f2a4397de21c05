/*
 * mtgp.h -- C ABI of the GB300 fast multitask Gaussian process library.
 *
 * The library evaluates, on one GPU, the exact MLE loss of a multitask GP whose Gram
 * matrix has the fast-MTGP structure of Sorokin, Robbe, Liu, Mak, Hickernell,
 * "Fast multitask Gaussian processes" (arXiv 2603.16014):
 *
 *   K((t,x),(t',x')) = R(t,t') Q(x,x')                                   (Eq. 3.1)
 *   R = W W^T + diag(v)                        (Sec. 3.1, the paper's B B^T + diag(zeta))
 *   Q(x,x') = prod_j (1 + eta_j K(x_j, x'_j))                            (Eq. 2.4, gamma = 1)
 *   K~ = K + sigma2 I                         (Sec. 3.1, one noise variance for all tasks)
 *   designs: shifted rank-1 lattices with the SI Bernoulli kernel of order 2 (Eq. 2.5)
 *            or digitally shifted base-2 digital nets with the DSI order-2 kernel (Eq. 2.6),
 *            common generator, per-task shifts, n_t = 2^{m_t}          (Condition 3.1)
 *
 * Conventions shared by every call
 *   - Return value: MTGP_OK or an MTGP_ERR_* code.  Argument errors are detected on the
 *     host and returned immediately; numerical errors found by a kernel (a non-positive
 *     pivot, a non-finite value) are recorded in a device status word that mtgp_sync()
 *     returns.  mtgp_last_error_string() describes the last host-side error of the calling
 *     thread.
 *   - Every array argument is a DEVICE pointer owned by the caller unless stated otherwise;
 *     the library never frees caller memory.  Host arrays are marked "host".
 *   - Calls are asynchronous on the given stream.  A handle must not be used from two
 *     streams at once (it owns one workspace).
 *   - Task order: arrays indexed by task use the caller's task order.  Internally tasks
 *     are reordered so that n_1 >= ... >= n_T (Condition 3.1: "may always be satisfied by
 *     reindexing"), ties keeping the caller's order.
 *   - Points are 32-bit fixed point: coordinate value = word / 2^32.
 */
#ifndef MTGP_H
#define MTGP_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mtgp_s mtgp_t;

enum {
    MTGP_OK = 0,
    MTGP_ERR_INVALID_ARG = 1,  /* bad size, null pointer, out-of-range flag               */
    MTGP_ERR_NOT_PD = 2,       /* a pivot / Schur complement <= 0 (Lambda not HPD numerically) */
    MTGP_ERR_NUMERIC = 3,      /* NaN or Inf in an input or an intermediate                */
    MTGP_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up                       */
    MTGP_ERR_UNSUPPORTED = 5,  /* valid request outside what the library implements        */
    MTGP_ERR_CUDA = 6,         /* a CUDA runtime call failed                               */
    MTGP_ERR_STATE = 7         /* call order violated (e.g. NLL before mtgp_set_y)         */
};

enum { MTGP_LATTICE = 0, MTGP_DNET = 1 };
enum { MTGP_FP64 = 0, MTGP_FP32_TRANSFORM = 1 };
/* OR-ed into mtgp_create's precision: one noise variance per task (xi_t of Sec. 3.1's data model)
 * instead of a shared sigma2; sigma2 and g_sigma2 then hold T values in caller task order. */
enum { MTGP_NOISE_PER_TASK = 16 };
/* OR-ed into mtgp_create's precision with MTGP_FP32_TRANSFORM: keep the per-frequency solve of the
 * equal-size digital-net kernels in FP64.  By default those kernels solve FP32-transform problems in
 * double-float arithmetic (pairs of FP32 values, about 48 significant bits, on the FP32 pipe; a
 * frequency whose pivots leave the double-float range is solved in FP64); every other solve is FP64. */
enum { MTGP_SOLVE_FP64 = 32 };

/* Limits of the library. */
#define MTGP_MAX_TASKS 8
#define MTGP_MAX_M 24      /* n_t <= 2^24 */
#define MTGP_MAX_DIM 32

/*
 * mtgp_create -- build a handle for one fit (Condition 3.1).
 *   kind      MTGP_LATTICE (Def. 2.1, SI kernel Eq. 2.5 with alpha = 2) or
 *             MTGP_DNET (Def. 2.2, DSI kernel Eq. 2.6 with b = (0, 1, 0, 0)).
 *   d         dimension, 1..MTGP_MAX_DIM.
 *   T         number of tasks, 1..MTGP_MAX_TASKS.
 *   m         host, T ints: n_t = 2^{m[t]}, 0 <= m[t] <= MTGP_MAX_M, any order.
 *   gen       host.  LATTICE: d generating-vector words g_j (z_i = v(i) g mod 1 computed as
 *             bitrev32(i) * g_j mod 2^32).  DNET: d x gen_cols words, row-major by coordinate:
 *             gen[j * gen_cols + p] is column g_p of coordinate j (bit 31 = digit 2^-1).
 *   gen_cols  DNET: number of generating-matrix columns, >= max m[t], <= 32. Ignored for LATTICE.
 *   shift     host, T x d words (caller task order): lattice shift Delta_t (added mod 2^32) or
 *             digital shift (XOR).
 *   precision MTGP_FP64 (FP64 throughout except the eta-gradient contractions of d <= 16, which run in
 *             double-float: they feed only d(NLL)/d(eta)), or MTGP_FP32_TRANSFORM (kernel columns and
 *             their transforms in FP32; y transforms and log-determinant sums in FP64 or double-float;
 *             per-frequency solves of equal-size digital nets in double-float unless MTGP_SOLVE_FP64 is
 *             OR-ed in, every other solve FP64; the posterior of equal-size digital nets in
 *             double-float), optionally OR MTGP_NOISE_PER_TASK (per-task noise variances; such handles
 *             use the general kernels, not the fused equal-size ones, and are refused by the batch and
 *             no-allocation calls).
 * Allocates the handle's device workspace on the current device.
 */
int mtgp_create(mtgp_t** out, int kind, int d, int T, const int* m, const uint32_t* gen,
                int gen_cols, const uint32_t* shift, int precision);

/* mtgp_destroy -- free the handle and its workspace (synchronises the device first). */
int mtgp_destroy(mtgp_t* h);

/*
 * mtgp_points -- write the design points x_{t,i} (Def. 2.1 / Def. 2.2, radical-inverse order)
 * as fixed-point words: x[(N_{t-1} + i) * d + j], tasks in caller order, N_{t-1} = n_1+..+n_{t-1}.
 */
int mtgp_points(mtgp_t* h, uint32_t* x, cudaStream_t stream);

/*
 * mtgp_set_y -- observations y (N doubles, tasks in caller order, each task in radical-inverse
 * order).  Computes yhat_t = V_{m_t}^dagger y_t (Theorem "fast MTGP computations") once; the
 * data are theta-independent.  Must precede every NLL / gradient / posterior call.
 */
int mtgp_set_y(mtgp_t* h, const double* y, cudaStream_t stream);

/*
 * mtgp_nll -- MLE loss at theta (Eq. 3.3) with tau profiled at its optimum (Eq. 3.4,
 * Theorem "fast MTGP computations" item 4).
 *   eta     d doubles (eta_j >= 0), W T x s doubles row-major (caller task order), 1 <= s <= T,
 *   v       T doubles > 0, sigma2 one double > 0 (T doubles, caller order, for a handle created
 *           with MTGP_NOISE_PER_TASK) -- all device pointers.
 *   out     3 doubles: [0] NLL = (L + N log 2 pi) / 2, [1] quad = r^T K~^-1 r, [2] log|K~|.
 *   tau     T doubles (caller order) or NULL: the optimal means.
 */
int mtgp_nll(mtgp_t* h, const double* eta, const double* W, int s, const double* v,
             const double* sigma2, double* out, double* tau, cudaStream_t stream);

/*
 * mtgp_nll_grad -- as mtgp_nll plus the gradient of the NLL (= half the gradient of L) with
 * respect to eta (d), W (T x s), v (T) and sigma2 (1, or T with MTGP_NOISE_PER_TASK), at the
 * optimal tau (tau minimises L, so
 * its own dependence on theta does not enter).  Gradient outputs may not be NULL.
 */
int mtgp_nll_grad(mtgp_t* h, const double* eta, const double* W, int s, const double* v,
                  const double* sigma2, double* out, double* tau, double* g_eta, double* g_W,
                  double* g_v, double* g_sigma2, cudaStream_t stream);

/*
 * mtgp_nll_grad_host -- mtgp_nll_grad with HOST buffers: the call copies theta in, evaluates and
 * copies the results out, all in stream order on `stream` (asynchronous for page-locked host
 * memory; the caller keeps both buffers alive and calls mtgp_sync before reading `out`).
 *   theta  host, packed eta (d) | W (T x s, caller task order, row-major) | v (T) | sigma2 (1, or T
 *          with MTGP_NOISE_PER_TASK): d + T s + T + (1 or T) doubles.
 *   out    host, packed [NLL, quad, logdet] (3) | tau (T) | g_eta (d) | g_W (T x s) | g_v (T) |
 *          g_sigma2 (1 or T): 3 + T + (size of theta) doubles.
 * The device staging buffer belongs to the handle: calls on one handle are ordered by their
 * stream (two streams on one handle race).  Page-locked buffers are reached by the kernels
 * themselves (theta read by a one-block staging kernel, the results written by the kernels that
 * produce them, no DMA copies); with profiling off, the first call for a given (theta, out, s) and
 * kernel configuration captures the launches into a CUDA graph owned by the handle and later calls
 * replay it (one launch).  Pageable buffers go through cudaMemcpyAsync, without a graph.  Errors
 * as mtgp_nll_grad.
 */
int mtgp_nll_grad_host(mtgp_t* h, const double* theta, int s, double* out, cudaStream_t stream);

/*
 * mtgp_posterior -- posterior mean and variance of f(t, x) (Eq. 3.2) at nq queries, with the
 * prior mean tau at its MLE optimum.
 *   xq     nq x d doubles in [0, 1] (row-major); each is mapped to the fixed-point word
 *          floor(x 2^32), 1.0 mapping to the largest word below 1 (Sec. 2.2.1 boundary rule).
 *   task   nq ints, caller task index of each query.
 *   mean   nq doubles (required); var nq doubles or NULL (NULL skips the variance).
 * Variance: equal sizes through per-frequency T x T factors; unequal nested sizes through the tree
 * solver's factor, class by class (queries in batches of the rows that fit in 64 M doubles).
 * FP32-transform digital nets with equal sizes, the order-2 DSI kernel, d <= 16 and n = 2^10 .. 2^18
 * evaluate both in double-float arithmetic from exact kernel values (the mean of a variance call comes
 * from the same kernel rows); the first call on a handle allocates its posterior scratch.
 */
int mtgp_posterior(mtgp_t* h, const double* eta, const double* W, int s, const double* v,
                   const double* sigma2, int nq, const double* xq, const int* task,
                   double* mean, double* var, cudaStream_t stream);

/* mtgp_sync -- wait for the stream, return the first error recorded on the device since the
 * last mtgp_sync (MTGP_OK if none) and clear it. */
int mtgp_sync(mtgp_t* h, cudaStream_t stream);

/* mtgp_last_error_string -- description of the calling thread's last host-side error. */
const char* mtgp_last_error_string(void);

/*
 * mtgp_profile -- enable (1) or disable (0) kernel timing on the handle.  When enabled, every kernel
 * the handle launches is bracketed by CUDA events on the call's stream (adds two event records per
 * launch; off by default).
 * mtgp_profile_read -- synchronise on the recorded events, aggregate by kernel name and clear the log.
 *   names     host, max_entries x 32 chars (NUL-terminated kernel names)
 *   total_ms  host, max_entries doubles: summed duration per name;  counts: launches per name
 *   n_out     number of distinct names (may exceed max_entries; only the first max_entries are written)
 */
int mtgp_profile(mtgp_t* h, int enable);
int mtgp_profile_read(mtgp_t* h, int max_entries, char* names, double* total_ms, int* counts, int* n_out);

/*
 * mtgp_nll_equal_static -- the NLL of mtgp_nll for one fit with equal task sizes, computed without
 * allocating any device memory.  The paper has no counterpart: this is a deployment variant for
 * callers that cannot call cudaMalloc (code where allocation is forbidden or unsafe: inside regions
 * that must not synchronise the device, allocator callbacks, plugin hosts that own the device heap,
 * processes that pre-reserved all free memory).  Every intermediate lives in one file-scope device
 * array of MTGP_STATIC_SCRATCH_BYTES (8 MiB), which each GPU that loads the library holds until
 * the process exits.
 *   kind, d, T, gen, gen_cols, shift, precision   as mtgp_create, with every task of size 2^m
 *                                                 (4 <= m); host arrays.
 *   y       device, T * 2^m observations (tasks in order, each in radical-inverse order).
 *   eta, W, s, v, sigma2, out, tau                as mtgp_nll (device pointers; tau may be NULL).
 *   status  device int or NULL: set to 0 by the call, then to the kernel status bits
 *           (1 = non-positive pivot, 2 = non-finite value) if any.
 * Returns MTGP_ERR_INVALID_ARG, with a message in mtgp_last_error_string, for arguments out of
 * range and for problems whose intermediates exceed the scratch array (checked before any device
 * work); nothing is allocated on any path.
 * The first call on each device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  All calls share the one
 * array and the call clears what must start at zero: calls whose work overlaps on the GPU (two
 * streams, two host threads) race and must be serialised by the caller.
 */
int mtgp_nll_equal_static(int kind, int d, int T, int m, const uint32_t* gen, int gen_cols,
                          const uint32_t* shift, int precision, const double* y, const double* eta,
                          const double* W, int s, const double* v, const double* sigma2, double* out,
                          double* tau, int* status, cudaStream_t stream);

/*
 * mtgp_set_smoothness -- the kernel's smoothness alpha, 1, 2 (default), 3 or 4.  Lattice handles:
 * the SI kernel of Eq. 2.5, (-1)^(alpha+1) (2 pi)^(2 alpha) / (2 alpha)! B_(2 alpha)((x - x') mod 1)
 * as the univariate factor of Eq. 2.4.  Digital-net handles: the single order K_alpha of the DSI
 * kernel of Eq. 2.6 (mixture weights b = e_alpha; alpha = 2 clears any weights set by
 * mtgp_set_dsi_weights).  Takes effect for the following calls on the handle; synchronous (waits
 * for the device), host only.
 */
int mtgp_set_smoothness(mtgp_t* h, int alpha);

/*
 * mtgp_set_dsi_weights -- the adaptive-smoothness DSI kernel of Eq. 2.6 for a digital-net handle:
 * univariate factor K(x, x') = sum_{a=1}^{4} b_a K_a(x XOR x') in Eq. 2.4, with
 *   K_1 = 1/6 - t_1/2 (the order-one Walsh kernel; the printed order-1 form is read with mean zero),
 *   K_2 = -1 - beta x + 5/2 (1 - t_1),  K_3, K_4 as printed in Eq. 2.6,
 * beta(x) = -floor(log2 x), t_nu = 2^(-nu beta), beta(0) = t_nu(0) = 0.
 *   b   device, 4 doubles >= 0 (checked by the following evaluations: non-finite or negative
 *       weights raise MTGP_ERR_NUMERIC at mtgp_sync), copied into the handle in stream order on
 *       `stream`; NULL returns the handle to the order-2 kernel alone (b = e_2, the default).
 * With weights set, every evaluation (mtgp_nll, mtgp_nll_grad, mtgp_posterior, mtgp_gcv,
 * mtgp_gcv_grad, mtgp_cubature) uses the mixture, through the general kernels (the fused
 * equal-size kernels evaluate the order-2 kernel only), and the gradient calls also form dL/db
 * (read it with mtgp_dsi_weights_grad).  Lattice handles: MTGP_ERR_UNSUPPORTED.
 */
int mtgp_set_dsi_weights(mtgp_t* h, const double* b, cudaStream_t stream);

/*
 * mtgp_dsi_weights_grad -- copy the gradient with respect to the mixture weights b (4 doubles,
 * device g_b) left by the last mtgp_nll_grad (gradient of the NLL, as g_eta) or mtgp_gcv_grad
 * (gradient of the GCV loss) on the handle, in stream order; zeros before the first gradient call
 * after mtgp_set_dsi_weights.  MTGP_ERR_INVALID_ARG when the handle has no weights set.
 */
int mtgp_dsi_weights_grad(mtgp_t* h, double* g_b, cudaStream_t stream);

/*
 * Multitask Bayesian cubature (Sec. 3.5, multitask cubature theorem) for the task integrals
 * mu_t = int f(t, x) dx under the fitted MTGP at the MLE mean.  The product kernels of Eq. 2.4 with
 * the SI or DSI factors integrate to gamma = 1 in each argument, so
 *   mu_hat = tau + R E K~^-1 (y - E^T tau)   (= tau_MLE up to rounding),
 *   Sigma  = R - R Pi R,  Pi = E K~^-1 E^T = n Lambda(0)^-1 (equal sizes) or from residue class 0.
 * mu (device, T) and Sigma (device, T x T row-major) in caller task order; a weighted combination
 * chi^T mu has mean chi^T mu_hat and variance chi^T Sigma chi.  Arguments and errors as mtgp_nll.
 */
int mtgp_cubature(mtgp_t* h, const double* eta, const double* W, int s, const double* v, const double* sigma2,
                  double* mu, double* Sigma, cudaStream_t stream);

/*
 * GCV loss (Sec. 2.2 and 3.2, Eq. 3.3, second form) at the GCV mean (Eq. 3.4, second form):
 *   tau solves (E K~^-2 E^T) tau = E K~^-2 y, r = y - E^T tau,
 *   L_GCV = r^T K~^-2 r / trace(K~^-1)^2 = ||Lambda~^-1 rhat||^2 / trace(Lambda~^-1)^2.
 * For equal sizes tau is the vector of sample means; for nested sizes E K~^-2 E^T = H H^* with H
 * from the residue class 0 of Lambda~^-1 (Theorem FMTGP item 4).  Arguments as mtgp_nll; out
 * (device, 3 doubles) receives [L_GCV, r^T K~^-2 r, trace(K~^-1)], tau (device, T, caller order,
 * nullable) the GCV mean.  No gradient.  Errors as mtgp_nll.
 */
int mtgp_gcv(mtgp_t* h, const double* eta, const double* W, int s, const double* v, const double* sigma2,
             double* out, double* tau, cudaStream_t stream);

/*
 * GCV loss and its gradient with respect to (eta, W, v, sigma2), equal task sizes (others:
 * MTGP_ERR_UNSUPPORTED).  tau_GCV minimises the numerator and the trace does not depend on tau, so
 * the gradient holds tau fixed.  With alpha = Lambda^-1 rhat, beta = Lambda^-1 alpha, A = ||alpha||^2
 * and B = trace Lambda^-1: dL = trace(G dLambda), G = -(alpha beta^H + beta alpha^H) / B^2 +
 * (2A / B^3) Lambda^-2, evaluated per frequency after the value pass.  Outputs as mtgp_gcv plus the
 * gradient arrays of mtgp_nll_grad (of L_GCV itself, not halved).
 */
int mtgp_gcv_grad(mtgp_t* h, const double* eta, const double* W, int s, const double* v, const double* sigma2,
                  double* out, double* tau, double* g_eta, double* g_W, double* g_v, double* g_sigma2,
                  cudaStream_t stream);

/*
 * Batched fits: many independent fits with equal task sizes (each fit: kind, d, T tasks of 2^m
 * points) evaluated and optimised together.  No counterpart in the paper beyond its optimisation
 * loop (Sec. 4.1 fits each model by a first-order optimiser on the MLE loss (3.3)); here every
 * optimiser step of all fits is one batched NLL + gradient evaluation plus one Adam update.
 *
 * Parameters of fit f are packed as [eta (d), W (T x s, row-major), v (T), sigma2 (1)], fits
 * concatenated (offsets from mtgp_batch_layout).  Adam acts on log eta, W, log v, log sigma2 with
 * beta1 = 0.9, beta2 = 0.999, eps = 1e-8; gradients returned by mtgp_batch_nll_grad are with respect
 * to the packed (natural) parameters.
 *
 * mtgp_batch_create -- host arrays of length nfits: kind, d, T, m, gen_cols, precision; gen and shift
 *   are the fits' generator / shift arrays (as mtgp_create) concatenated; s is W's column count for
 *   every fit (1 <= s <= T).  precision[f] is MTGP_FP64 or MTGP_FP32_TRANSFORM for fit f (as
 *   mtgp_create, without MTGP_NOISE_PER_TASK): FP32 transforms meet the 1e-5 relative NLL tolerance on
 *   digital nets, while the SI spectrum of a lattice decays below FP32 transform noise, so lattice fits
 *   should take MTGP_FP64.  Fits of both precisions run in one batch (separate kernel classes).
 *   MTGP_ERR_UNSUPPORTED if a fit's size is outside the fused kernels (m >= 4, per-CTA tiles <= 96 KB).
 * mtgp_batch_layout -- host arrays of nfits + 1 offsets into the packed parameters and observations.
 * mtgp_batch_set_y -- device, all fits' observations concatenated (each fit as mtgp_set_y).
 * mtgp_batch_set_theta / mtgp_batch_get_theta -- device packed parameters (natural scale); set
 *   also resets the Adam moments and step count.
 * mtgp_batch_nll_grad -- device outputs: nll (nfits, NLL of each fit), grad (packed), either NULL.
 * mtgp_batch_adam -- `steps` Adam steps at learning rate lr; trace (device, steps x nfits, or NULL)
 *   receives each step's NLL before its update.  use_graph = 1 captures the steps in one CUDA graph
 *   on the first call (stream must not be the legacy default stream) and replays it afterwards.
 * mtgp_batch_autotune -- times the candidate transform splits of each distinct (kind, T, m,
 *   dimension bucket) on one representative fit (reps timed runs each), keeps the fastest for all
 *   fits of that key and rebuilds the launch tables; chosen (host, nfits, or NULL) receives the
 *   splits.  Needs observations and parameters set; synchronises the device.
 * mtgp_batch_fit -- fit every model of the batch by `steps` Adam steps on its MLE loss (Sec. 4.1's
 *   optimisation loop, run for all fits at once): theta0 (device, packed natural parameters) starts
 *   the run and resets the Adam moments (as mtgp_batch_set_theta); NULL continues from the current
 *   parameters and optimiser state (e.g. those mtgp_propose set).  lr > 0 is the step size and
 *   use_graph, trace as mtgp_batch_adam.  theta_out (device, packed, or NULL) receives the final
 *   parameters and nll_out (device, nfits, or NULL) the NLL at them (one more batched evaluation).
 *   Needs mtgp_batch_set_y first; asynchronous on `stream` (a graph run needs a non-default stream).
 */
typedef struct mtgp_batch_s mtgp_batch_t;
int mtgp_batch_create(mtgp_batch_t** out, int nfits, const int* kind, const int* d, const int* T, const int* m,
                      const uint32_t* gen, const int* gen_cols, const uint32_t* shift, int s, const int* precision);
int mtgp_batch_destroy(mtgp_batch_t* b);
int mtgp_batch_layout(const mtgp_batch_t* b, long long* param_offsets, long long* y_offsets);
int mtgp_batch_set_y(mtgp_batch_t* b, const double* y, cudaStream_t stream);
int mtgp_batch_set_theta(mtgp_batch_t* b, const double* theta, cudaStream_t stream);
int mtgp_batch_get_theta(mtgp_batch_t* b, double* theta, cudaStream_t stream);
int mtgp_batch_nll_grad(mtgp_batch_t* b, double* nll, double* grad, cudaStream_t stream);
int mtgp_batch_adam(mtgp_batch_t* b, int steps, double lr, int use_graph, double* trace, cudaStream_t stream);
int mtgp_batch_autotune(mtgp_batch_t* b, int reps, int* chosen, cudaStream_t stream);
int mtgp_batch_fit(mtgp_batch_t* b, const double* theta0, int steps, double lr, int use_graph, double* theta_out,
                   double* nll_out, double* trace, cudaStream_t stream);

/*
 * Learned proposal of starting hyper-parameters.  The paper has no counterpart: it starts every fit's
 * optimiser (Sec. 4.1) from a fixed point.  A small MLP maps a fixed-size spectral summary of a fit
 * to its parameters; starting the optimiser there saves steps when the prediction is close.
 *
 * mtgp_batch_features -- feat (device, nfits x 258 FP32, row per fit): for each caller task t < 8 and
 *   bin k < 32, log(mean |yhat_t(f)|^2 + 1e-30) over the frequencies f = 1..n-1 with
 *   bin(f) = floor(4 q(f) / m), q(f) = 8 floor(log2 f) + (the three bits of f after its leading one,
 *   zero-filled), yhat_t = V^dagger y_t of Sec. 3.3 (computed by mtgp_batch_set_y, which must come
 *   first); an empty bin repeats the previous bin; tasks t >= T are 0; then m and d.
 * mtgp_batch_targets -- target, mask (device, nfits x 37 FP32): from the current parameters
 *   [log eta_j (j < 12), W (8 x 2, row-major), log v_t (t < 8), log sigma2], mask 1 where the entry
 *   exists (j < d, t < T).  W is canonicalised first: multiplied on the right by the orthogonal 2 x 2
 *   matrix that gives W[0][1] = 0, W[0][0] >= 0, W[1][1] >= 0 (R = W W^T + diag(v) is unchanged).
 *   A fit with a non-finite entry (e.g. an optimiser run that diverged) gets target 0 and mask 0.
 * mtgp_batch_set_theta_proposal -- pred (device, nfits x 37 FP32, layout as the targets) becomes the
 *   parameters: log entries are clamped to [-40, 20] and exponentiated, W is taken as is.  Resets the
 *   Adam moments and step count like mtgp_batch_set_theta.
 * All three need s = 2 and d <= 12 for every fit (else MTGP_ERR_UNSUPPORTED); the first call builds a
 * small per-fit table on the device (synchronous allocation).
 */
int mtgp_batch_features(mtgp_batch_t* b, float* feat, cudaStream_t stream);
int mtgp_batch_targets(mtgp_batch_t* b, float* target, float* mask, cudaStream_t stream);
int mtgp_batch_set_theta_proposal(mtgp_batch_t* b, const float* pred, cudaStream_t stream);

/*
 * Multilayer perceptron with BF16 weights and FP32 accumulation (the proposal network): L layers,
 * h_{l+1} = act(h_l W_l^T + b_l) with ReLU on hidden layers and the identity on the last; the input
 * is standardised x' = (x - mu) / sd per column first.  Masters are FP32; the GEMMs read BF16 copies
 * of the weights, of x' and of the hidden activations, and accumulate in FP32 on the tensor cores.
 *
 * mtgp_mlp_create -- widths (host, nlayers + 1 entries, each 1..4096), max_batch rows per call.
 *   Weights start at zero with mu = 0, sd = 1: set them with mtgp_mlp_set_params.
 * mtgp_mlp_set_params / mtgp_mlp_get_params -- params (host FP32): per layer W_l (out x in, row-major)
 *   then b_l (out); mu, sd (host, widths[0] each, NULL to keep mu = 0 / sd = 1 on set, or to skip on
 *   get).  set also clears the optimiser state.  Both synchronise the device.
 * mtgp_mlp_fit_scaling -- mu and sd from the columns of x (device, rows x widths[0]); sd is floored
 *   at 1e-3.
 * mtgp_mlp_forward -- y (device, B x widths[L]) from x (device, B x widths[0]); 1 <= B <= max_batch.
 * mtgp_mlp_gradients -- masked squared loss sum(mask (out - target)^2) / max(sum(mask), 1) over the
 *   batch and its gradient.  rows (device, B int, or NULL for 0..B-1) selects the rows of x, target
 *   and mask (each with widths[0] or widths[L] columns) that form the batch; every entry must index
 *   a row of those arrays (not checked).  loss (device, 1 float)
 *   and grads (device, packed like params) may be NULL.
 * mtgp_mlp_train_step -- one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr on
 *   the same loss; loss as above.
 * The handle's buffers are reused by every call: calls on one handle must be ordered on one stream.
 */
typedef struct mtgp_mlp_s mtgp_mlp_t;
int mtgp_mlp_create(mtgp_mlp_t** out, int nlayers, const int* widths, int max_batch);
int mtgp_mlp_destroy(mtgp_mlp_t* m);
int mtgp_mlp_set_params(mtgp_mlp_t* m, const float* params, const float* mu, const float* sd);
int mtgp_mlp_get_params(mtgp_mlp_t* m, float* params, float* mu, float* sd);
int mtgp_mlp_fit_scaling(mtgp_mlp_t* m, int rows, const float* x, cudaStream_t stream);
int mtgp_mlp_forward(mtgp_mlp_t* m, int B, const float* x, float* y, cudaStream_t stream);
int mtgp_mlp_gradients(mtgp_mlp_t* m, int B, const float* x, const float* target, const float* mask,
                       const int* rows, float* grads, float* loss, cudaStream_t stream);
int mtgp_mlp_train_step(mtgp_mlp_t* m, int B, const float* x, const float* target, const float* mask,
                        const int* rows, float lr, float* loss, cudaStream_t stream);

/*
 * mtgp_propose -- the learned starting point of every fit in the batch, in one call: the spectral
 * features of mtgp_batch_features, the network's forward pass (in chunks of its max_batch rows) and
 * mtgp_batch_set_theta_proposal on the prediction.  A following mtgp_batch_fit with theta0 = NULL
 * starts the optimiser there.  No counterpart in the paper (it starts each fit from a fixed point).
 *   net     a network mapping 258 features to 37 outputs (mtgp_mlp_create widths 258, ..., 37), with
 *           its parameters and input scaling set; otherwise MTGP_ERR_INVALID_ARG.
 *   pred    device, nfits x 37 FP32, or NULL: receives the prediction (layout of mtgp_batch_targets).
 *   judge   0: every fit takes the prediction.  1: the exact MLE loss judges five candidates per fit and
 *           each fit keeps the one with the lowest NLL (one batched NLL + gradient evaluation per
 *           candidate): with c the log parameters set before the call (e.g. the plain optimiser's fixed
 *           start) and p the prediction's (W linearly), candidate 0 = p, 1 = p with sigma2 x 100,
 *           2 = (p + c) / 2, 3 = (p + 3 c) / 4, 4 = c.  2: the same judge over candidates 3 and 4 only
 *           (two evaluations), the more robust start for a later optimiser run (the nearer candidates
 *           more often lead it to a worse optimum).  The judged start is never worse than the caller's
 *           own start.  Other values: MTGP_ERR_INVALID_ARG.
 *   chosen  device, nfits ints, or NULL (judge = 1, 2): the candidate each fit kept (0 .. 4).
 * Needs mtgp_batch_set_y first, s = 2 and d <= 12 for every fit (else MTGP_ERR_UNSUPPORTED).  The
 * first call allocates the batch's feature, prediction and judge buffers (synchronously); later calls
 * are asynchronous on `stream`.  The network's buffers are used: order calls on one network on one stream.
 */
int mtgp_propose(mtgp_batch_t* b, mtgp_mlp_t* net, float* pred, int judge, int* chosen, cudaStream_t stream);

/*
 * mtgp_selftest_arith -- evaluates one of the library's arithmetic building blocks element-wise, for
 * testing its error bound against an FP64 reference (no counterpart in the paper).  x, y, out: device,
 * n doubles (y only for ops 3-5 and 8).  The double-float operations take their FP64 inputs rounded to
 * double-float (about 48 significant bits) and return the double-float result as a double.
 *   op 0  1 / x by the FP64 solvers' reciprocal (hardware approximation + one third-order refinement)
 *   op 1  x rounded to double-float and back
 *   op 2  1 / x in double-float (FP32 approximation + one Newton-Raphson step)
 *   op 3  x * y,  op 4  x + y,  op 5  x - y * y  (double-float)
 *   op 6  log of the product of x over each group of 32 consecutive elements (the double-float
 *         log-determinant accumulator and its double-float logarithm, ln m = 2 atanh((m-1)/(m+1))),
 *         written to the group's first element, 0 elsewhere; n % 32 == 0
 *   op 7  2^33 K(X / 2^32) of the order-2 DSI kernel (Eq. 2.6) in double-float, X = x (an integer in
 *         [0, 2^32)): the exact integer 3 2^32 - 2 b X - 5 2^(32 - b)
 *   op 8  the SI kernel of smoothness y (1..4, Eq. 2.5) at u = X / 2^32 in double-float, X = x
 * Asynchronous on `stream`; MTGP_ERR_INVALID_ARG for an unknown op or missing arrays.
 */
int mtgp_selftest_arith(int op, long long n, const double* x, const double* y, double* out, cudaStream_t stream);

/* mtgp_workspace_bytes -- device bytes the handle holds (for capacity planning). */
long long mtgp_workspace_bytes(const mtgp_t* h);

#ifdef __cplusplus
}
#endif
#endif /* MTGP_H */
