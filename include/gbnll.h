/*
 * gbnll.h -- C ABI of the GB300 (sm_103a) unbinned maximum-likelihood hot path.
 *
 * The library evaluates, for a fixed data sample and a parameter vector theta,
 *     NLL(theta) = - sum_i w_i ln P(x_i | theta)                (paper Sec. 2.1, Eq. 1)
 * and its analytic gradient dNLL/dtheta (Sec. 2.1 and Sec. 2.2 ask for analytic first
 * derivatives for gradient-based minimisers), in IEEE FP64 on the GPU, and minimises it
 * with a host quasi-Newton minimiser (Sec. 2.1: the minimiser runs on the host and the
 * accelerator evaluates the likelihood).  w_i = 1 unless weights are loaded.
 *
 * Models (fixed parameter order):
 *   NLL_MODEL_MASS1D (Sec. 2.4.1, Eq. 2; Sec. 3.2): observable m on [ma, mb];
 *     P = fsig G(m; mu, sigma) + (1 - fsig) E(m; alpha), each normalised on [ma, mb];
 *     theta = [mu, sigma, alpha, fsig].
 *   NLL_MODEL_KSTARMUMU4D: observables (m, cos theta_l, cos theta_K, phi) on
 *     [ma, mb] x [-1, 1] x [-1, 1] x [-pi, pi];
 *     P = fsig G(m) A(angles) + (1 - fsig) E(m) prod_j C_j(x_j) / Nc_j, with A the
 *     angular rate of Sec. 2.4.2 Eq. 3 and C_j = 1 + c1_j x + c2_j (2x^2 - 1) in
 *     x = cos theta_l, cos theta_K, phi/pi (the paper's angular benchmark has no mass
 *     dimension or background; this product background is the library's 4D model);
 *     theta = [mu, sigma, FL, S3, S4, S5, AFB, S7, S8, S9, alpha,
 *              c1_ctl, c2_ctl, c1_ctk, c2_ctk, c1_phi, c2_phi, fsig].
 *
 * Conventions for every call:
 *   - Every function returns an nll_status; none aborts or throws.  nll_last_error()
 *     gives the text of the model's most recent error.
 *   - Pointers passed in are borrowed for the duration of the call only.  The library
 *     owns all device memory it allocates (event copies, reduction buffers) and frees
 *     it in nll_destroy().
 *   - A model is bound to one device and one CUDA stream.  Calls on one model are
 *     serialised on that stream and block the calling host thread until their results
 *     are on the host.  A model is not thread-safe; different models are independent.
 *   - Arrays of doubles are IEEE binary64.  Event columns are structure-of-arrays.
 *   - Device memory: every model, batch and server counts the device memory it allocates
 *     against a limit read at its creation from the environment variable
 *     GBNLL_DEVICE_ALLOC_LIMIT (bytes; unset or 0: none).  An allocation past the limit fails
 *     like a failed cudaMalloc: the call returns NLL_ERR_OOM, the object keeps its previous
 *     state (a model or batch without a sample after a failed load) and can be destroyed.  This
 *     lets callers and tests provoke device-memory exhaustion from the host.
 */
#ifndef GBNLL_H
#define GBNLL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nll_model nll_model; /* opaque; owned by the library */

typedef enum {
    NLL_OK = 0,
    NLL_ERR_ARG = 1,              /* invalid argument, size, range or parameter value     */
    NLL_ERR_CUDA = 2,             /* a CUDA runtime call failed                           */
    NLL_ERR_OOM = 3,              /* device or pinned host allocation failed              */
    NLL_ERR_NONPOSITIVE_PDF = 4,  /* some P_i <= 0 or not finite; *nll_out = +inf         */
    NLL_ERR_NOT_CONVERGED = 5,    /* minimiser stopped before its convergence test passed */
    NLL_ERR_TIMEOUT = 6,          /* a bounded device-side wait ran out                   */
    NLL_ERR_STATE = 7             /* call out of order (e.g. evaluate before loading)     */
} nll_status;

typedef enum { NLL_MODEL_MASS1D = 1, NLL_MODEL_KSTARMUMU4D = 2 } nll_model_kind;

/* Kernel variants for the 4D model's angular part (paper Sec. 2.4.2):
 *   NLL_VARIANT_AUTO       precomputed basis when loaded with precompute, else direct;
 *   NLL_VARIANT_PRECOMPUTE event-only angular terms built once at load and read per eval;
 *   NLL_VARIANT_DIRECT     angular terms recomputed from the angles at every eval. */
typedef enum { NLL_VARIANT_AUTO = 0, NLL_VARIANT_PRECOMPUTE = 1, NLL_VARIANT_DIRECT = 2 } nll_variant;

/*
 * nll_create_model -- create a model of `kind` on CUDA device `device`.
 *   obs_ranges   host array: [ma, mb] for MASS1D; [ma, mb, -1, 1, -1, 1, -pi, pi] for
 *                KSTARMUMU4D (the angular ranges must be exactly these; ma < mb finite).
 *                Paper Sec. 2.4.1 normalises over a fixed observable range.
 *   cuda_stream  a cudaStream_t cast to uintptr_t on which every launch and copy of this
 *                model is issued; 0 is CUDA's default (legacy) stream, as everywhere in CUDA
 *                (torch's default stream also has handle 0).  The stream is borrowed: the
 *                caller keeps it alive until nll_destroy().
 *   out          receives the model handle (NULL on error).
 * Errors: NLL_ERR_ARG (kind, ranges), NLL_ERR_CUDA (device), NLL_ERR_OOM.
 */
int nll_create_model(int kind, const double* obs_ranges, int device, uintptr_t cuda_stream, nll_model** out);

/*
 * nll_load_events -- give the model a data sample (replacing any previous one).
 *   columns      ndim pointers (1 for MASS1D: m; 4 for 4D: m, ctl, ctk, phi), each to
 *                n_events doubles.
 *   on_device    0: host pointers, 1: device pointers on the model's device; the library
 *                copies them into its own 256-byte-aligned SoA store (padded to a tile
 *                multiple) before returning.  Host columns the device can read -- pinned
 *                or registered memory, and ordinary pageable memory on a device with
 *                cudaDevAttrPageableMemoryAccess -- are read in place by the load's
 *                statistics kernel, which stores the events as it checks them (one pass,
 *                no copy-engine transfer or host-side staging); other host memory is
 *                copied by cudaMemcpyAsync.
 *                2 (in place): nothing is copied or stored; every evaluation reads the
 *                caller's buffers where they are.  They must be memory the model's device can
 *                read -- its own device memory, managed memory, pinned or registered host
 *                memory, or any host memory when the device reports
 *                cudaDevAttrPageableMemoryAccess (a coherent CPU-GPU link, as on Grace
 *                systems) -- each 16-byte aligned (checked; NLL_ERR_ARG otherwise), and the
 *                caller keeps them alive and unchanged until the next load or nll_destroy.
 *                Meant for samples evaluated once or a few times (a stream of batches): the
 *                transfer then overlaps the evaluation instead of preceding it.  The 4D model
 *                uses the direct variant (no precompute).  Events outside the ranges are
 *                reported by the evaluation (NLL_ERR_ARG) instead of by the load.
 *   weights      n_events per-event weights w_i (same memory space), or NULL for w_i = 1.
 *   precompute   4D only: 1 = build the event-only angular basis once here (paper
 *                Sec. 2.4.2 event-dependent precompute), 0 = keep only the raw angles
 *                (ignored in place).
 * Events outside the observable ranges, or non-finite values/weights, are rejected with
 * NLL_ERR_ARG and the model keeps no sample.  n_events may be 0 (NLL = 0, gradient 0).
 */
int nll_load_events(nll_model* m, const double* const* columns, const double* weights, int64_t n_events,
                    int on_device, int precompute);

/*
 * nll_eval -- NLL(theta) (paper Eq. 1) for the loaded sample.
 *   theta        host array of n_params = nll_num_params(m) doubles, in the model's order.
 *                sigma > 0, 0 <= fsig <= 1, all finite; 4D: 2 - (2/3) c2_j > 0.
 *   nll_out      host double.
 * Returns NLL_ERR_NONPOSITIVE_PDF with *nll_out = +inf if some P_i <= 0 or is not finite.
 * Synchronous: returns once the results are on the host (the last launch writes them to
 * mapped host memory and sets completion words the call polls, so it may return a few
 * microseconds before the stream reports the launch complete; later work on the model's
 * stream is ordered after it as usual).
 */
int nll_eval(nll_model* m, const double* theta, int n_params, double* nll_out);

/*
 * nll_eval_grad -- NLL(theta) and its gradient in one fused pass over the events.
 *   grad_out     host array of n_params doubles, dNLL/dtheta_k in the model's order.
 * Requires 0 < fsig < 1 (the fsig derivative divides the component sums by fsig and
 * 1 - fsig); otherwise as nll_eval.
 */
int nll_eval_grad(nll_model* m, const double* theta, int n_params, double* nll_out, double* grad_out);

/* Minimiser options and result (paper Sec. 2.1: Migrad-style variable-metric minimiser
 * on the host; Sec. 3.1: uncertainties from the inverse Hessian, HESSE). */
typedef struct {
    double tol_edm; /* stop when EDM = g^T V g / 2 < tol_edm (e.g. 1e-8; <= 0 -> 1e-8)       */
    int max_iter;   /* quasi-Newton iterations (<= 0 -> 500)                                  */
    int strategy;   /* 0: start from diag(step^2); 1: start from a finite-difference Hessian;
                       2: start from the analytic Hessian (nll_eval_hess);
                       3 (batched and served fits; fit_minimise rejects it): as 2, the start
                       matrix of every fit from part of its events -- its first 1024 events, or
                       4 x 1024 spread over samples of more than 8192 -- scaled to the whole
                       sample; it only preconditions the quasi-Newton steps (the minimum and,
                       with hessian 2 / 3, the covariance are those of the whole sample);
                       4 (fit_minimise): damped Newton steps with the analytic Hessian at every
                       iterate (one nll_eval_hess pass each, line search included); the
                       covariance is the inverse Hessian of the final point (sandwich with
                       hessian 3, any other hessian value acts as 2).  Far fewer passes than
                       the quasi-Newton route, so faster where a pass is mostly launch latency
                       (samples of up to ~10^5 events);
                       5 (batched and served fits; fit_minimise rejects it): as 2, the start
                       matrix from an event pass in single precision (staging, slot products
                       and per-512-event sums in float, relative error ~1e-6); a start matrix
                       only preconditions, so the minimum and the covariance (hessian 2 / 3,
                       always in double precision) are those of strategy 2, while the pass
                       costs a fraction of the double-precision one.  Unlike 2, the fit loop
                       evaluates the start point itself (in double precision)            */
    int hessian;    /* 0: covariance from the quasi-Newton matrix; 1: finite-difference
                       Hessian of the analytic gradient at the minimum plus Newton polish;
                       2: the same with the analytic Hessian, covariance H^-1;
                       3: as 2, covariance H^-1 W H^-1 (weighted fits, see nll_eval_hess).
                       Values 2 and 3 (and strategies 2 and 4) need second derivatives of a
                       model: fit_minimise_fcn rejects them with NLL_ERR_ARG.  Batched and served fits
                       run the analytic passes on the device (see nll_batch_fit; a server queues
                       the start-matrix pass with the first step after admission and polishes
                       at nll_server_poll). */
} fit_options;

#define FIT_MAXPAR 32
typedef struct {
    double theta[FIT_MAXPAR];               /* fitted parameters (fixed ones unchanged)       */
    double err[FIT_MAXPAR];                 /* sqrt(diag(cov)); 0 for fixed parameters        */
    double cov[FIT_MAXPAR * FIT_MAXPAR];    /* covariance, row-major n_params x n_params      */
    double nll, edm;                        /* objective and estimated distance to minimum    */
    int n_eval, n_iter, status;             /* evaluations, iterations, nll_status of the fit */
} fit_result;

/*
 * fit_minimise -- minimise the model's NLL with the library's quasi-Newton (BFGS)
 * minimiser, evaluating NLL and gradient on the GPU at each step.
 *   theta0, lo, hi, step  host arrays of n_params: start point, bounds (lo < hi bounds the
 *                parameter through a smooth sine transform; lo >= hi means unbounded), and
 *                initial step sizes (> 0).  fixed[k] != 0 keeps parameter k at theta0[k].
 *   opt          options (NULL -> defaults); out: result (always filled as far as reached).
 * Returns NLL_OK on convergence, NLL_ERR_NOT_CONVERGED, or an evaluation error.
 */
int fit_minimise(nll_model* m, const double* theta0, const double* lo, const double* hi, const double* step,
                 const int* fixed, int n_params, const fit_options* opt, fit_result* out);

/*
 * fit_minimise_fcn -- the same minimiser on a caller-supplied objective (host callback).
 *   fcn(user, theta, nll_out, grad_out) must fill *nll_out and grad_out[n_params] and
 *   return 0 on success, non-zero to reject the point.  No GPU is involved.
 */
typedef int (*fit_fcn)(void* user, const double* theta, double* nll_out, double* grad_out);
int fit_minimise_fcn(fit_fcn fcn, void* user, const double* theta0, const double* lo, const double* hi,
                     const double* step, const int* fixed, int n_params, const fit_options* opt,
                     fit_result* out);

/*
 * nll_eval_hess -- NLL, gradient and the analytic Hessian of the NLL in one device pass
 * (paper Sec. 2.1: analytic Hessian for the HESSE uncertainties; Fisher information for
 * weighted fits), plus optionally the squared-weight score matrix
 *     W_ab = sum_i w_i^2 (d ln P_i / d theta_a)(d ln P_i / d theta_b),
 * so that H^-1 W H^-1 is the asymptotic covariance of a weighted fit (Langenbruch,
 * Eur. Phys. J. C 82 (2022) 393).
 *   theta     host array of n_params (0 < fsig < 1, as nll_eval_grad)
 *   nll_out   host scalar; grad_out host n_params or NULL
 *   hess_out  host n_params x n_params, row-major, symmetric: d^2 NLL / dtheta_a dtheta_b
 *   w2_out    host n_params x n_params or NULL (W; equals the Hessian's expectation for w = 1)
 * Deterministic for a given device.  Status as nll_eval_grad (NLL_ERR_NONPOSITIVE_PDF fills
 * the outputs with +inf / NaN).  Its cost is a few gradient evaluations (one FMA per event
 * per matrix entry), against 2 n_params of them for a finite-difference Hessian.
 */
int nll_eval_hess(nll_model* m, const double* theta, int n_params, double* nll_out, double* grad_out,
                  double* hess_out, double* w2_out);

/* Slots of the Hessian pass: per-event products it sums (one FP64 FMA per event each) for
 * model `kind`, with or without weights and W.  -1 for an unknown kind.  No GPU needed. */
int nll_hess_num_slots(int kind, int weighted, int want_w2);

/* Number of parameters of the model (4 or 18) and the name of parameter i. */
int nll_num_params(const nll_model* m);
const char* nll_param_name(const nll_model* m, int i);

/* Text of the most recent error on this model ("" if none).  Valid until the next call. */
const char* nll_last_error(const nll_model* m);

/* Free the model and all its device and host buffers.  NULL is accepted. */
void nll_destroy(nll_model* m);

/*
 * Launch configuration and measurement.
 *   nll_set_launch  blocks per SM (1..32) and threads per block (64..1024, multiple of 64)
 *                   of the fused kernel, and the 4D variant (nll_variant).  0 keeps a value.
 *   nll_autotune    times the candidate launch shapes (and both 4D variants when the basis is
 *                   loaded) on the loaded sample and keeps the fastest; blocks the host.  With
 *                   the environment variable GBNLL_TUNE_CACHE naming a file, a result kept
 *                   there for the same device, model, variant choice, weights, gradient,
 *                   in-place mode and power-of-two sample size is taken without timing, and a
 *                   new measurement is appended to it (plain text, one line per result;
 *                   nll_batch_autotune likewise, keyed by model, weights, basis and the
 *                   power-of-two classes of the toy count and the mean toy size).
 *   nll_set_profiling / nll_last_kernel_ms   when profiling is on, each evaluation records
 *                   CUDA events on the model's stream around its launches (the fused
 *                   kernel and the final-sum kernel behind it; for nll_eval_hess the
 *                   Hessian kernel and its slot totals); nll_last_kernel_ms waits for the
 *                   last one and returns its duration in milliseconds (NLL_ERR_STATE if no
 *                   evaluation was timed since profiling was switched on).
 *   nll_get_launch  reports blocks per SM, threads per block, variant and the SM count.
 */
int nll_set_launch(nll_model* m, int blocks_per_sm, int threads_per_block, int variant);
int nll_get_launch(const nll_model* m, int* blocks_per_sm, int* threads_per_block, int* variant, int* sm_count);
int nll_autotune(nll_model* m);
int nll_set_profiling(nll_model* m, int on);
int nll_last_kernel_ms(const nll_model* m, double* ms);

/*
 * nll_precomputed_basis -- copy the event-only angular basis built at load (4D,
 * precompute = 1) to `out` (host, row-major [n_events][13]): for each event
 *   h0, hFL, h_S3, h_S4, h_S5, h_AFB, h_S7, h_S8, h_S9, T2(ctl), T2(ctk), phi/pi, T2(phi/pi)
 * where A = h0 + FL hFL + sum_k S_k h_k (paper Sec. 2.4.2, Eq. 3 regrouped by parameter)
 * and T2(x) = 2x^2 - 1.  NLL_ERR_STATE if no basis was built.
 */
int nll_precomputed_basis(nll_model* m, double* out);

/*
 * nll_calibrate_fp64 -- diagnostic: FP64 throughput of device `device`, measured with
 * independent dependency chains over 8 blocks of 256 threads per SM (about 0.1 s).
 *   rates        host array of 6 doubles, operations per second of:
 *                [0] DFMA, [1] CUDA exp(), [2] CUDA 1.0/x (plus one DADD), [3] CUDA log()
 *                (plus one DADD), [4] the library's table exp, [5] the library's reciprocal
 *                (plus one DADD).  2 * rates[0] is the FP64 roofline in flop/s; rates[0] /
 *                rates[i] is the cost of operation i in DFMA issue slots.
 * The fused kernels do more FP64 work per byte than the GPU's FP64-to-HBM ratio, so they are
 * FP64-issue bound and this is their roofline.
 */
int nll_calibrate_fp64(int device, double* rates);

/*
 * nll_diag_math -- diagnostic: evaluate the library's device building blocks on n host
 * inputs x, writing host outputs y (fn 0: the exponential used by the kernels, Tang's table
 * method in fixed-point integer arithmetic, which takes its argument pre-scaled: y =
 * exp(x ln2/1024); fn 1: the reciprocal, a single-precision seed refined in integer
 * arithmetic; fn 2 / fn 3: sin x / cos x by the table method in integer arithmetic, for
 * |x| < 1024, as the 4D kernels use it for phi; fn 4: ln x after Tang's table method in
 * integer arithmetic, for positive normal x, as the weighted kernels use it; fn 5: the
 * hardware approximation of 1/x alone (rcp.approx.ftz.f64); fn 6: that approximation plus
 * one Newton step; fn 7: the square root in integer arithmetic, as the angular basis uses
 * it).  For accuracy tests against the host's extended precision; allocates temporary device
 * buffers; NLL_ERR_ARG for another fn.
 */
int nll_diag_math(int device, int fn, const double* x, double* y, int64_t n);

/* ------------------------------------------------------------------------------------
 * Batched pseudo-experiments (paper Sec. 2.5 and Sec. 3.1: fit validation and coverage
 * studies generate and fit many toys; Sec. 1: O(1e5) toys for coverage corrections).
 * A batch holds many independent samples of one model, of uneven sizes (CSR layout), on
 * one device.  Each minimiser step of every toy is one step of a device-resident loop:
 *   prepare  -- hoist the parameter-only terms of every active toy's trial point(s) on the
 *               device (Sec. 2.4.1), one work item per (toy, point);
 *   evaluate -- one persistent kernel: blocks pull work units (item x event tile) from a
 *               device counter and write each unit's sums (the fused NLL+gradient pass of
 *               nll_eval_grad);
 *   update   -- one warp per toy sums its units in tile order, assembles NLL and gradient and
 *               advances that toy's minimiser (BFGS, Armijo line search, sine-transform bounds,
 *               finite-difference Hessian of the analytic gradient at the minimum).
 * The three launches and a one-thread control kernel form the body of a while node of a CUDA
 * graph: the control kernel continues the loop while some toy is still fitting, so one graph
 * launch runs the whole fit loop on the device.  Schedules: tile_events = 0 gives one work unit per toy and point
 * (CTA-per-toy); tile_events > 0 splits every toy into tiles of that many events whose sums
 * are combined in tile order (split-toy).  Results are deterministic for a given schedule.
 * ------------------------------------------------------------------------------------ */
typedef struct nll_batch nll_batch; /* opaque; owned by the library */

/* Create a batch of `kind` on `device`, ranges as nll_create_model.  The batch runs on a
 * stream of its own (graph capture needs one); every call first waits for the work queued on
 * `cuda_stream` (0 = CUDA's default stream) and returns when its results are on the host. */
int nll_batch_create(int kind, const double* obs_ranges, int device, uintptr_t cuda_stream, nll_batch** out);

/*
 * nll_batch_load -- copy n_toys samples into the batch.
 *   offsets      host int64 array of n_toys + 1 entries; toy t owns events
 *                [offsets[t], offsets[t+1]) of the columns (non-decreasing, offsets[0] = 0).
 *   columns      ndim host pointers (as nll_load_events), offsets[n_toys] doubles each.
 *   weights      host per-event weights or NULL.
 *   precompute   4D only: build the event-only angular basis (paper Sec. 2.4.2).
 * Events outside the ranges are rejected (NLL_ERR_ARG).  Toys may be empty.
 */
int nll_batch_load(nll_batch* b, const int64_t* offsets, int n_toys, const double* const* columns,
                   const double* weights, int precompute);

/*
 * nll_batch_generate -- generate the toys on the device instead of loading them (paper
 * Sec. 2.5: accept-reject on the accelerator with the parameters fixed, so parameter-only
 * terms fold into constants).  Toy t gets counts[t] events drawn at `theta` from stream t of
 * a counter-based SplitMix64 generator seeded with `seed`; the result depends only on
 * (seed, t, event index), not on the launch.  precompute as nll_batch_load.
 * Returns NLL_ERR_ARG for an invalid theta, NLL_ERR_NOT_CONVERGED if some event exhausted its
 * accept-reject tries (the batch is then empty).
 */
int nll_batch_generate(nll_batch* b, const double* theta, const int64_t* counts, int n_toys, uint64_t seed,
                       int precompute);

/*
 * nll_generate -- generate n_events events of `kind` at `theta` into caller-owned device
 * columns (ndim pointers, n_events doubles each) on `device`/`cuda_stream`, from stream
 * `stream` of the generator seeded with `seed` (the same events as toy `stream` of
 * nll_batch_generate).  Allocates small temporary device buffers.  Blocks until done.
 */
int nll_generate(int kind, const double* obs_ranges, const double* theta, int64_t n_events, uint64_t seed,
                 uint64_t stream, int device, uintptr_t cuda_stream, double* const* dev_columns);

/* Diagnostic: the first n uniforms in (0, 1) of stream (seed, stream) of the device generator
 * (SplitMix64: value k = mix(state + (k+1) gamma), state = mix(seed ^ mix(stream gamma + 1))). */
int nll_diag_uniforms(uint64_t seed, uint64_t stream, int64_t n, int device, double* host_out);

/*
 * nll_batch_eval_grad -- one evaluation of every toy at its own parameter point.
 *   thetas       host [n_toys][npar]; nll_out host [n_toys]; grad_out host [n_toys][npar].
 *   status_out   host [n_toys] nll_status per toy (NULL allowed).
 * Returns NLL_OK if every toy evaluated, else the first failing toy's status.
 */
int nll_batch_eval_grad(nll_batch* b, const double* thetas, double* nll_out, double* grad_out, int* status_out);

/*
 * nll_batch_fit -- minimise every toy's NLL on the device (see above).
 *   theta0       host [n_toys][npar] start points, or [npar] shared by all toys if
 *                shared_start != 0; lo, hi, step, fixed as fit_minimise (shared by all toys).
 *   opt          tol_edm, max_iter, strategy (1: start from a finite-difference Hessian;
 *                2: from the analytic Hessian of every toy, one batched pass before the
 *                loop; 3: the same pass over part of every toy's events; 5: the same pass
 *                in single precision; see fit_options),
 *                hessian (1: finite-difference Hessian of the analytic gradient at the
 *                minimum for the covariance; 2: analytic Hessian, covariance H^-1; 3: as 2,
 *                covariance H^-1 W H^-1 for weighted toys -- one batched pass after the loop,
 *                no Newton polish; 0: covariance from the BFGS matrix).
 *   results      host array of n_toys fit_result.
 *   steps_out    number of device steps (iterations of the device-resident loop) used, or NULL.
 * Returns NLL_OK when every toy converged, else NLL_ERR_NOT_CONVERGED (see results[].status).
 */
int nll_batch_fit(nll_batch* b, const double* theta0, int shared_start, const double* lo, const double* hi,
                  const double* step, const int* fixed, const fit_options* opt, fit_result* results,
                  int* steps_out);

/*
 * nll_batch_fit_arrays -- nll_batch_fit with the results in plain per-toy arrays instead of
 * fit_result records (a fit_result holds FIT_MAXPAR-sized fields, over 8 KB per toy): the same
 * fit, arguments and return value.  Every output is host memory owned by the caller, or NULL
 * when not wanted:
 *   theta_out    [n_toys][npar] fitted parameters (fixed ones unchanged);
 *   err_out      [n_toys][npar] sqrt(diag(cov)), 0 for fixed parameters;
 *   cov_out      [n_toys][npar][npar] covariance, rows and columns of fixed parameters 0;
 *   nll_out, edm_out [n_toys]; n_eval_out, n_iter_out, status_out [n_toys] (nll_status).
 * Where the device can write every given output (pinned or managed memory, or ordinary host
 * memory on a system with pageable-memory access such as Grace-Blackwell) and status_out is
 * given, the last kernel of the fit writes them in place; otherwise the host unpacks them.
 */
int nll_batch_fit_arrays(nll_batch* b, const double* theta0, int shared_start, const double* lo, const double* hi,
                         const double* step, const int* fixed, const fit_options* opt, double* theta_out,
                         double* err_out, double* cov_out, double* nll_out, double* edm_out, int* n_eval_out,
                         int* n_iter_out, int* status_out, int* steps_out);

/*
 * nll_batch_eval_hess -- NLL, gradient, analytic Hessian (and optionally W = sum w^2 s s^T)
 * of every toy at its own parameter point, in one device pass (the per-toy version of
 * nll_eval_hess; paper Sec. 2.1).
 *   thetas       host [n_toys][n_params], or one shared point if shared != 0.
 *   nll_out      host [n_toys]; grad_out host [n_toys][n_params] or NULL;
 *   hess_out     host [n_toys][n_params][n_params]; w2_out the same layout, or NULL.
 *   status_out   host [n_toys] nll_status per toy (NLL_ERR_ARG: invalid parameter point;
 *                NLL_ERR_NONPOSITIVE_PDF: density not positive), or NULL.
 * Returns the first non-OK toy status, or NLL_OK; the outputs of such toys are +inf / NaN.
 */
int nll_batch_eval_hess(nll_batch* b, const double* thetas, int shared, double* nll_out, double* grad_out,
                        double* hess_out, double* w2_out, int* status_out);

/* Schedule: tile_events = 0 (CTA-per-toy) or > 0 (split-toy, multiple of 2);
 * blocks_per_sm of the persistent evaluation kernel (0 keeps the value). */
int nll_batch_set_schedule(nll_batch* b, int tile_events, int blocks_per_sm);
int nll_batch_get_schedule(const nll_batch* b, int* tile_events, int* blocks_per_sm);
/* Time both schedules (and tile sizes) on the loaded toys and keep the fastest. */
int nll_batch_autotune(nll_batch* b);
int nll_batch_num_toys(const nll_batch* b);
const char* nll_batch_last_error(const nll_batch* b);
void nll_batch_destroy(nll_batch* b);

/* ------------------------------------------------------------------------------------
 * Serving: continuous batching of independent fits of one model kind.  A server owns
 * `max_slots` fit slots and an event pool of `pool_events` events on the device (the HBM
 * budget).  A submitted fit is admitted into a free slot if the pool has a free range for
 * its events; every nll_server_step advances all busy slots by one device step of the
 * batched machinery above (one CUDA graph replay); finished fits are collected with
 * nll_server_poll, which frees their slot and pool range for the next admissions.  A fit's
 * result does not depend on which other fits share the steps (each fit's sums are reduced
 * in its own fixed order).
 * ------------------------------------------------------------------------------------ */
typedef struct nll_server nll_server; /* opaque; owned by the library */

/*
 * nll_server_create -- kind, obs_ranges and device as nll_create_model.
 *   max_slots    concurrent fits (>= 1).     pool_events  device event capacity (>= 1).
 *   tile_events  split-toy tile size (even, >= 128; 0 = 4096).
 *   lo, hi, step, fixed, opt   minimiser settings shared by every fit (as fit_minimise).
 * The server runs on its own CUDA stream.
 */
int nll_server_create(int kind, const double* obs_ranges, int device, int max_slots, int64_t pool_events,
                      int tile_events, const double* lo, const double* hi, const double* step, const int* fixed,
                      const fit_options* opt, nll_server** out);

/*
 * nll_server_submit -- admit one fit: n_events events (host SoA columns; weights must be NULL,
 * a server serves unweighted fits) and its start point theta0 (host, npar doubles).  On
 * success *request_id identifies the fit and its events are on the device.  The events go to
 * the device on the server's collection stream (highest stream priority; host columns the
 * device can read -- pinned, or pageable with pageable-memory access -- are read in place by
 * the range-check kernel, others copied) and the call waits only for that copy and the range check, not for
 * the steps in flight; the fit joins the steps queued after it.
 * Returns NLL_ERR_STATE (nothing admitted) when no slot or no pool range is free: the
 * caller keeps the request queued and retries after nll_server_poll returned finished fits.
 * Returns NLL_ERR_ARG for events outside the ranges (checked on the device after the copy;
 * the pool range is released again) or more events than the whole pool.
 */
int nll_server_submit(nll_server* s, const double* const* columns, const double* weights, int64_t n_events,
                      const double* theta0, int64_t* request_id);

/* Queue n_steps device steps (graph replays) advancing every busy slot; returns without
 * waiting, so steps of servers on different streams overlap on the device.  With strategy 2
 * the call first queues one analytic Hessian pass over the fits admitted since the last step
 * (their start matrices) on the server's step stream, ahead of the steps (no wait).
 * nll_server_sync waits for everything queued. */
int nll_server_step(nll_server* s, int n_steps);
int nll_server_sync(nll_server* s);

/*
 * nll_server_progress -- non-blocking: *steps_in_flight receives the number of queued steps
 * not yet completed (of the last 64), *finished the number of fits that have finished and
 * wait for nll_server_poll (either output may be NULL).  A request loop keeps a couple of
 * steps queued and polls when fits have finished, so the device never waits for the host.
 */
int nll_server_progress(const nll_server* s, int* steps_in_flight, int* finished);

/*
 * nll_server_poll -- collect up to max_results finished fits: ids_out[i] and results[i]
 * (host arrays); *n_out receives the count (0 when none has finished; the call does not wait
 * for steps in flight).  Their slots and pool ranges are released.  With hessian 2 / 3 the
 * finished fits are first polished with the analytic Hessian (Newton passes, covariance) on
 * the server's collection stream, while the steps of the other fits go on.
 */
int nll_server_poll(nll_server* s, int64_t* ids_out, fit_result* results, int max_results, int* n_out);

/*
 * nll_server_cancel -- withdraw an admitted fit that has not been polled yet: waits for the
 * queued steps, marks the fit finished on the device and releases its slot and pool range
 * without returning a result.  NLL_ERR_ARG if no such request is in the server.
 */
int nll_server_cancel(nll_server* s, int64_t request_id);

/* Busy slots, free slots and free pool events (any output may be NULL). */
int nll_server_status(const nll_server* s, int* busy, int* free_slots, int64_t* free_events);
const char* nll_server_last_error(const nll_server* s);
void nll_server_destroy(nll_server* s);

/*
 * nll_eval_grad_4d_noalloc -- NLL and gradient of the 4D model for a sample that stays in
 * the caller's device memory, without allocating any device memory.  The paper has no
 * counterpart: this entry exists for callers that cannot call cudaMalloc -- for example code
 * running where another allocator owns the device's memory (a framework that has reserved
 * the memory in its own pool), or loops that cannot afford cudaMalloc's implicit device-wide
 * synchronisation.  It runs the fused kernel of an in-place 4D model (nll_load_events with
 * on_device = 2): the direct angular variant (the basis is recomputed from the angles), loads
 * that never read past event n_events - 1, and the range check and sum w (m - ma) in the same
 * pass, so nothing per event is stored and one launch (plus its final sums) does the work.
 *   obs_ranges   [ma, mb, -1, 1, -1, 1, -pi, pi] (as nll_create_model).
 *   dev_columns  4 device pointers on the current device (m, ctl, ctk, phi), each 16-byte
 *                aligned (checked), holding at least n_events doubles.
 *   dev_weights  device pointer with the same layout, or NULL for w_i = 1.
 *   theta        host array of 18 parameters (order of nll_create_model); 0 < fsig < 1.
 *   blocks       grid size of the fused kernel, 0 = two blocks per SM; at most
 *                NLL_NOALLOC_MAX_BLOCKS, larger values are rejected with NLL_ERR_ARG.
 *   cuda_stream  stream of the launches and copies (0 = CUDA's default stream); the caller
 *                orders the writes of the columns before it.
 *   nll_out, grad_out  host outputs (1 and 18 doubles).  The call blocks until they are set.
 * Scratch: the block partials and the final sums live in one static __device__ array of
 * (23 x NLL_NOALLOC_MAX_BLOCKS + 32) doubles (about 189 KB), which every GPU that loads this
 * library holds until the process exits.  All calls share it and it keeps the last call's
 * contents; nothing in it needs clearing, since every launch writes each value it reads.
 * Calls that overlap on the GPU (from different host threads or streams) race on it and
 * must be serialised by the caller.  The first call on a device looks up the array's device
 * address and uploads the exponential and sin/cos table for that device (no allocation); make
 * that first call before any stream capture.  Errors: NLL_ERR_ARG (sizes, alignment, ranges,
 * parameters, events outside the ranges or negative weights: outputs +inf / NaN),
 * NLL_ERR_NONPOSITIVE_PDF, NLL_ERR_CUDA.  No text via nll_last_error.
 */
#define NLL_NOALLOC_MAX_BLOCKS 1024
int nll_eval_grad_4d_noalloc(const double* obs_ranges, const double* const* dev_columns, const double* dev_weights,
                             int64_t n_events, const double* theta, int n_params, int blocks, uintptr_t cuda_stream,
                             double* nll_out, double* grad_out);

#ifdef __cplusplus
}
#endif

#endif /* GBNLL_H */
