/*
 * img.h - C ABI of the GB300 bounded least-squares radio imager.
 *
 * The library estimates a sky image sigma (one real power per pixel) from an
 * array covariance matrix R_hat, following Sardarabadi, Leshem & van der Veen,
 * "Radio astronomical image formation using constrained least squares and
 * Krylov subspaces":
 *
 *   min_sigma 1/2 || W (r_hat - Psi sigma) ||^2   s.t.  0 <= sigma <= gamma
 *
 * with Psi = conj(A) o A the Khatri-Rao operator of the steering matrix A
 * (Sec. III-A, eq. bAt), W = I for constrained LS (eq. CLS) or the whitening
 * conj(L^-1) kron L^-1 with R_hat = L L^H plus the Jacobi change of variable
 * D for preconditioned WLS (eq. preWLS), and gamma the matched-filter or MVDR
 * dirty image (Sec. III-D).  The active-set method of Table I decides which
 * pixels are free; each equality subproblem is solved by LSQR (Sec. V-A) on
 * the operator pair Psi v = vect(A diag(v) A^H) and
 * Psi^H u = vectdiag(A^H U A) (Sec. V-B), never storing Psi or A.
 *
 * All work runs in CUDA kernels on one GPU; there is no CPU fallback.  A
 * missing or unusable GPU makes img_create return IMG_ECUDA.
 *
 * Conventions for every entry point
 *   - Matrices are column-major.  Complex numbers are interleaved (re, im)
 *     pairs of float (IMG_C64) or double (IMG_C128).
 *   - Pixel i = i_l + n_l * i_m  (column-major vectorisation of the image).
 *   - `on_device` = 0: the pointer is host memory (pageable or pinned).
 *     `on_device` = 1: the pointer is device memory of the context's device.
 *   - The caller owns every buffer it passes; the library copies what it
 *     keeps and never frees caller memory.
 *   - Calls on one context are not thread-safe; separate contexts are
 *     independent.  Every call returns after its results are in the
 *     caller's buffer (it synchronises the context's stream), except
 *     img_set_covariance with on_device = 1, which only enqueues the copy,
 *     and img_psi / img_psi_adj with on_device = 2 (stream-ordered).
 *   - No C++ exception crosses this boundary; failures are status codes.
 *   - K > 1 snapshots (Sec. II): one context per snapshot, combined by
 *     img_snapshot_image and img_snapshot_ls_image.
 *   - Environment: IMG_DEBUG (any value) reports a failing CUDA call of the
 *     host API on stderr with its source line; IMG_SOLVE_GRAPH=0 runs the
 *     solver's loop for p > 64 from the host instead of inside its CUDA graph
 *     (the same kernels in the same order, same results), for tools such as
 *     kernel profilers that cannot look inside graphs with conditional nodes.
 */
#ifndef IMG_GB300_H
#define IMG_GB300_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct img_ctx img_ctx;

typedef enum {
    IMG_OK = 0,
    IMG_EINVAL = 1,     /* bad argument or call order                        */
    IMG_ENOMEM = 2,     /* device allocation failed or a capacity exceeded   */
    IMG_ENOTPD = 3,     /* R_hat is not positive definite (Cholesky failed)  */
    IMG_ENOTCONV = 4,   /* active-set loop hit max_outer; partial image kept */
    IMG_ETIMEOUT = 5,   /* a bounded device wait ran out                     */
    IMG_ECUDA = 6       /* CUDA runtime error (no device, launch failure)    */
} img_status;

enum { IMG_COST_LS = 0, IMG_COST_PWLS = 1 };           /* eq. CLS / eq. preWLS   */
enum { IMG_BOUND_MF = 0, IMG_BOUND_MVDR = 1 };         /* eq. mfupper / mvdr_upper */
enum { IMG_INFLATE_NONE = 0,                           /* gamma = dirty          */
       IMG_INFLATE_RATIO = 1,                          /* (1 + alpha) dirty      */
       IMG_INFLATE_STD = 2 };                          /* dirty + alpha std      */
enum { IMG_C64 = 0, IMG_C128 = 1 };
/* Arithmetic of the operator products Psi and Psi^H.  The split forms run
 * tcgen05 tensor-core MMAs on v = hi + lo 16-bit parts with FP32
 * accumulation (3 products).  The solver uses them at every p <= 384: up to
 * p = 64 the whole Table I loop of a job runs in one CTA; above that it runs
 * as one CUDA graph per job (its loop and branches in device-side
 * conditional nodes) whose kernels spread each product over the GPU.  The
 * stand-alone operators (img_psi, img_psi_adj, the dirty / MVDR images)
 * use them up to p = 384 as well.  IMG_PREC_FP32 runs
 * everything on CUDA cores, the solver in one CTA per job. */
enum { IMG_PREC_FP32 = 0,       /* FP32 on CUDA cores                        */
       IMG_PREC_F16X3 = 1,      /* split FP16, power-of-two scaled: ~FP32    */
       IMG_PREC_BF16X3 = 2 };   /* split BF16: ~16 significant bits          */
enum { IMG_SET_L = 0, IMG_SET_U = 1, IMG_SET_F = 2 };  /* pixel sets (Sec. IV-A) */

/*
 * Problem description.  img_create copies every field and array.
 *   p        antennas, 2 <= p <= 384
 *   n_l,n_m  grid size, Q = n_l * n_m <= 2^24
 *   ant_xyz  host, p x 3 row-major (x_k, y_k, z_k) in units of the reference
 *            wavelength.  z_k must be 0 (planar array): the separable
 *            steering tables need it.  Non-zero z gives IMG_EINVAL.
 *   l, m     host, direction cosines of the grid lines (n_l and n_m values)
 *   lambda   wavelength in reference units (> 0); phases are x_k l / lambda
 *   Steering vector (Sec. II, Sec. IV-D, unit norm, sign -j):
 *     a_{k,i} = p^{-1/2} exp(-j 2 pi (x_k l_{i_l} + y_k m_{i_m}) / lambda)
 *   cost     IMG_COST_LS or IMG_COST_PWLS
 *   bound    IMG_BOUND_MF or IMG_BOUND_MVDR
 *   bias_c   0: C = 1;  1: C = N / (N - p)       (Appendix A, eq. C)
 *   inflate, alpha   upper-bound inflation (Sec. III-D and Appendix A)
 *   kappa    detection threshold eps_i = kappa * std_i of the cost's dirty
 *            image (Sec. IV-C); 0 asks for the exact KKT point
 *   eps_floor  eps_i >= eps_floor * max(dirty image of the cost)
 *   lsqr_atol, lsqr_btol, lsqr_maxit  LSQR stopping rules (Paige-Saunders);
 *            maxit 0 means 4 f + 20 for f free pixels
 *   max_outer  cap on passes of the Table I loop (0: 10 Q + 100)
 *   feas_tol  relative feasibility tolerance of the subproblem solution z:
 *            -feas_tol u_i <= z_i <= (1 + feas_tol) u_i counts as feasible
 *            and z is clipped into [0, u_i].  The paper gives no tolerance;
 *            it matters because a lone free pixel's solution equals its
 *            bound exactly (PWLS with the MVDR bound and C = 1, CLS with the
 *            MF bound), so without one rounding decides the first test.
 *   precision  IMG_PREC_*
 *   support_cap  most pixels allowed off the lower bound at once (|F u U|);
 *            0 means min(Q, 16384).  Exceeding it ends the solve with
 *            IMG_ENOMEM.
 *   stream   cudaStream_t to run on, or NULL for a stream the context owns.
 */
typedef struct {
    int p, n_l, n_m;
    const double *ant_xyz;
    const double *l, *m;
    double lambda;
    int cost, bound, bias_c, inflate;
    double alpha, kappa, eps_floor;
    double lsqr_atol, lsqr_btol;
    int lsqr_maxit, max_outer;
    double feas_tol;
    int precision;
    int support_cap;
    void *stream;
} img_params;

/* Per-solve report. */
typedef struct {
    int status;          /* img_status of the solve                          */
    int outer;           /* passes of the Table I loop                       */
    int lsqr_iters;      /* LSQR iterations summed over all subproblems      */
    int n_free;          /* |F| at return                                    */
    int n_upper;         /* |U| at return                                    */
    int converged;       /* 1 when no multiplier is below its threshold      */
    double lambda_min;   /* smallest multiplier at the last gradient         */
    double op_flops;     /* algorithmic operator flops (Psi: 4p^2|S|,
                            Psi^H: 8p^2|S|) spent in this solve              */
    double cyc_total;    /* SM clock cycles of the solve (p <= 64); for the
                            graph-driven solver (p > 64) nanoseconds, and
                            cyc_aux[0] = kernels the solve executed          */
    double cyc_gradient; /* ... of which in full-image gradients             */
    double cyc_lsqr;     /* ... of which in LSQR subproblems                 */
    double cyc_lsqr_fwd; /* ... of which in LSQR's forward products M v      */
    double cyc_lsqr_adj; /* ... of which in LSQR's adjoint products M^H u    */
    double cyc_aux[6];   /* finer LSQR phases (diagnostic): forward chunks,
                            G read-out, u update, B build, adjoint MMA wait,
                            adjoint epilogues                               */
    double t_begin_ns;   /* device global timer when the job's CTA started   */
    double t_end_ns;     /* ... and when it finished                         */
} img_solve_info;

/* Fill *prm with defaults: PWLS, MVDR bound, C = 1, no inflation, kappa 6,
 * eps_floor 1e-6, LSQR atol = btol = 1e-6, maxit 0, max_outer 0,
 * feas_tol 1e-5, FP32. */
void img_params_default(img_params *prm);

/* Validate *prm, copy it, and allocate all device state for one job on the
 * current CUDA device.  *out is NULL on failure.  Errors: IMG_EINVAL (bad
 * sizes, z != 0, lambda <= 0, unknown enum), IMG_ENOMEM, IMG_ECUDA. */
img_status img_create(const img_params *prm, img_ctx **out);

/* Load the sample covariance R_hat = (1/N) sum_n y[n] y[n]^H (Sec. II).
 *   R      p x p Hermitian, column-major, dtype IMG_C64 or IMG_C128
 *   N      number of samples; must exceed p (R_hat singular otherwise and
 *          C undefined) -> else IMG_EINVAL
 * Host input is checked for finite, Hermitian (relative 1e-6) values with a
 * positive real diagonal; device input is copied asynchronously on the
 * context's stream (the caller keeps it alive until the next call on this
 * context returns).  Previous bounds and images are invalidated.  The
 * Cholesky factor is computed on the device at the next call that needs it;
 * a non-PD R_hat then makes that call return IMG_ENOTPD. */
img_status img_set_covariance(img_ctx *ctx, const void *R, int dtype,
                              long long N, int on_device);

/* Matched-filter dirty image sigma_MF,i = a_i^H R_hat a_i (eq. mfdimg, K=1)
 * written to out[0..Q).  Errors: IMG_EINVAL before img_set_covariance,
 * IMG_ENOTPD. */
img_status img_dirty(img_ctx *ctx, double *out, int on_device);

/* MVDR upper bound C / (a_i^H R_hat^-1 a_i) (eq. wmvdr with K = 1 and the
 * unbiased form with C, Sec. III-D), inflated as configured, into
 * out[0..Q).  It is the solver's gamma when bound = IMG_BOUND_MVDR.  The
 * denominator is evaluated in whitened form, ||L^-1 a_i||^2 with R_hat =
 * L L^H, in every arithmetic: a sum of squares keeps its rounding error
 * relative to itself at a bright source, where the quadratic form does not. */
img_status img_mvdr_bound(img_ctx *ctx, double *out, int on_device);

/* Bounded least-squares image (Table I with LSQR subproblems) into
 * sigma[0..Q).  info may be NULL.  Returns IMG_ENOTCONV when max_outer is
 * reached (sigma holds the last feasible image), IMG_ENOMEM when
 * support_cap is exceeded. */
img_status img_solve(img_ctx *ctx, double *sigma, img_solve_info *info,
                     int on_device);

/* Pixel sets of the last solve (IMG_SET_L / _U / _F per pixel) into
 * sets[0..Q), host memory. */
img_status img_get_sets(img_ctx *ctx, unsigned char *sets);

/* Gradient g (eq. gls or eq. gmvdr, in the solver variable) at the last
 * solve's final image into grad[0..Q), host memory. */
img_status img_get_gradient(img_ctx *ctx, double *grad);

/* Decisions of the last solve in order (Table I): events[k] encodes the
 * kind in bits 24..25 (0: pixel freed, 1: pixel clamped to L, 2: clamped
 * to U) and the pixel in bits 0..23; values[k] is the multiplier lambda_i
 * of a freed pixel or the step mu_max of a clamp.  At most `capacity`
 * entries are written (host memory); *count receives the total number of
 * decisions, which may exceed what was recorded when the log filled. */
img_status img_get_events(img_ctx *ctx, int *events, double *values, int capacity,
                          int *count);

/* Forward operator Psi x = vect(A diag(x) A^H) (notation section; Sec. V-B):
 * x[0..Q) real (double) -> Kout p x p complex128 column-major. */
img_status img_psi(img_ctx *ctx, const double *x, double *Kout, int on_device);

/* Adjoint operator (Psi^H vect(U))_i = Re(a_i^H U a_i) (Sec. V-B):
 * U p x p Hermitian complex128 column-major -> out[0..Q) double.
 * Tensor-core arithmetic (IMG_PREC_F16X3 / BF16X3): up to p = 256 in the
 * warp-specialised kernel that streams the operand from global memory, for
 * 256 < p <= 384 on the solver's (tile, unit) work-item kernel (whose
 * buffers the first such call allocates); the forward (img_psi) forms
 * tensor-core Gram blocks up to p = 384.
 * img_psi and img_psi_adj also take on_device = 2: device pointers, work
 * queued on the context's stream and the call returns without waiting
 * (the caller orders or synchronises with that stream). */
img_status img_psi_adj(img_ctx *ctx, const double *U, double *out, int on_device);

/* Failure-detection self-test of the bounded waits that every tensor-core
 * kernel uses (not part of the paper): one CTA on the current device waits on
 * an mbarrier that receives its arrival only when arrive != 0, gives up after
 * `polls` polls (1 .. 2^26) and frees its tensor memory on the normal exit
 * path.  Returns IMG_ETIMEOUT when the wait ran out, IMG_OK when it completed,
 * IMG_EINVAL for polls outside the range, IMG_ECUDA on a CUDA error.  The
 * device stays usable either way; no fault or trap is involved. */
img_status img_check_wait(unsigned polls, int arrive);

/* Unconstrained LS / WLS image with every pixel free (Sec. III-B/C: the LS
 * and WLS images; Sec. V-A: LSQR): min ||b - M x|| over all Q pixels with
 * M = Psi, b = vect(R_hat) (IMG_COST_LS) or M = W Psi D^-1, b = W vect(R_hat)
 * (IMG_COST_PWLS, W = conj(L^-1) kron L^-1), cold start x0 = 0, no bounds.
 * The bidiagonalisation runs on the device (operators as in img_psi /
 * img_psi_adj, FP64 scalar recurrences in a one-thread kernel); the
 * Paige-Saunders stopping tests with the context's lsqr_atol / lsqr_btol are
 * checked every 10 iterations.  maxit <= 0: 200 iterations at most.
 * sigma[0..Q) receives the image (host or device per on_device); info (may
 * be NULL): lsqr_iters, converged (1 when a stopping test held),
 * lambda_min = final residual norm estimate, op_flops, t_end_ns = wall time.
 * Work buffers are allocated on the first call and kept with the context.
 * Errors: IMG_EINVAL (no covariance), IMG_ENOTPD, IMG_ECUDA. */
img_status img_ls_image(img_ctx *ctx, int maxit, double *sigma, img_solve_info *info, int on_device);

/* Dirty images over K > 1 snapshots (Sec. II: one sky seen by an array that
 * turns with the Earth, one sample covariance R_hat_k per snapshot).  Each
 * snapshot is a context of its own: snap[k] holds snapshot k's antenna
 * positions and covariance.  With d_{i,k} = a_{i,k}^H R_hat_k a_{i,k} and
 * h_{i,k} = a_{i,k}^H R_hat_k^{-1} a_{i,k} (each context's own dirty image and
 * MVDR denominator), out[0..Q) receives
 *   IMG_SNAP_MF    (1/K) sum_k d_{i,k}               MF dirty image, Sec. III-C
 *   IMG_SNAP_MVDR  C K / sum_k h_{i,k}               unbiased MVDR, Sec. III-D, eq. C
 *   IMG_SNAP_ASSC  C / max_k h_{i,k}                 ASSC bound, eq. ASSC0
 * with C = N/(N-p) when bias_c is set, else 1; no inflation is applied.
 * Sums run in snapshot order in FP64 over the contexts' FP32 per-pixel
 * values, so K = 1 reproduces img_dirty and (uninflated) img_mvdr_bound bit
 * for bit.  1 <= K <= IMG_MAX_SNAPSHOTS.  Every context must hold a
 * covariance, use the same device, and agree on p, the grid (n_l, n_m, l,
 * m), lambda, N and bias_c; otherwise IMG_EINVAL.  Each context's factor and
 * bounds are computed if needed (IMG_ENOTPD if one fails); the combination
 * runs on snap[0]'s stream and the call returns after it finished.  out is
 * host or device memory per on_device. */
enum { IMG_SNAP_MF = 0, IMG_SNAP_MVDR = 1, IMG_SNAP_ASSC = 2 };
#define IMG_MAX_SNAPSHOTS 32
img_status img_snapshot_image(img_ctx *const *snap, int K, int kind, double *out, int on_device);

/* Unconstrained LS / WLS image over K snapshots (Sec. II stacked model,
 * eq. vectRtotal; Sec. III-B/C images; Sec. V-A LSQR), every pixel free:
 * min over x of sum_k ||b_k - M_k x||^2 with, per snapshot k (context
 * snap[k]), M_k = Psi_k, b_k = vect(R_hat_k) (IMG_COST_LS) or
 * M_k = W_k Psi_k D^-1, b_k = W_k vect(R_hat_k), W_k = conj(L_k^-1) kron L_k^-1
 * (IMG_COST_PWLS), D = diag((sum_k h_{i,k})^2 / (K C)) (eq. D), sigma = D^-1 x.
 * The weighting acts on each snapshot's block (the paper writes it with the
 * block-diagonal R_hat).  LSQR as in img_ls_image: device-side Golub-Kahan
 * over the K blocks of u (one p x p block per snapshot), the snapshots'
 * operators run one after another on snap[0]'s stream and M^H u sums them in
 * snapshot order; snap[0]'s lsqr_atol / lsqr_btol, tests every 10
 * iterations, maxit <= 0: 200.  The contexts must satisfy the conditions of
 * img_snapshot_image and share the cost.  Each call allocates its work
 * buffers (2 K p^2 complex + O(Q)) and frees them before returning.
 * sigma[0..Q) host or device per on_device; info as in img_ls_image with
 * op_flops summed over the snapshots. */
img_status img_snapshot_ls_image(img_ctx *const *snap, int K, int maxit, double *sigma, img_solve_info *info,
                                 int on_device);

/* Factor R_hat, dirty images and bounds of several jobs in single launches
 * (the step img_solve_batch would otherwise run first).  Every context must
 * hold a covariance and use the same device; runs on ctxs[0]'s stream.
 * Returns the first job's IMG_ENOTPD if any factorisation failed. */
img_status img_prepare_batch(img_ctx *const *ctxs, int n);

/* Batch of independent jobs in single launches (the paper has no batching;
 * jobs are independent, Sec. V-B).  Every context must hold a covariance and
 * use the same device.  sigma[j] receives job j's image (host or device per
 * on_device), infos[j] its report (may be NULL).  Uses ctxs[0]'s stream.
 * Returns the first non-OK job status, or IMG_OK. */
img_status img_solve_batch(img_ctx *const *ctxs, int n, double *const *sigma,
                           img_solve_info *infos, int on_device);

/* Forward operator K = Psi x (as img_psi with IMG_PREC_FP32) for callers
 * that cannot allocate device memory - code inside a host framework whose
 * allocator owns the GPU's memory, or a real-time loop that must not hit
 * cudaMalloc's implicit synchronisation.  The paper has no counterpart: it is
 * a deployment variant.  No context is needed and nothing is allocated: the
 * steering tables and split-K partial sums live in one static device array
 * of 2.25 MiB that every GPU loading the library holds until exit.
 *   p <= 64, n_l <= 256, n_m <= 256, n_l * n_m <= 65536; larger sizes give
 *   IMG_ENOMEM (beyond the fixed capacity), bad arguments IMG_EINVAL.
 *   ant_xyz (p x 3 row-major, z ignored), l (n_l), m (n_m), x (Q doubles):
 *   device memory.  Kout: device memory, p x p complex128 column-major.
 *   stream: cudaStream_t or NULL; the call synchronises it before returning.
 * The first call on a device looks up the array's device address (once per
 * device and CUDA context: after cudaDeviceReset the next call looks it up
 * again); make that first call before any stream capture.  A launch failure
 * of this call itself gives IMG_ECUDA; errors left by earlier, unrelated work
 * are neither reported nor cleared.  Every call reuses the same array: calls
 * that overlap on the GPU (other streams or threads) race with each other;
 * serialise them. */
img_status img_psi_noalloc(int p, int n_l, int n_m, const double *ant_xyz, const double *l,
                           const double *m, double lambda, const double *x, double *Kout,
                           void *stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching of independent jobs (not in the paper; jobs are
 * independent, Sec. V-B).  A scheduler thread admits submitted jobs while
 * fewer than max_inflight_jobs are on the GPU and the job contexts fit in
 * hbm_budget_bytes (contexts of the same p, n_l, n_m are pooled and reused),
 * and launches each admitted group - factor, bounds, solve - on one of
 * n_streams streams.  Later groups run beside earlier ones on the device.
 * A job's result does not depend on what else is in flight. */
typedef struct img_server img_server;
typedef struct {
    size_t hbm_budget_bytes;    /* device memory for pooled job contexts        */
    int max_inflight_jobs;      /* jobs on the GPU at once (0: 2 x SM count)     */
    int max_batch;              /* most jobs per launch group (0: 2); a free
                                   stream takes ceil(pending / free streams)    */
    int n_streams;              /* launch streams (0: 128, the number of kernels
                                   a GB300 runs at once)                        */
    int max_pixels;             /* largest Q accepted (0: 65536); sizes the
                                   pinned result buffers made at creation       */
} img_server_params;

/* Defaults: 8 GiB budget, 2 x SMs in flight, groups of up to 2, 128 streams,
 * 65536 pixels.  Nothing is allocated while jobs run except job contexts of a
 * shape the pool lacks (img_server_reserve avoids even that).
 * Independent streams only overlap when CUDA_DEVICE_MAX_CONNECTIONS (set
 * before CUDA initialises) gives them separate hardware queues; 32 is the
 * most CUDA allows. */
void img_server_params_default(img_server_params *p);
img_status img_server_create(const img_server_params *prm, img_server **out);
/* Pre-create `count` pooled contexts for jobs shaped like *prm (p, n_l, n_m
 * and support cap), so that admission later allocates nothing.  IMG_ENOMEM
 * when the budget holds fewer (those that fit are kept). */
img_status img_server_reserve(img_server *s, const img_params *prm, int count);
/* Queue one job: *prm describes it as for img_create (arrays copied), R and N
 * as for img_set_covariance (host memory, copied).  *job_id identifies it.
 * IMG_EINVAL for jobs with more than max_pixels pixels. */
img_status img_server_submit(img_server *s, const img_params *prm, const void *R, int dtype,
                             long long N, long long *job_id);
/* Wait up to timeout_ms for job_id; on completion copy its image (Q doubles,
 * host) and report (either may be NULL), set *latency_ms (submit to done,
 * may be NULL), forget the job and return its solve status.  IMG_ETIMEOUT
 * when it is still running (call again), IMG_EINVAL for an unknown id. */
img_status img_server_wait(img_server *s, long long job_id, double *sigma, img_solve_info *info,
                           double timeout_ms, double *latency_ms);
/* Finish queued work, stop the scheduler and free everything. */
void img_server_destroy(img_server *s);

/* Release all device memory of ctx.  NULL is allowed. */
void img_destroy(img_ctx *ctx);

/* Static string for a status code. */
const char *img_status_str(img_status s);

#ifdef __cplusplus
}
#endif
#endif /* IMG_GB300_H */
