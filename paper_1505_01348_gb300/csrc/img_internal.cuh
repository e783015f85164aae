// Internal device-side job layout shared by the kernels and the host API.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/img.h"

namespace img {

constexpr int kThreads = 256;      // threads per CTA in every kernel
constexpr int kTile = 64;          // pixels per operator chunk / matrix tile edge

// Per-job report written by the solver (mirrors img_solve_info).
struct DevInfo {
    int status;
    int outer;
    int lsqr_iters;
    int n_free;
    int n_upper;
    int converged;
    double lambda_min;
    double op_flops;
    double cyc_total;
    double cyc_gradient;
    double cyc_lsqr;
    double cyc_lsqr_fwd;
    double cyc_lsqr_adj;
    double cyc_aux[6];
    unsigned long long t_begin_ns;   // device global timer at the job's start and end
    unsigned long long t_end_ns;
};

// Everything one imaging job keeps on the device.  All pointers are device
// memory carved from one allocation owned by the host context.
struct JobDev {
    // sizes and parameters
    int p, n_l, n_m, Q;
    int cost, bound, bias_c, inflate;
    int lsqr_maxit, max_outer, cap, precision;
    double alpha, kappa, eps_floor, lam, lsqr_atol, lsqr_btol, feas_tol;
    long long N;
    // geometry (copied from the host)
    const double *ant;     // p*3 row-major
    const double *lg;      // n_l
    const double *mg;      // n_m
    // covariance and factors (column-major p x p)
    double2 *R64;          // R_hat
    double2 *L64;          // Cholesky factor, lower
    double2 *Li64;         // L^-1, lower
    float2 *R32;           // R_hat
    float2 *Ri32;          // R_hat^-1
    float2 *Li32;          // L^-1
    float2 *LiH32;         // L^-H (column n holds the conjugate of row n of L^-1)
    // separable steering tables, pixel-major: El[il*p + k], Em[im*p + k]
    float2 *El;
    float2 *Em;
    // per-pixel arrays (Q)
    float *dirty;          // MF dirty image
    float *h;              // a^H R^-1 a
    float *scale;          // s_i: sigma_i = s_i x_i (1/D_i for PWLS, 1 for LS)
    float *eps;            // detection threshold in gradient units
    float *grad;           // last gradient (solver variable)
    double *upper;         // bound in the solver variable
    double *gamma;         // bound in sigma units
    double *mvb;           // MVDR bound C/h (inflated as configured)
    double *x;             // solver variable
    double *sigma;         // output image
    unsigned char *set;    // IMG_SET_*
    int *slot;             // support slot of a pixel or -1
    // support S = F u U: pixel ids and cached (whitened) steering vectors
    int *supp;             // cap
    float2 *cvec;          // cap * p, c_i = T a_i (T = L^-1 for PWLS, I for LS)
    float *cmax;           // cap, max over k of |Re c_i[k]|, |Im c_i[k]|
    int *fpos;             // cap, positions in supp of the free pixels
    float *v, *w, *xs;     // cap, LSQR vectors indexed by F position
    float *sF;             // cap, s_i of the free pixels in F order (per LSQR solve)
    float2 *W0, *W1, *W2;  // p*p scratch matrices
    // chunked B images of R_hat and R_hat^-1 for the wide tensor-core
    // operators (64 < p <= 256), and their scales
    unsigned char *Bimg;
    float *Bscale;
    unsigned *Bmax;      // max |entry| bits of the operators being imaged (atomicMax)
    // decision log (Table I order): kind << 24 | pixel, and lambda or mu
    int *ev;
    float *evv;
    int ev_cap;
    int *ev_count;
    // status and report
    DevInfo *info;
    int *flags;            // [0]: factor status, [1]: bounds valid
};

// Kernel launchers (defined in the .cu files, called by the host API).
// `jobs` is a device array of n job pointers.
cudaError_t launch_tables(JobDev *const *jobs, int n, cudaStream_t st);
cudaError_t launch_factor(JobDev *const *jobs, int n, cudaStream_t st);
// mode 1/2 use tensor cores: the shared-memory operator for p <= 64, the
// streamed (wide) operator for 64 < p <= 256.
cudaError_t launch_bounds(JobDev *const *jobs, int n, int max_tiles, int max_p, int mode,
                          cudaStream_t st);
cudaError_t launch_finalize(JobDev *const *jobs, int n, cudaStream_t st, int *batch_status);
// mode: 0 CUDA-core FP32 operators, 1 tensor cores FP16x3, 2 tensor cores BF16x3
cudaError_t launch_solve(JobDev *const *jobs, int n, int max_p, int mode, DevInfo *batch_info,
                         double *const *sigma_out, cudaStream_t st);
// Factor, bounds and solve of each job inside its own CTA (one launch).
cudaError_t launch_job(JobDev *const *jobs, int n, int max_p, int mode, DevInfo *batch_info,
                       double *const *sigma_out, cudaStream_t st);
cudaError_t launch_psi(const JobDev *job_dev, const float *wx, float2 *part, int nparts, int Q,
                       int p, int mode, double2 *Kout, cudaStream_t st);
// Bounded-wait self-test (one CTA; *status: IMG_OK or IMG_ETIMEOUT).
cudaError_t launch_wait_selftest(unsigned polls, int arrive, int *status, cudaStream_t st);

// Full-image LSQR (all pixels free): device vectors and FP64 scalars
// (kLsScalars doubles, indexed by kLs*); Q floats v, w, x, wx,
// Q doubles y; p x p complex u, Mv, T1, Uw (FP32) and Kd (FP64).
constexpr int kLsScalars = 16;
enum : int { kLsSsU = 0, kLsSsV, kLsAlpha, kLsBeta, kLsRhobar, kLsPhibar, kLsAnorm2, kLsT1, kLsT2, kLsIa,
             kLsBnorm, kLsRnorm, kLsArnorm, kLsUs, kLsXnorm2, kLsCount };
static_assert(kLsCount <= kLsScalars, "LSQR scalar block");
struct LsBufs {
    float2 *u, *Mv, *T1, *Uw;
    double2 *Kd;
    float *v, *w, *x, *wx;
    double *y, *sc;
};
// u = b / ||b||, v = M^H u / alpha, w = v, x = 0 (eq. initbeta, eq. initu).
cudaError_t ls_begin(const JobDev *jd, const JobDev &hj, LsBufs &b, int mode, cudaStream_t st);
// One Golub-Kahan step (eq. lanczos) with the Paige-Saunders rotation and
// the x, w updates.  mode 0: CUDA-core operators (part/nparts scratch);
// 1/2: tensor-core operators (fwd_part scratch).
cudaError_t ls_iterate(const JobDev *jd, const JobDev &hj, LsBufs &b, int mode, float *fwd_part, float2 *part,
                       int nparts, cudaStream_t st);
// sigma = scale o x (device, Q doubles); *xnorm2 (device) = ||x||^2 if given.
cudaError_t ls_finish(const JobDev &hj, LsBufs &b, double *sigma, double *xnorm2, cudaStream_t st);
cudaError_t ls_xnorm2(const JobDev &hj, LsBufs &b, double *out, cudaStream_t st);

// Per-snapshot arrays for the K-snapshot dirty images (passed by value).
struct SnapPtrs {
    const float *d[IMG_MAX_SNAPSHOTS];   // MF dirty image of snapshot k
    const float *h[IMG_MAX_SNAPSHOTS];   // a^H R_k^-1 a of snapshot k
};
// Full-image LSQR over K snapshots (stacked operator of Sec. II, eq.
// vectRtotal): u holds K blocks of p x p (b.u and b.Mv have K * p^2
// entries), v, w, x are shared, M^H u sums the snapshots' adjoints in
// snapshot order.  hj[k] is snapshot k's host mirror with scale replaced by
// the K-snapshot scale (1/D of eq. D for PWLS, 1 for CLS); snapshots run one
// after another on the given stream, sharing the scratch in b.
struct LsSnap {
    int K = 0;
    const JobDev *jd[IMG_MAX_SNAPSHOTS] = {};
    JobDev hj[IMG_MAX_SNAPSHOTS] = {};
    int mode[IMG_MAX_SNAPSHOTS] = {};
    float *fwd_part[IMG_MAX_SNAPSHOTS] = {};
    float2 *part[IMG_MAX_SNAPSHOTS] = {};
    int nparts[IMG_MAX_SNAPSHOTS] = {};
    double *yk = nullptr;      // Q doubles: one snapshot's M_k^H u_k
};
cudaError_t ls_snap_begin(const LsSnap &s, LsBufs &b, cudaStream_t st);
cudaError_t ls_snap_iterate(const LsSnap &s, LsBufs &b, cudaStream_t st);
cudaError_t launch_snap_scale(const SnapPtrs &sp, int K, int Q, int pwls, double C, float *scale, cudaStream_t st);

// Wide tensor-core forward K = Psi w (64 < p <= 256, mode 1 or 2): wbits is
// a device word (cleared here), part a scratch of psi_wide_part_floats(SMs)
// floats; Kout p x p complex128.
size_t psi_wide_part_floats(int sms);
cudaError_t launch_psi_wide(const JobDev *job_dev, unsigned *wbits, const float *wx, float *part, int Q, int p,
                            int n_l, int n_m, int mode, double2 *Kout, cudaStream_t st);
// Wide tensor-core adjoint (64 < p <= 256, mode 1 or 2) from U in FP32
// (u64 false) or FP64 complex (converted while the operand image is
// written); bmax is the job's Bmax (device), cleared here.
cudaError_t launch_psi_adj_wide(const JobDev *job_dev, unsigned *bmax, const void *U, bool u64, double *out,
                                int Q, int p, int mode, cudaStream_t st);
cudaError_t launch_psi_adj(const JobDev *job_dev, const float2 *U, double *out, int Q, int p,
                           int mode, cudaStream_t st);
cudaError_t launch_z2c(const double2 *src, float2 *dst, int n, cudaStream_t st);
cudaError_t launch_c2z(const float2 *src, double2 *dst, int n, cudaStream_t st);
cudaError_t launch_d2f(const double *src, float *dst, int n, cudaStream_t st);
cudaError_t launch_to_double(const float *src, double *dst, int n, cudaStream_t st);
cudaError_t launch_snapshot_image(const SnapPtrs &sp, int K, int Q, int kind, double C, double *out,
                                  cudaStream_t st);

// Wide tensor-core solver (64 < p <= 384, mode 1 or 2): the whole Table I
// loop of one job as a CUDA graph with device-side conditional nodes.
// ws_create allocates its buffers and instantiates the graph for the job's
// device arrays; ws_launch queues one solve on a stream.
struct WsHost;
cudaError_t ws_create(const JobDev &hj, const JobDev *dj, int mode, WsHost **out);
cudaError_t ws_launch(WsHost *w, cudaStream_t st);
// Dirty image (hj.dirty) and MVDR denominators (hj.h) of the job on the
// work-item tensor-core adjoint, after its factor (for 256 < p <= 384).
cudaError_t ws_bounds(WsHost *w, const JobDev &hj, cudaStream_t st);
// out_i = Re(a_i^H U a_i) for every pixel on the same kernels (U p x p FP32
// complex on the device, out Q doubles on the device).
cudaError_t ws_psi_adj(WsHost *w, const JobDev &hj, const float2 *U, double *out, cudaStream_t st);
size_t ws_size(const JobDev &hj);         // device bytes ws_create allocates
void ws_destroy(WsHost *w);

size_t solve_smem_bytes(int p, int mode);
constexpr int kMaxTcP = 64;   // tensor-core solver: 2p x 2p operand tiles in shared memory
constexpr int kMaxWideP = 256; // streamed tensor-core operators (bounds, Psi^H)
constexpr int kMaxWideSolveP = 384;  // graph-driven tensor-core solver above kMaxTcP
constexpr int kMaxWideFwdP = 384;    // tensor-core Gram-block forward (img_psi)
size_t bounds_smem_bytes(int p);

}  // namespace img
