// Host side of the C ABI declared in include/img.h: validation, device
// memory layout of a job, and the launch sequence of every call.
#include <chrono>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/img.h"
#include "img_internal.cuh"
#include "tc_wide.cuh"

using img::DevInfo;
using img::JobDev;

struct img_ctx {
    img_params prm;
    std::vector<double> ant, l, m;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *dmem = nullptr;
    size_t dbytes = 0;
    JobDev hj{};                 // host mirror (device pointers)
    JobDev *dj = nullptr;        // device copy of hj
    JobDev **djp = nullptr;      // device array {dj} for single-job launches
    bool has_cov = false;
    bool prepared = false;
    int prep_status = IMG_OK;
    bool solved = false;
    // operator scratch
    float *wx = nullptr;
    float2 *part = nullptr;
    int nparts = 0;
    float2 *U32 = nullptr;
    double2 *Z = nullptr;        // p*p complex128 staging
    double *outd = nullptr;      // Q doubles staging
    float *fwd_part = nullptr;   // partial Gram blocks of the wide forward (allocated on first use)
    void *ls_mem = nullptr;      // full-image LSQR vectors (allocated on first use)
    cudaGraphExec_t ls_exec = nullptr;   // one LSQR iteration as a CUDA graph (own stream only)
    img::WsHost *ws = nullptr;   // graph-driven wide solver (created on the first wide solve)
    cudaEvent_t ev = nullptr;    // ordering event for batched wide solves
};

namespace {

constexpr int kMaxP = 384;

img_status cuda_status(cudaError_t e) { return e == cudaSuccess ? IMG_OK : IMG_ECUDA; }

// With IMG_DEBUG set in the environment, a failing CUDA call is reported on
// stderr with its source line before the status code is returned.
void report_cuda(cudaError_t e, const char *what, int line) {
    static const bool on = getenv("IMG_DEBUG") != nullptr;
    if (on) fprintf(stderr, "img: %s failed at img_api.cu:%d: %s\n", what, line, cudaGetErrorString(e));
}

#define CK(x)                                        \
    do {                                             \
        cudaError_t _e = (x);                        \
        if (_e != cudaSuccess) {                     \
            report_cuda(_e, #x, __LINE__);           \
            return IMG_ECUDA;                        \
        }                                            \
    } while (0)

// NVTX range over one API call (a no-op unless a profiler is attached), so
// traces show set_covariance / factor+bounds / solve / operators per call.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

struct Carver {
    char *base;
    size_t off = 0;
    template <class T>
    T *take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T *p = reinterpret_cast<T *>(base ? base + off : nullptr);
        off += n * sizeof(T);
        return p;
    }
};

// Lay out every device array of one job; with base == nullptr only sizes.
size_t carve(img_ctx *c, char *base) {
    const int p = c->prm.p, nl = c->prm.n_l, nm = c->prm.n_m;
    const int Q = nl * nm;
    const int cap = c->hj.cap;
    Carver cv{base};
    JobDev &J = c->hj;
    J.ant = cv.take<double>(3 * (size_t)p);
    J.lg = cv.take<double>(nl);
    J.mg = cv.take<double>(nm);
    const size_t pp = (size_t)p * p;
    J.R64 = cv.take<double2>(pp);
    J.L64 = cv.take<double2>(pp);
    J.Li64 = cv.take<double2>(pp);
    J.R32 = cv.take<float2>(pp);
    J.Ri32 = cv.take<float2>(pp);
    J.Li32 = cv.take<float2>(pp);
    J.LiH32 = cv.take<float2>(pp);
    J.El = cv.take<float2>((size_t)nl * p);
    J.Em = cv.take<float2>((size_t)nm * p);
    J.dirty = cv.take<float>(Q);
    J.h = cv.take<float>(Q);
    J.scale = cv.take<float>(Q);
    J.eps = cv.take<float>(Q);
    J.grad = cv.take<float>(Q);
    J.upper = cv.take<double>(Q);
    J.gamma = cv.take<double>(Q);
    J.mvb = cv.take<double>(Q);
    J.x = cv.take<double>(Q);
    J.sigma = cv.take<double>(Q);
    J.set = cv.take<unsigned char>(Q);
    J.slot = cv.take<int>(Q);
    J.supp = cv.take<int>(cap);
    J.cvec = cv.take<float2>((size_t)cap * p);
    J.cmax = cv.take<float>(cap);
    J.fpos = cv.take<int>(cap);
    J.v = cv.take<float>(cap);
    J.w = cv.take<float>(cap);
    J.sF = cv.take<float>(cap);
    J.xs = cv.take<float>(2 * (size_t)cap);
    J.W0 = cv.take<float2>(pp);
    J.W1 = cv.take<float2>(pp);
    J.W2 = cv.take<float2>(pp);
    J.ev = cv.take<int>(J.ev_cap);
    J.evv = cv.take<float>(J.ev_cap);
    J.ev_count = cv.take<int>(1);
    J.Bimg = p <= img::kMaxWideP ? cv.take<unsigned char>(2 * img::wide_B_bytes(p)) : nullptr;
    J.Bscale = cv.take<float>(2);
    J.Bmax = cv.take<unsigned>(2);           // also the forward's max |w| word at every p
    J.info = cv.take<DevInfo>(1);
    J.flags = cv.take<int>(4);
    c->dj = cv.take<JobDev>(1);
    c->djp = cv.take<JobDev *>(1);
    c->wx = cv.take<float>(Q);
    c->part = cv.take<float2>((size_t)c->nparts * pp);
    c->U32 = cv.take<float2>(pp);
    c->Z = cv.take<double2>(pp);
    c->outd = cv.take<double>(Q);
    return cv.off + 256;
}

// Arithmetic of the solver for one context: tensor cores when requested and
// the 2p x 2p operand tiles fit in shared memory, CUDA cores otherwise.
int mode_of(const img_ctx *c) {
    return (c->prm.precision != IMG_PREC_FP32 && c->prm.p <= img::kMaxTcP) ? c->prm.precision : 0;
}

// Arithmetic of the stand-alone operators (dirty image, bounds, Psi, Psi^H):
// tensor cores up to p = 256.  Bounds stream their operand above p = 64;
// img_psi / img_psi_adj use the pipelined streamed kernels at every p.
int op_mode_of(const img_ctx *c) {
    return (c->prm.precision != IMG_PREC_FP32 && c->prm.p <= img::kMaxWideP) ? c->prm.precision : 0;
}

// Arithmetic of the stand-alone forward (img_psi): tensor-core Gram blocks up
// to p = 384, or 0 for CUDA cores.
int fwd_mode_of(const img_ctx *c) {
    return (c->prm.precision != IMG_PREC_FP32 && c->prm.p <= img::kMaxWideFwdP) ? c->prm.precision : 0;
}

// Arithmetic of the graph-driven wide solver (64 < p <= 384, tensor cores),
// or 0 when the job takes the one-CTA solver.
int wide_of(const img_ctx *c) {
    return (c->prm.precision != IMG_PREC_FP32 && c->prm.p > img::kMaxTcP && c->prm.p <= img::kMaxWideSolveP)
               ? c->prm.precision
               : 0;
}

// The wide solver's buffers and graph, made on the first wide solve of a
// context (the graph holds the context's device pointers, which never move).
img_status wide_ready(img_ctx *c) {
    if (c->ws) return IMG_OK;
    const cudaError_t e = img::ws_create(c->hj, c->dj, wide_of(c), &c->ws);
    if (e != cudaSuccess) report_cuda(e, "ws_create", __LINE__);
    if (e == cudaErrorMemoryAllocation) return IMG_ENOMEM;
    return e == cudaSuccess ? IMG_OK : IMG_ECUDA;
}

// Dirty image and MVDR denominators on the work-item tensor-core adjoint of
// the wide solver (tensor-core jobs with 256 < p <= 384, where the streamed
// operator of tc_wide.cuh does not reach).
bool items_bounds(const img_ctx *c) { return wide_of(c) != 0 && c->prm.p > img::kMaxWideP; }

bool finite_all(const double *v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

img_status sync(img_ctx *c) { return cuda_status(cudaStreamSynchronize(c->stream)); }

// Factor, dirty image, bounds (once per covariance).
img_status prepare(img_ctx *c) {
    const Range range_("img.prepare");
    if (!c->has_cov) return IMG_EINVAL;
    if (c->prepared) return (img_status)c->prep_status;
    CK(img::launch_factor(c->djp, 1, c->stream));
    if (items_bounds(c)) {
        img_status st = wide_ready(c);
        if (st != IMG_OK) return st;
        CK(img::ws_bounds(c->ws, c->hj, c->stream));
    } else {
        const int ntiles = (c->hj.Q + img::kTile - 1) / img::kTile;
        CK(img::launch_bounds(c->djp, 1, ntiles, c->prm.p, op_mode_of(c), c->stream));
    }
    CK(img::launch_finalize(c->djp, 1, c->stream, nullptr));
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, c->hj.flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->prepared = true;
    c->prep_status = flag == 0 ? IMG_OK : IMG_ENOTPD;
    return (img_status)c->prep_status;
}

img_status copy_out_double(img_ctx *c, const double *src, double *dst, size_t n, int on_device) {
    CK(cudaMemcpyAsync(dst, src, n * sizeof(double),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
}

img_status copy_out_float(img_ctx *c, const float *src, double *dst, size_t n, int on_device) {
    if (on_device) {
        CK(img::launch_to_double(src, dst, (int)n, c->stream));
        return sync(c);
    }
    CK(img::launch_to_double(src, c->outd, (int)n, c->stream));
    return copy_out_double(c, c->outd, dst, n, 0);
}

// Batch workspace shared by img_solve_batch calls (grown on demand).
struct BatchWs {
    std::mutex mu;
    int cap = 0;
    int device = -1;
    JobDev **jobs = nullptr;
    DevInfo *infos = nullptr;
    double **sig = nullptr;
    int *status = nullptr;
};
BatchWs g_ws;

img_status ws_reserve(int n, int device) {
    if (g_ws.cap >= n && g_ws.device == device) return IMG_OK;
    if (g_ws.jobs) {
        cudaFree(g_ws.jobs);
        g_ws.jobs = nullptr;
    }
    int cap = 64;
    while (cap < n) cap *= 2;
    size_t bytes = cap * (sizeof(JobDev *) + sizeof(DevInfo) + sizeof(double *) + sizeof(int)) + 1024;
    char *b = nullptr;
    CK(cudaMalloc(&b, bytes));
    g_ws.jobs = reinterpret_cast<JobDev **>(b);
    g_ws.sig = reinterpret_cast<double **>(b + cap * sizeof(JobDev *));
    g_ws.infos = reinterpret_cast<DevInfo *>(
        b + ((cap * (sizeof(JobDev *) + sizeof(double *)) + 255) & ~size_t(255)));
    g_ws.status = reinterpret_cast<int *>(reinterpret_cast<char *>(g_ws.infos) + cap * sizeof(DevInfo));
    g_ws.cap = cap;
    g_ws.device = device;
    return IMG_OK;
}

void fill_info(img_solve_info *o, const DevInfo &d) {
    o->status = d.status;
    o->outer = d.outer;
    o->lsqr_iters = d.lsqr_iters;
    o->n_free = d.n_free;
    o->n_upper = d.n_upper;
    o->converged = d.converged;
    o->lambda_min = d.lambda_min;
    o->op_flops = d.op_flops;
    o->cyc_total = d.cyc_total;
    o->cyc_gradient = d.cyc_gradient;
    o->cyc_lsqr = d.cyc_lsqr;
    o->cyc_lsqr_fwd = d.cyc_lsqr_fwd;
    o->cyc_lsqr_adj = d.cyc_lsqr_adj;
    for (int k = 0; k < 6; ++k) o->cyc_aux[k] = d.cyc_aux[k];
    o->t_begin_ns = (double)d.t_begin_ns;
    o->t_end_ns = (double)d.t_end_ns;
}

}  // namespace

extern "C" {

void img_params_default(img_params *prm) {
    if (!prm) return;
    std::memset(prm, 0, sizeof(*prm));
    prm->lambda = 1.0;
    prm->cost = IMG_COST_PWLS;
    prm->bound = IMG_BOUND_MVDR;
    prm->bias_c = 0;
    prm->inflate = IMG_INFLATE_NONE;
    prm->alpha = 6.0;
    prm->kappa = 6.0;
    prm->eps_floor = 1e-6;
    prm->lsqr_atol = 1e-6;
    prm->lsqr_btol = 1e-6;
    prm->feas_tol = 1e-5;
    prm->precision = IMG_PREC_FP32;
}

const char *img_status_str(img_status s) {
    switch (s) {
        case IMG_OK: return "ok";
        case IMG_EINVAL: return "invalid argument or call order";
        case IMG_ENOMEM: return "out of memory or capacity";
        case IMG_ENOTPD: return "covariance not positive definite";
        case IMG_ENOTCONV: return "active-set loop did not converge";
        case IMG_ETIMEOUT: return "device wait timed out";
        case IMG_ECUDA: return "CUDA error";
    }
    return "unknown status";
}

img_status img_create(const img_params *prm, img_ctx **out) {
    if (!out) return IMG_EINVAL;
    *out = nullptr;
    if (!prm) return IMG_EINVAL;
    const img_params &P = *prm;
    if (P.p < 2 || P.p > kMaxP || P.n_l < 1 || P.n_m < 1) return IMG_EINVAL;
    if ((long long)P.n_l * P.n_m > (1LL << 24)) return IMG_EINVAL;
    if (!P.ant_xyz || !P.l || !P.m) return IMG_EINVAL;
    if (!(P.lambda > 0.0) || !std::isfinite(P.lambda)) return IMG_EINVAL;
    if (P.cost != IMG_COST_LS && P.cost != IMG_COST_PWLS) return IMG_EINVAL;
    if (P.bound != IMG_BOUND_MF && P.bound != IMG_BOUND_MVDR) return IMG_EINVAL;
    if (P.inflate < IMG_INFLATE_NONE || P.inflate > IMG_INFLATE_STD) return IMG_EINVAL;
    if (P.precision < IMG_PREC_FP32 || P.precision > IMG_PREC_BF16X3) return IMG_EINVAL;
    if (!(P.kappa >= 0.0) || !(P.eps_floor >= 0.0) || !(P.alpha >= 0.0)) return IMG_EINVAL;
    if (!(P.lsqr_atol >= 0.0) || !(P.lsqr_btol >= 0.0) || P.lsqr_maxit < 0 || P.max_outer < 0)
        return IMG_EINVAL;
    if (!(P.feas_tol >= 0.0) || !(P.feas_tol < 1.0)) return IMG_EINVAL;
    if (P.support_cap < 0) return IMG_EINVAL;
    if (!finite_all(P.ant_xyz, 3 * (size_t)P.p) || !finite_all(P.l, P.n_l) || !finite_all(P.m, P.n_m))
        return IMG_EINVAL;
    for (int k = 0; k < P.p; ++k)
        if (P.ant_xyz[3 * k + 2] != 0.0) return IMG_EINVAL;

    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return IMG_ECUDA;
    img_ctx *c = new (std::nothrow) img_ctx();
    if (!c) return IMG_ENOMEM;
    c->prm = P;
    c->ant.assign(P.ant_xyz, P.ant_xyz + 3 * P.p);
    c->l.assign(P.l, P.l + P.n_l);
    c->m.assign(P.m, P.m + P.n_m);
    c->prm.ant_xyz = c->ant.data();
    c->prm.l = c->l.data();
    c->prm.m = c->m.data();
    cudaGetDevice(&c->device);
    if (P.stream) {
        c->stream = (cudaStream_t)P.stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return IMG_ECUDA;
        }
        c->own_stream = true;
    }
    const int Q = P.n_l * P.n_m;
    JobDev &J = c->hj;
    J.p = P.p;
    J.n_l = P.n_l;
    J.n_m = P.n_m;
    J.Q = Q;
    J.cost = P.cost;
    J.bound = P.bound;
    J.bias_c = P.bias_c ? 1 : 0;
    J.inflate = P.inflate;
    J.lsqr_maxit = P.lsqr_maxit;
    J.max_outer = P.max_outer;
    J.cap = P.support_cap > 0 ? std::min(P.support_cap, Q) : std::min(Q, 16384);
    J.ev_cap = (int)std::min<long long>(P.max_outer > 0 ? P.max_outer : 10LL * Q + 100, 1 << 20);
    J.precision = P.precision;
    J.alpha = P.alpha;
    J.kappa = P.kappa;
    J.eps_floor = P.eps_floor;
    J.lam = P.lambda;
    J.lsqr_atol = P.lsqr_atol;
    J.lsqr_btol = P.lsqr_btol;
    J.feas_tol = P.feas_tol;
    J.N = 0;
    {
        int sms = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        const size_t pp8 = (size_t)P.p * P.p * sizeof(float2);
        int np = 2 * std::max(1, sms);
        const int lim = (int)std::max<size_t>(1, (4u << 20) / pp8);
        c->nparts = std::max(1, std::min(np, lim));
    }
    c->dbytes = carve(c, nullptr);
    if (cudaMalloc(&c->dmem, c->dbytes) != cudaSuccess) {
        if (c->own_stream) cudaStreamDestroy(c->stream);
        delete c;
        return IMG_ENOMEM;
    }
    carve(c, reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(c->dmem) + 255) & ~uintptr_t(255)));
    img_status st = IMG_OK;
    int init_flags[4] = {-1, 0, 0, 0};
    if (cudaMemcpyAsync((void *)J.ant, c->ant.data(), 3 * P.p * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync((void *)J.lg, c->l.data(), P.n_l * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync((void *)J.mg, c->m.data(), P.n_m * sizeof(double), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(J.flags, init_flags, sizeof(init_flags), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->dj, &J, sizeof(JobDev), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->djp, &c->dj, sizeof(JobDev *), cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        img::launch_tables(c->djp, 1, c->stream) != cudaSuccess ||
        cudaStreamSynchronize(c->stream) != cudaSuccess)
        st = IMG_ECUDA;
    if (st != IMG_OK) {
        img_destroy(c);
        return st;
    }
    *out = c;
    return IMG_OK;
}

img_status img_set_covariance(img_ctx *c, const void *R, int dtype, long long N, int on_device) {
    const Range range_("img.set_covariance");
    if (!c || !R) return IMG_EINVAL;
    if (dtype != IMG_C64 && dtype != IMG_C128) return IMG_EINVAL;
    const int p = c->prm.p;
    if (N <= p) return IMG_EINVAL;
    const size_t pp = (size_t)p * p;
    c->has_cov = false;
    c->prepared = false;
    c->solved = false;
    if (!on_device) {
        std::vector<double> z(2 * pp);
        if (dtype == IMG_C128) {
            std::memcpy(z.data(), R, 2 * pp * sizeof(double));
        } else {
            const float *f = static_cast<const float *>(R);
            for (size_t e = 0; e < 2 * pp; ++e) z[e] = f[e];
        }
        if (!finite_all(z.data(), z.size())) return IMG_EINVAL;
        double mx = 0.0;
        for (double v : z) mx = std::max(mx, std::fabs(v));
        for (int k = 0; k < p; ++k) {
            if (!(z[2 * ((size_t)k * p + k)] > 0.0)) return IMG_EINVAL;
            for (int l = 0; l < p; ++l) {
                const double *a = &z[2 * ((size_t)l * p + k)];
                const double *b = &z[2 * ((size_t)k * p + l)];
                if (std::fabs(a[0] - b[0]) > 1e-6 * mx || std::fabs(a[1] + b[1]) > 1e-6 * mx)
                    return IMG_EINVAL;
            }
        }
        CK(cudaMemcpyAsync(c->hj.R64, z.data(), 2 * pp * sizeof(double), cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        if (dtype == IMG_C128) {
            CK(cudaMemcpyAsync(c->hj.R64, R, pp * sizeof(double2), cudaMemcpyDeviceToDevice, c->stream));
        } else {
            CK(img::launch_c2z(static_cast<const float2 *>(R), c->hj.R64, (int)pp, c->stream));
        }
    }
    // N and the cleared factor/bounds flags; pageable sources are staged by
    // the runtime before cudaMemcpyAsync returns, so locals are safe here.
    c->hj.N = N;
    CK(cudaMemcpyAsync(&c->dj->N, &c->hj.N, sizeof(long long), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->hj.flags, 0xff, sizeof(int), c->stream));
    CK(cudaMemsetAsync(c->hj.flags + 1, 0, sizeof(int), c->stream));
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    c->has_cov = true;
    return IMG_OK;
}

img_status img_dirty(img_ctx *c, double *out, int on_device) {
    const Range range_("img.dirty");
    if (!c || !out) return IMG_EINVAL;
    img_status st = prepare(c);
    if (st != IMG_OK) return st;
    return copy_out_float(c, c->hj.dirty, out, c->hj.Q, on_device);
}

img_status img_mvdr_bound(img_ctx *c, double *out, int on_device) {
    const Range range_("img.mvdr_bound");
    if (!c || !out) return IMG_EINVAL;
    img_status st = prepare(c);
    if (st != IMG_OK) return st;
    return copy_out_double(c, c->hj.mvb, out, c->hj.Q, on_device);
}

img_status img_solve(img_ctx *c, double *sigma, img_solve_info *info, int on_device) {
    const Range range_("img.solve");
    if (!c || !sigma) return IMG_EINVAL;
    img_status st = prepare(c);
    if (st != IMG_OK) return st;
    if (wide_of(c)) {
        st = wide_ready(c);
        if (st != IMG_OK) return st;
        CK(img::ws_launch(c->ws, c->stream));
    } else {
        CK(img::launch_solve(c->djp, 1, c->prm.p, mode_of(c), nullptr, nullptr, c->stream));
    }
    DevInfo d{};
    CK(cudaMemcpyAsync(&d, c->hj.info, sizeof(DevInfo), cudaMemcpyDeviceToHost, c->stream));
    st = copy_out_double(c, c->hj.sigma, sigma, c->hj.Q, on_device);
    if (st != IMG_OK) return st;
    if (info) fill_info(info, d);
    c->solved = true;
    return (img_status)d.status;
}

img_status img_get_sets(img_ctx *c, unsigned char *sets) {
    if (!c || !sets || !c->solved) return IMG_EINVAL;
    CK(cudaMemcpyAsync(sets, c->hj.set, c->hj.Q, cudaMemcpyDeviceToHost, c->stream));
    return sync(c);
}

img_status img_get_gradient(img_ctx *c, double *grad) {
    if (!c || !grad || !c->solved) return IMG_EINVAL;
    return copy_out_float(c, c->hj.grad, grad, c->hj.Q, 0);
}

img_status img_get_events(img_ctx *c, int *events, double *values, int capacity, int *count) {
    if (!c || !count || capacity < 0 || !c->solved) return IMG_EINVAL;
    int n = 0;
    CK(cudaMemcpyAsync(&n, c->hj.ev_count, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *count = n;
    const int m = std::min(std::min(n, capacity), c->hj.ev_cap);
    if (m > 0 && events)
        CK(cudaMemcpyAsync(events, c->hj.ev, m * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if (m > 0 && values) {
        std::vector<float> v(m);
        CK(cudaMemcpyAsync(v.data(), c->hj.evv, m * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (int k = 0; k < m; ++k) values[k] = v[k];
    }
    return sync(c);
}

img_status img_psi(img_ctx *c, const double *x, double *Kout, int on_device) {
    const Range range_("img.psi");
    if (!c || !x || !Kout) return IMG_EINVAL;
    const int Q = c->hj.Q, p = c->prm.p;
    if (on_device) {
        CK(img::launch_d2f(x, c->wx, Q, c->stream));
    } else {
        std::vector<float> f(Q);
        for (int i = 0; i < Q; ++i) f[i] = (float)x[i];
        CK(cudaMemcpyAsync(c->wx, f.data(), Q * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    const int om = fwd_mode_of(c);
    if (om != 0) {
        // tensor-core Gram blocks; their partial sums need a scratch buffer
        if (!c->fwd_part) {
            int sms = 1;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
            CK(cudaMalloc(&c->fwd_part, img::psi_wide_part_floats(sms) * sizeof(float)));
        }
        CK(img::launch_psi_wide(c->dj, c->hj.Bmax + 1, c->wx, c->fwd_part, Q, p, c->prm.n_l, c->prm.n_m, om, c->Z,
                                c->stream));
    } else {
        CK(img::launch_psi(c->dj, c->wx, c->part, c->nparts, Q, p, mode_of(c), c->Z, c->stream));
    }
    CK(cudaMemcpyAsync(Kout, c->Z, (size_t)p * p * sizeof(double2),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    if (on_device == 2) return IMG_OK;           // stream-ordered, no host wait
    return sync(c);
}

img_status img_psi_adj(img_ctx *c, const double *U, double *out, int on_device) {
    const Range range_("img.psi_adj");
    if (!c || !U || !out) return IMG_EINVAL;
    const int Q = c->hj.Q, p = c->prm.p;
    const int om = op_mode_of(c);
    if (om != 0) {
        // streamed tensor-core operator: its operand image is built from the
        // complex128 U directly (the caller's device buffer, or a staged copy)
        const double2 *Ud = reinterpret_cast<const double2 *>(U);
        if (!on_device) {
            CK(cudaMemcpyAsync(c->Z, U, (size_t)p * p * sizeof(double2), cudaMemcpyHostToDevice, c->stream));
            Ud = c->Z;
        }
        CK(img::launch_psi_adj_wide(c->dj, c->hj.Bmax, Ud, true, on_device ? out : c->outd, Q, p, om,
                                    c->stream));
        if (on_device == 2) return IMG_OK;
        if (on_device) return sync(c);
        return copy_out_double(c, c->outd, out, Q, 0);
    }
    CK(cudaMemcpyAsync(c->Z, U, (size_t)p * p * sizeof(double2),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream));
    CK(img::launch_z2c(c->Z, c->U32, p * p, c->stream));
    if (items_bounds(c)) {
        // 256 < p <= 384 on tensor cores: the solver's work-item adjoint
        img_status st = wide_ready(c);
        if (st != IMG_OK) return st;
        CK(img::ws_psi_adj(c->ws, c->hj, c->U32, on_device ? out : c->outd, c->stream));
    } else {
        CK(img::launch_psi_adj(c->dj, c->U32, on_device ? out : c->outd, Q, p, op_mode_of(c), c->stream));
    }
    if (on_device == 2) return IMG_OK;           // stream-ordered, no host wait
    if (on_device) return sync(c);
    return copy_out_double(c, c->outd, out, Q, 0);
}

}  // extern "C"

namespace {

// The snapshot entry points take one context per snapshot: all hold a
// covariance and agree on device, p, grid, wavelength, N and bias constant.
img_status check_snapshots(img_ctx *const *snap, int K) {
    if (!snap || K < 1 || K > IMG_MAX_SNAPSHOTS) return IMG_EINVAL;
    for (int k = 0; k < K; ++k)
        if (!snap[k] || !snap[k]->has_cov) return IMG_EINVAL;
    const img_ctx *c0 = snap[0];
    for (int k = 1; k < K; ++k) {
        const img_ctx *c = snap[k];
        if (c->device != c0->device || c->prm.p != c0->prm.p || c->prm.n_l != c0->prm.n_l ||
            c->prm.n_m != c0->prm.n_m || c->prm.lambda != c0->prm.lambda ||
            c->prm.bias_c != c0->prm.bias_c || c->hj.N != c0->hj.N || c->l != c0->l || c->m != c0->m)
            return IMG_EINVAL;
    }
    return IMG_OK;
}

// Device allocation freed on scope exit (every return path).
struct DevBuf {
    void *ptr = nullptr;
    ~DevBuf() {
        if (ptr) cudaFree(ptr);
    }
};

}  // namespace

extern "C" {

img_status img_snapshot_image(img_ctx *const *snap, int K, int kind, double *out, int on_device) {
    const Range range_("img.snapshot_image");
    if (!out) return IMG_EINVAL;
    if (kind != IMG_SNAP_MF && kind != IMG_SNAP_MVDR && kind != IMG_SNAP_ASSC) return IMG_EINVAL;
    const img_status chk = check_snapshots(snap, K);
    if (chk != IMG_OK) return chk;
    img_ctx *c0 = snap[0];
    for (int k = 0; k < K; ++k) {
        const img_status st = prepare(snap[k]);     // synchronises snapshot k's stream
        if (st != IMG_OK) return st;
    }
    img::SnapPtrs sp{};
    for (int k = 0; k < K; ++k) {
        sp.d[k] = snap[k]->hj.dirty;
        sp.h[k] = snap[k]->hj.h;
    }
    const long long N = c0->hj.N;
    const int p = c0->prm.p;
    const double C = c0->prm.bias_c ? (double)N / (double)(N - p) : 1.0;
    const int Q = c0->hj.Q;
    CK(img::launch_snapshot_image(sp, K, Q, kind, C, on_device ? out : c0->outd, c0->stream));
    if (on_device) return sync(c0);
    return copy_out_double(c0, c0->outd, out, Q, 0);
}

img_status img_snapshot_ls_image(img_ctx *const *snap, int K, int maxit, double *sigma, img_solve_info *info,
                                 int on_device) {
    const Range range_("img.snapshot_ls_image");
    if (!sigma) return IMG_EINVAL;
    img_status st = check_snapshots(snap, K);
    if (st != IMG_OK) return st;
    img_ctx *c0 = snap[0];
    for (int k = 1; k < K; ++k)
        if (snap[k]->prm.cost != c0->prm.cost) return IMG_EINVAL;
    for (int k = 0; k < K; ++k) {
        st = prepare(snap[k]);
        if (st != IMG_OK) return st;
        if (op_mode_of(snap[k]) != 0 && !snap[k]->fwd_part) {
            int sms = 1;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, snap[k]->device);
            CK(cudaMalloc(&snap[k]->fwd_part, img::psi_wide_part_floats(sms) * sizeof(float)));
        }
    }
    const int Q = c0->hj.Q, p = c0->prm.p, pp = p * p;
    // K blocks of u and M v, shared p x p scratch, Q-vectors v, w, x, wx and
    // the K-snapshot scale, y / yk / sigma staging, scalars: one allocation
    // for the call
    auto al = [](size_t n) { return (n + 255) / 256 * 256; };
    const size_t need = 2 * al((size_t)K * pp * sizeof(float2)) + 2 * al((size_t)pp * sizeof(float2)) +
                        al((size_t)pp * sizeof(double2)) + 5 * al((size_t)Q * sizeof(float)) +
                        3 * al((size_t)Q * sizeof(double)) + al(img::kLsScalars * sizeof(double));
    DevBuf mem;
    CK(cudaMalloc(&mem.ptr, need));
    char *m = static_cast<char *>(mem.ptr);
    auto take = [&](size_t n) {
        char *r = m;
        m += al(n);
        return r;
    };
    img::LsBufs b;
    b.u = reinterpret_cast<float2 *>(take((size_t)K * pp * sizeof(float2)));
    b.Mv = reinterpret_cast<float2 *>(take((size_t)K * pp * sizeof(float2)));
    b.T1 = reinterpret_cast<float2 *>(take((size_t)pp * sizeof(float2)));
    b.Uw = reinterpret_cast<float2 *>(take((size_t)pp * sizeof(float2)));
    b.Kd = reinterpret_cast<double2 *>(take((size_t)pp * sizeof(double2)));
    b.v = reinterpret_cast<float *>(take((size_t)Q * sizeof(float)));
    b.w = reinterpret_cast<float *>(take((size_t)Q * sizeof(float)));
    b.x = reinterpret_cast<float *>(take((size_t)Q * sizeof(float)));
    b.wx = reinterpret_cast<float *>(take((size_t)Q * sizeof(float)));
    float *scale = reinterpret_cast<float *>(take((size_t)Q * sizeof(float)));
    b.y = reinterpret_cast<double *>(take((size_t)Q * sizeof(double)));
    double *yk = reinterpret_cast<double *>(take((size_t)Q * sizeof(double)));
    double *sig = reinterpret_cast<double *>(take((size_t)Q * sizeof(double)));
    b.sc = reinterpret_cast<double *>(take(img::kLsScalars * sizeof(double)));

    img::SnapPtrs sp{};
    img::LsSnap s;
    s.K = K;
    s.yk = yk;
    for (int k = 0; k < K; ++k) {
        sp.d[k] = snap[k]->hj.dirty;
        sp.h[k] = snap[k]->hj.h;
        s.jd[k] = snap[k]->dj;
        s.hj[k] = snap[k]->hj;
        s.hj[k].scale = scale;
        s.mode[k] = op_mode_of(snap[k]);
        s.fwd_part[k] = snap[k]->fwd_part;
        s.part[k] = snap[k]->part;
        s.nparts[k] = snap[k]->nparts;
    }
    const long long N = c0->hj.N;
    const double C = c0->prm.bias_c ? (double)N / (double)(N - p) : 1.0;
    cudaStream_t stream = c0->stream;
    const auto t0 = std::chrono::steady_clock::now();
    CK(img::launch_snap_scale(sp, K, Q, c0->prm.cost == IMG_COST_PWLS, C, scale, stream));
    CK(img::ls_snap_begin(s, b, stream));
    const int lim = maxit > 0 ? maxit : 200;
    const double atol = c0->prm.lsqr_atol, btol = c0->prm.lsqr_btol;
    int it = 0, istop = 3;
    double h[img::kLsScalars] = {};
    for (it = 1; it <= lim; ++it) {
        CK(img::ls_snap_iterate(s, b, stream));
        if (it % 10 == 0 || it == lim) {
            // Paige-Saunders stopping tests on the host, every 10 iterations
            CK(img::ls_xnorm2(s.hj[0], b, b.sc + img::kLsXnorm2, stream));
            CK(cudaMemcpyAsync(h, b.sc, sizeof(h), cudaMemcpyDeviceToHost, stream));
            CK(cudaStreamSynchronize(stream));
            const double anorm = std::sqrt(h[img::kLsAnorm2]), xnorm = std::sqrt(h[img::kLsXnorm2]);
            if (h[img::kLsRnorm] <= btol * h[img::kLsBnorm] + atol * anorm * xnorm) {
                istop = 1;
                break;
            }
            if (h[img::kLsArnorm] <= atol * anorm * h[img::kLsRnorm]) {
                istop = 2;
                break;
            }
        }
    }
    if (it > lim) it = lim;
    CK(img::ls_finish(s.hj[0], b, on_device ? sigma : sig, nullptr, stream));
    if (!on_device) CK(cudaMemcpyAsync(sigma, sig, (size_t)Q * sizeof(double), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->status = IMG_OK;
        info->lsqr_iters = it;
        info->n_free = Q;
        info->converged = istop < 3 ? 1 : 0;
        info->lambda_min = h[img::kLsRnorm];
        info->op_flops = ((double)(it + 1) * 8.0 * pp * Q + (double)it * 4.0 * pp * Q) * K;
        info->t_end_ns = secs * 1e9;
    }
    return IMG_OK;
}

img_status img_check_wait(unsigned polls, int arrive) {
    if (polls == 0 || polls > (1u << 26)) return IMG_EINVAL;
    int *d = nullptr;
    CK(cudaMalloc(&d, sizeof(int)));
    int h = -1;
    cudaError_t e = img::launch_wait_selftest(polls, arrive ? 1 : 0, d, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return IMG_ECUDA;
    return h == IMG_OK ? IMG_OK : IMG_ETIMEOUT;
}

img_status img_ls_image(img_ctx *c, int maxit, double *sigma, img_solve_info *info, int on_device) {
    const Range range_("img.ls_image");
    if (!c || !sigma || !c->has_cov) return IMG_EINVAL;
    img_status st = prepare(c);
    if (st != IMG_OK) return st;
    const int Q = c->hj.Q, p = c->prm.p, pp = p * p;
    const int mode = op_mode_of(c);
    // vectors: u, Mv, T1, Uw (p^2 float2), Kd (p^2 double2), v, w, x, wx (Q
    // floats), y and sigma staging (Q doubles), scalars
    auto al = [](size_t n) { return (n + 255) / 256 * 256; };
    const size_t need = 4 * al((size_t)pp * sizeof(float2)) + al((size_t)pp * sizeof(double2)) +
                        4 * al((size_t)Q * sizeof(float)) + 2 * al((size_t)Q * sizeof(double)) +
                        al(img::kLsScalars * sizeof(double));
    if (!c->ls_mem) CK(cudaMalloc(&c->ls_mem, need));
    if (mode != 0 && !c->fwd_part) {
        int sms = 1;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        CK(cudaMalloc(&c->fwd_part, img::psi_wide_part_floats(sms) * sizeof(float)));
    }
    char *m = static_cast<char *>(c->ls_mem);
    auto take = [&](size_t n) {
        char *r = m;
        m += al(n);
        return r;
    };
    img::LsBufs b;
    b.u = reinterpret_cast<float2 *>(take((size_t)pp * sizeof(float2)));
    b.Mv = reinterpret_cast<float2 *>(take((size_t)pp * sizeof(float2)));
    b.T1 = reinterpret_cast<float2 *>(take((size_t)pp * sizeof(float2)));
    b.Uw = reinterpret_cast<float2 *>(take((size_t)pp * sizeof(float2)));
    b.Kd = reinterpret_cast<double2 *>(take((size_t)pp * sizeof(double2)));
    b.v = reinterpret_cast<float *>(take((size_t)Q * sizeof(float)));
    b.w = reinterpret_cast<float *>(take((size_t)Q * sizeof(float)));
    b.x = reinterpret_cast<float *>(take((size_t)Q * sizeof(float)));
    b.wx = reinterpret_cast<float *>(take((size_t)Q * sizeof(float)));
    b.y = reinterpret_cast<double *>(take((size_t)Q * sizeof(double)));
    double *sig = reinterpret_cast<double *>(take((size_t)Q * sizeof(double)));
    b.sc = reinterpret_cast<double *>(take(img::kLsScalars * sizeof(double)));
    const auto t0 = std::chrono::steady_clock::now();
    CK(img::ls_begin(c->dj, c->hj, b, mode, c->stream));
    const int lim = maxit > 0 ? maxit : 200;
    const double atol = c->prm.lsqr_atol, btol = c->prm.lsqr_btol;
    int it = 0, istop = 3;
    double h[img::kLsScalars] = {};
    for (it = 1; it <= lim; ++it) {
        if (c->ls_exec) {
            CK(cudaGraphLaunch(c->ls_exec, c->stream));
        } else {
            CK(img::ls_iterate(c->dj, c->hj, b, mode, c->fwd_part, c->part, c->nparts, c->stream));
            if (c->own_stream) {
                // the iteration is a fixed sequence of ~15 launches on buffers the
                // context keeps: record it once as a graph and replay it (the
                // first, direct iteration has set every kernel attribute)
                cudaGraph_t g = nullptr;
                if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                    const cudaError_t e1 =
                        img::ls_iterate(c->dj, c->hj, b, mode, c->fwd_part, c->part, c->nparts, c->stream);
                    const cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);
                    if (e1 == cudaSuccess && e2 == cudaSuccess && g) {
                        if (cudaGraphInstantiate(&c->ls_exec, g, 0) != cudaSuccess) c->ls_exec = nullptr;
                    }
                    if (g) cudaGraphDestroy(g);
                }
                cudaGetLastError();      // a failed capture leaves direct launches in place
            }
        }
        if (it % 10 == 0 || it == lim) {
            // Paige-Saunders stopping tests on the host, every 10 iterations
            CK(img::ls_xnorm2(c->hj, b, b.sc + img::kLsXnorm2, c->stream));
            CK(cudaMemcpyAsync(h, b.sc, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
            CK(cudaStreamSynchronize(c->stream));
            const double anorm = std::sqrt(h[img::kLsAnorm2]), xnorm = std::sqrt(h[img::kLsXnorm2]);
            if (h[img::kLsRnorm] <= btol * h[img::kLsBnorm] + atol * anorm * xnorm) {
                istop = 1;
                break;
            }
            if (h[img::kLsArnorm] <= atol * anorm * h[img::kLsRnorm]) {
                istop = 2;
                break;
            }
        }
    }
    if (it > lim) it = lim;
    CK(img::ls_finish(c->hj, b, on_device ? sigma : sig, nullptr, c->stream));
    if (!on_device) CK(cudaMemcpyAsync(sigma, sig, (size_t)Q * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) {
        std::memset(info, 0, sizeof(*info));
        info->status = IMG_OK;
        info->outer = 0;
        info->lsqr_iters = it;
        info->n_free = Q;
        info->converged = istop < 3 ? 1 : 0;
        info->lambda_min = h[img::kLsRnorm];
        info->op_flops = (double)(it + 1) * 8.0 * pp * Q + (double)it * 4.0 * pp * Q;
        info->t_begin_ns = 0.0;
        info->t_end_ns = secs * 1e9;
    }
    return IMG_OK;
}

}  // extern "C"

namespace {

// Jobs of a batch grouped by operator arithmetic (one launch per group):
// order[] lists job indices group by group; groups[k] = [begin, end).
// Keys 0..2: solver and bounds in arithmetic k (FP32, F16X3, BF16X3, the
// latter two for p <= 64); keys 3, 4: bounds on the streamed tensor-core
// operator in F16X3 / BF16X3 (64 < p <= 256), solver on CUDA cores.
// Key 5: tensor-core jobs with 256 < p <= 384, whose bounds run on the
// work-item adjoint one job at a time (and whose solve is a graph).
constexpr int kGroups = 6;
constexpr int kItemsGroup = 5;
struct Groups {
    std::vector<int> order;
    int begin[kGroups] = {}, end[kGroups] = {};
    int max_p[kGroups] = {}, max_tiles[kGroups] = {1, 1, 1, 1, 1, 1};
    static int solve_mode(int k) { return k <= 2 ? k : 0; }
    static int bounds_mode(int k) { return k <= 2 ? k : (k <= 4 ? k - 2 : 0); }
};

int group_key(const img_ctx *c) {
    if (items_bounds(c)) return kItemsGroup;
    const int m = mode_of(c), om = op_mode_of(c);
    return (m == 0 && om != 0) ? om + 2 : m;
}

Groups group_by_mode(img_ctx *const *ctxs, int n) {
    Groups g;
    for (int m = 0; m < kGroups; ++m) {
        g.begin[m] = (int)g.order.size();
        for (int j = 0; j < n; ++j) {
            if (group_key(ctxs[j]) != m) continue;
            g.order.push_back(j);
            g.max_p[m] = std::max(g.max_p[m], ctxs[j]->prm.p);
            g.max_tiles[m] = std::max(g.max_tiles[m], (ctxs[j]->hj.Q + img::kTile - 1) / img::kTile);
        }
        g.end[m] = (int)g.order.size();
    }
    return g;
}

img_status check_batch(img_ctx *const *ctxs, int n) {
    if (!ctxs || n <= 0) return IMG_EINVAL;
    for (int j = 0; j < n; ++j) {
        if (!ctxs[j] || !ctxs[j]->has_cov) return IMG_EINVAL;
        if (ctxs[j]->device != ctxs[0]->device) return IMG_EINVAL;
    }
    return IMG_OK;
}

// Factor + bounds of the listed jobs (device pointer array already in
// g_ws.jobs in group order), one launch per kernel and group; the bounds of
// the work-item group run job by job.
img_status launch_prepare(img_ctx *const *ctxs, const Groups &g, cudaStream_t s, int *status_out) {
    for (int m = 0; m < kGroups; ++m) {
        const int nb = g.end[m] - g.begin[m];
        if (!nb) continue;
        JobDev *const *jp = g_ws.jobs + g.begin[m];
        CK(img::launch_factor(jp, nb, s));
        if (m == kItemsGroup) {
            for (int q = g.begin[m]; q < g.end[m]; ++q) {
                img_ctx *c = ctxs[g.order[q]];
                img_status st = wide_ready(c);
                if (st != IMG_OK) return st;
                CK(img::ws_bounds(c->ws, c->hj, s));
            }
        } else {
            CK(img::launch_bounds(jp, nb, g.max_tiles[m], g.max_p[m], Groups::bounds_mode(m), s));
        }
        CK(img::launch_finalize(jp, nb, s, status_out ? status_out + g.begin[m] : nullptr));
    }
    return IMG_OK;
}

}  // namespace

extern "C" {

img_status img_prepare_batch(img_ctx *const *ctxs, int n) {
    const Range range_("img.prepare_batch");
    img_status st = check_batch(ctxs, n);
    if (st != IMG_OK) return st;
    std::lock_guard<std::mutex> lock(g_ws.mu);
    st = ws_reserve(n, ctxs[0]->device);
    if (st != IMG_OK) return st;
    cudaStream_t s = ctxs[0]->stream;
    for (int j = 0; j < n; ++j)
        if (ctxs[j]->stream != s) CK(cudaStreamSynchronize(ctxs[j]->stream));
    const Groups g = group_by_mode(ctxs, n);
    std::vector<JobDev *> ptrs(n);
    for (int q = 0; q < n; ++q) ptrs[q] = ctxs[g.order[q]]->dj;
    CK(cudaMemcpyAsync(g_ws.jobs, ptrs.data(), n * sizeof(JobDev *), cudaMemcpyHostToDevice, s));
    st = launch_prepare(ctxs, g, s, g_ws.status);
    if (st != IMG_OK) return st;
    std::vector<int> flags(n);
    CK(cudaMemcpyAsync(flags.data(), g_ws.status, n * sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    img_status first = IMG_OK;
    for (int q = 0; q < n; ++q) {
        img_ctx *c = ctxs[g.order[q]];
        c->prepared = true;
        c->prep_status = flags[q] == 0 ? IMG_OK : IMG_ENOTPD;
    }
    for (int j = 0; j < n; ++j)
        if (first == IMG_OK && ctxs[j]->prep_status != IMG_OK) first = (img_status)ctxs[j]->prep_status;
    return first;
}

img_status img_solve_batch(img_ctx *const *ctxs, int n, double *const *sigma, img_solve_info *infos,
                           int on_device) {
    const Range range_("img.solve_batch");
    img_status st = check_batch(ctxs, n);
    if (st != IMG_OK) return st;
    if (!sigma) return IMG_EINVAL;
    for (int j = 0; j < n; ++j)
        if (!sigma[j]) return IMG_EINVAL;
    std::lock_guard<std::mutex> lock(g_ws.mu);
    st = ws_reserve(n, ctxs[0]->device);
    if (st != IMG_OK) return st;
    cudaStream_t s = ctxs[0]->stream;
    for (int j = 0; j < n; ++j)
        if (ctxs[j]->stream != s) CK(cudaStreamSynchronize(ctxs[j]->stream));
    const Groups g = group_by_mode(ctxs, n);
    std::vector<JobDev *> ptrs(n);
    std::vector<double *> outs(n);
    bool need_prep = false;
    for (int q = 0; q < n; ++q) {
        ptrs[q] = ctxs[g.order[q]]->dj;
        outs[q] = sigma[g.order[q]];
        need_prep |= !ctxs[g.order[q]]->prepared;
    }
    CK(cudaMemcpyAsync(g_ws.jobs, ptrs.data(), n * sizeof(JobDev *), cudaMemcpyHostToDevice, s));
    if (need_prep) {
        // prepared jobs are simply recomputed: same inputs, same results
        st = launch_prepare(ctxs, g, s, nullptr);
        if (st != IMG_OK) return st;
    }
    // wide jobs (64 < p <= 384 on tensor cores) run their solve graphs, each
    // on its context's stream after the batch's factor and bounds; the other
    // jobs run the one-CTA solver, one launch per arithmetic group
    std::vector<int> wide;
    for (int j = 0; j < n; ++j)
        if (wide_of(ctxs[j])) {
            st = wide_ready(ctxs[j]);
            if (st != IMG_OK) return st;
            wide.push_back(j);
        }
    if (!wide.empty()) {
        cudaEvent_t ready = nullptr;
        CK(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        CK(cudaEventRecord(ready, s));
        for (int j : wide) {
            img_ctx *c = ctxs[j];
            if (!c->ev) CK(cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming));
            CK(cudaStreamWaitEvent(c->stream, ready, 0));
            CK(img::ws_launch(c->ws, c->stream));
            CK(cudaEventRecord(c->ev, c->stream));
        }
        CK(cudaEventDestroy(ready));
    }
    if (on_device)
        CK(cudaMemcpyAsync(g_ws.sig, outs.data(), n * sizeof(double *), cudaMemcpyHostToDevice, s));
    for (int m = 0; m < kGroups; ++m) {
        std::vector<int> idx;               // positions q of this group's one-CTA jobs
        for (int q = g.begin[m]; q < g.end[m]; ++q)
            if (!wide_of(ctxs[g.order[q]])) idx.push_back(q);
        if (idx.empty()) continue;
        const bool contiguous = (int)idx.size() == g.end[m] - g.begin[m];
        if (contiguous) {
            CK(img::launch_solve(g_ws.jobs + g.begin[m], (int)idx.size(), g.max_p[m], Groups::solve_mode(m),
                                 g_ws.infos + g.begin[m], on_device ? g_ws.sig + g.begin[m] : nullptr, s));
        } else {
            for (int q : idx)
                CK(img::launch_solve(g_ws.jobs + q, 1, ctxs[g.order[q]]->prm.p, Groups::solve_mode(m), g_ws.infos + q,
                                     on_device ? g_ws.sig + q : nullptr, s));
        }
    }
    for (int j : wide) CK(cudaStreamWaitEvent(s, ctxs[j]->ev, 0));
    std::vector<DevInfo> d(n);
    CK(cudaMemcpyAsync(d.data(), g_ws.infos, n * sizeof(DevInfo), cudaMemcpyDeviceToHost, s));
    std::vector<DevInfo> dw(wide.size());
    for (size_t k = 0; k < wide.size(); ++k) {
        img_ctx *c = ctxs[wide[k]];
        CK(cudaMemcpyAsync(&dw[k], c->hj.info, sizeof(DevInfo), cudaMemcpyDeviceToHost, s));
        if (on_device)
            CK(cudaMemcpyAsync(sigma[wide[k]], c->hj.sigma, c->hj.Q * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    if (!on_device)
        for (int j = 0; j < n; ++j)
            CK(cudaMemcpyAsync(sigma[j], ctxs[j]->hj.sigma, ctxs[j]->hj.Q * sizeof(double),
                               cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    img_status first = IMG_OK;
    std::vector<DevInfo> byjob(n);
    for (int q = 0; q < n; ++q) byjob[g.order[q]] = d[q];
    for (size_t k = 0; k < wide.size(); ++k) byjob[wide[k]] = dw[k];
    for (int j = 0; j < n; ++j) {
        ctxs[j]->prepared = true;
        ctxs[j]->prep_status = byjob[j].status == IMG_ENOTPD ? IMG_ENOTPD : IMG_OK;
        ctxs[j]->solved = true;
        if (infos) fill_info(&infos[j], byjob[j]);
        if (first == IMG_OK && byjob[j].status != IMG_OK) first = (img_status)byjob[j].status;
    }
    return first;
}

void img_destroy(img_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->dmem) cudaFree(c->dmem);
    if (c->fwd_part) cudaFree(c->fwd_part);
    if (c->ls_exec) cudaGraphExecDestroy(c->ls_exec);
    if (c->ls_mem) cudaFree(c->ls_mem);
    if (c->ws) img::ws_destroy(c->ws);
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"

// ============================================================== serving
// Continuous batching of independent imaging jobs (not in the paper).  A
// scheduler thread admits queued jobs while in-flight slots and the HBM
// budget allow, reuses pooled job contexts of the same shape, and launches
// each admitted group (factor, bounds, solve) on a free stream of a small
// pool; groups launched later run next to earlier ones on the device, whose
// block scheduler places the new CTAs as SMs free up.  No kernel waits on the
// host: completion is an event the scheduler polls.
#include <chrono>
#include <cstdio>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <algorithm>

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

struct SJob {
    long long id = 0;
    img_params prm{};
    std::vector<double> ant, l, m, R;    // geometry and complex128 covariance (interleaved)
    long long N = 0;
    double t_submit = 0, t_start = 0, t_done = 0;
    int state = 0;                       // 0 queued, 1 on the GPU, 2 done
    img_status st = IMG_OK;
    std::vector<double> sigma;
    img_solve_info info{};
    img_ctx *ctx = nullptr;
};

struct SSlot {                           // one launch stream and its workspace
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    JobDev **jobs = nullptr;
    DevInfo *infos = nullptr;
    int *status = nullptr;
    DevInfo *h_infos = nullptr;          // pinned
    char *h_stage = nullptr;             // pinned staging of the group's inputs
    size_t stage_cap = 0, stage_off = 0;
    double *h_sigma = nullptr;           // pinned images of the group (grown on demand)
    size_t sigma_cap = 0;
    std::vector<size_t> sigma_off;
    std::vector<SJob *> group;
    bool busy = false;

    // Pinned copy of `bytes` from src; falls back to the (pageable) source
    // when the arena is full.
    const void *stage(const void *src, size_t bytes) {
        const size_t off = (stage_off + 255) & ~size_t(255);
        if (!h_stage || off + bytes > stage_cap) return src;
        std::memcpy(h_stage + off, src, bytes);
        stage_off = off + bytes;
        return h_stage + off;
    }
};

using ShapeKey = std::tuple<int, int, int, int>;   // p, n_l, n_m, support cap

ShapeKey key_of(const img_params &p) {
    const int Q = p.n_l * p.n_m;
    const int cap = p.support_cap > 0 ? std::min(p.support_cap, Q) : std::min(Q, 16384);
    return ShapeKey(p.p, p.n_l, p.n_m, cap);
}

// Load a job's parameters, geometry and covariance into a pooled context of
// the same shape (asynchronous on the slot's stream, inputs staged in the
// slot's pinned arena).
img_status reconfigure(img_ctx *c, SJob *j, SSlot &sl) {
    cudaStream_t s = sl.s;
    JobDev &J = c->hj;
    const img_params &P = j->prm;
    c->prm = P;
    c->ant = j->ant;
    c->l = j->l;
    c->m = j->m;
    c->prm.ant_xyz = c->ant.data();
    c->prm.l = c->l.data();
    c->prm.m = c->m.data();
    c->prm.stream = nullptr;
    J.cost = P.cost;
    J.bound = P.bound;
    J.bias_c = P.bias_c ? 1 : 0;
    J.inflate = P.inflate;
    J.lsqr_maxit = P.lsqr_maxit;
    J.max_outer = P.max_outer;
    J.precision = P.precision;
    J.alpha = P.alpha;
    J.kappa = P.kappa;
    J.eps_floor = P.eps_floor;
    J.lam = P.lambda;
    J.lsqr_atol = P.lsqr_atol;
    J.lsqr_btol = P.lsqr_btol;
    J.feas_tol = P.feas_tol;
    J.N = j->N;
    const int p = P.p;
    auto h2d = [&](void *dst, const void *src, size_t bytes) {
        return cudaMemcpyAsync(dst, sl.stage(src, bytes), bytes, cudaMemcpyHostToDevice, s);
    };
    CK(h2d((void *)J.ant, c->ant.data(), 3 * p * sizeof(double)));
    CK(h2d((void *)J.lg, c->l.data(), P.n_l * sizeof(double)));
    CK(h2d((void *)J.mg, c->m.data(), P.n_m * sizeof(double)));
    CK(h2d(J.R64, j->R.data(), (size_t)p * p * sizeof(double2)));
    CK(cudaMemsetAsync(J.flags, 0xff, sizeof(int), s));
    CK(cudaMemsetAsync(J.flags + 1, 0, sizeof(int), s));
    CK(h2d(c->dj, &J, sizeof(JobDev)));
    // the steering tables are recomputed inside the job's kernel
    c->has_cov = true;
    c->prepared = false;
    c->solved = false;
    return IMG_OK;
}

}  // namespace

struct img_server {
    img_server_params prm{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread th;
    bool stop = false;
    long long next_id = 0;
    std::unordered_map<long long, std::unique_ptr<SJob>> jobs;
    std::deque<SJob *> pending;
    std::map<ShapeKey, std::vector<img_ctx *>> free_ctx;
    std::vector<img_ctx *> all_ctx;
    size_t bytes_used = 0;
    int inflight = 0;
    std::vector<SSlot> slots;
    img_status fatal = IMG_OK;

    img_ctx *acquire(SJob *j) {
        auto &v = free_ctx[key_of(j->prm)];
        if (!v.empty()) {
            img_ctx *c = v.back();
            v.pop_back();
            return c;
        }
        img_params p = j->prm;
        p.ant_xyz = j->ant.data();
        p.l = j->l.data();
        p.m = j->m.data();
        p.stream = nullptr;
        // size check against the budget before allocating
        img_ctx probe;
        probe.prm = p;
        probe.hj.cap = std::get<3>(key_of(p));
        probe.hj.ev_cap = (int)std::min<long long>(p.max_outer > 0 ? p.max_outer : 10LL * p.n_l * p.n_m + 100,
                                                  1 << 20);
        {
            int sms = 1;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
            const size_t pp8 = (size_t)p.p * p.p * sizeof(float2);
            probe.nparts = std::max(1, std::min(2 * std::max(1, sms), (int)std::max<size_t>(1, (4u << 20) / pp8)));
        }
        probe.hj.p = p.p;
        probe.hj.Q = p.n_l * p.n_m;
        probe.hj.cost = p.cost;
        const size_t need = carve(&probe, nullptr) + (wide_of(&probe) ? img::ws_size(probe.hj) : 0);
        if (bytes_used + need > prm.hbm_budget_bytes) return nullptr;
        img_ctx *c = nullptr;
        if (img_create(&p, &c) != IMG_OK) return nullptr;
        if (wide_of(c) && wide_ready(c) != IMG_OK) {
            img_destroy(c);
            return nullptr;
        }
        c->dbytes += wide_of(c) ? img::ws_size(c->hj) : 0;
        bytes_used += c->dbytes;
        all_ctx.push_back(c);
        return c;
    }

    void release(img_ctx *c) { free_ctx[key_of(c->prm)].push_back(c); }

    // Free every pooled (idle) context; only called with nothing in flight.
    void evict_free() {
        for (auto &kv : free_ctx) {
            for (img_ctx *c : kv.second) {
                bytes_used -= c->dbytes;
                all_ctx.erase(std::find(all_ctx.begin(), all_ctx.end(), c));
                img_destroy(c);
            }
            kv.second.clear();
        }
    }

    img_status launch(SSlot &sl, std::vector<SJob *> &group) {
        const int n = (int)group.size();
        std::vector<img_ctx *> ctxs(n);
        sl.stage_off = 0;
        for (int q = 0; q < n; ++q) {
            ctxs[q] = group[q]->ctx;
            img_status st = reconfigure(ctxs[q], group[q], sl);
            if (st != IMG_OK) return st;
        }
        const Groups g = group_by_mode(ctxs.data(), n);
        std::vector<JobDev *> ptrs(n);
        for (int q = 0; q < n; ++q) ptrs[q] = ctxs[g.order[q]]->dj;
        CK(cudaMemcpyAsync(sl.jobs, sl.stage(ptrs.data(), n * sizeof(JobDev *)), n * sizeof(JobDev *),
                           cudaMemcpyHostToDevice, sl.s));
        // jobs [q0, q0 + nb) of group md on the one-CTA solver
        auto launch_range = [&](int md, int q0, int nb, int max_p, int max_tiles) -> img_status {
            JobDev *const *jp = sl.jobs + q0;
            if (md <= 2) {
                // one fused kernel: tables, factor, bounds and solve in one CTA per job
                CK(img::launch_job(jp, nb, max_p, md, sl.infos + q0, nullptr, sl.s));
            } else {
                CK(img::launch_tables(jp, nb, sl.s));
                CK(img::launch_factor(jp, nb, sl.s));
                CK(img::launch_bounds(jp, nb, max_tiles, max_p, Groups::bounds_mode(md), sl.s));
                CK(img::launch_finalize(jp, nb, sl.s, nullptr));
                CK(img::launch_solve(jp, nb, max_p, Groups::solve_mode(md), sl.infos + q0, nullptr, sl.s));
            }
            return IMG_OK;
        };
        for (int md = 0; md < kGroups; ++md) {
            std::vector<int> narrow;
            for (int q = g.begin[md]; q < g.end[md]; ++q) {
                img_ctx *c = ctxs[g.order[q]];
                if (!wide_of(c)) {
                    narrow.push_back(q);
                    continue;
                }
                // wide arrays on tensor cores: tables, factor and bounds (streamed
                // operator up to p = 256), then the job's solve graph
                JobDev *const *jp = sl.jobs + q;
                const int tiles = (c->hj.Q + img::kTile - 1) / img::kTile;
                img_status wst = wide_ready(c);
                if (wst != IMG_OK) return wst;
                CK(img::launch_tables(jp, 1, sl.s));
                CK(img::launch_factor(jp, 1, sl.s));
                if (items_bounds(c)) CK(img::ws_bounds(c->ws, c->hj, sl.s));
                else CK(img::launch_bounds(jp, 1, tiles, c->prm.p, op_mode_of(c), sl.s));
                CK(img::launch_finalize(jp, 1, sl.s, nullptr));
                CK(img::ws_launch(c->ws, sl.s));
                CK(cudaMemcpyAsync(sl.infos + q, c->hj.info, sizeof(DevInfo), cudaMemcpyDeviceToDevice, sl.s));
            }
            if (narrow.empty()) continue;
            img_status rst = IMG_OK;
            if ((int)narrow.size() == g.end[md] - g.begin[md]) {
                rst = launch_range(md, g.begin[md], (int)narrow.size(), g.max_p[md], g.max_tiles[md]);
            } else {
                for (int q : narrow) {
                    img_ctx *c = ctxs[g.order[q]];
                    rst = launch_range(md, q, 1, c->prm.p, (c->hj.Q + img::kTile - 1) / img::kTile);
                    if (rst != IMG_OK) break;
                }
            }
            if (rst != IMG_OK) return rst;
        }
        CK(cudaMemcpyAsync(sl.h_infos, sl.infos, n * sizeof(DevInfo), cudaMemcpyDeviceToHost, sl.s));
        // results in group order: remember the permutation
        sl.group.assign(n, nullptr);
        for (int q = 0; q < n; ++q) sl.group[q] = group[g.order[q]];
        // pinned result space was sized at creation (max_batch x max_pixels);
        // allocating pinned memory here would synchronise with running jobs
        size_t need = 0;
        sl.sigma_off.assign(n, 0);
        for (int q = 0; q < n; ++q) {
            sl.sigma_off[q] = need;
            need += sl.group[q]->ctx->hj.Q;
        }
        if (need > sl.sigma_cap) return IMG_ENOMEM;
        for (int q = 0; q < n; ++q) {
            img_ctx *c = sl.group[q]->ctx;
            CK(cudaMemcpyAsync(sl.h_sigma + sl.sigma_off[q], c->hj.sigma, c->hj.Q * sizeof(double),
                               cudaMemcpyDeviceToHost, sl.s));
        }
        CK(cudaEventRecord(sl.ev, sl.s));
        sl.busy = true;
        return IMG_OK;
    }

    // Publish a completed group (results already in the slot's pinned
    // buffers).  Called with the lock held; makes no CUDA calls.
    void finish(SSlot &sl) {
        const int n = (int)sl.group.size();
        const double t = now_ms();
        for (int q = 0; q < n; ++q) {
            SJob *j = sl.group[q];
            const int Q = j->ctx->hj.Q;
            j->sigma.assign(sl.h_sigma + sl.sigma_off[q], sl.h_sigma + sl.sigma_off[q] + Q);
            fill_info(&j->info, sl.h_infos[q]);
            j->st = (img_status)sl.h_infos[q].status;
            j->t_done = t;
            j->state = 2;
            release(j->ctx);
            j->ctx = nullptr;
        }
        inflight -= n;
        sl.group.clear();
        sl.busy = false;
    }

    // Scheduler: poll completions and launch admitted groups outside the
    // lock; hold it only to move jobs between the queue, the slots and done.
    void loop() {
        cudaSetDevice(device);
        std::vector<SSlot *> done, idle;
        std::vector<std::pair<SSlot *, std::vector<SJob *>>> plan;
        while (true) {
            done.clear();
            for (auto &sl : slots)
                if (sl.busy && cudaEventQuery(sl.ev) == cudaSuccess) done.push_back(&sl);
            plan.clear();
            {
                std::unique_lock<std::mutex> lk(mu);
                for (SSlot *sl : done) finish(*sl);
                if (!done.empty()) cv_done.notify_all();
                // admission: each free slot takes its share of the pending jobs
                // (one job per launch at low load, up to max_batch when jobs
                // outnumber free slots)
                idle.clear();
                for (auto &sl : slots)
                    if (!sl.busy) idle.push_back(&sl);
                int free_slots = (int)idle.size();
                for (SSlot *sl : idle) {
                    if (pending.empty()) break;
                    const int share = std::max(1, std::min(prm.max_batch,
                                                           ((int)pending.size() + free_slots - 1) / free_slots));
                    --free_slots;
                    std::vector<SJob *> group;
                    while (!pending.empty() && inflight < prm.max_inflight_jobs && (int)group.size() < share) {
                        SJob *j = pending.front();
                        img_ctx *c = acquire(j);
                        if (!c && inflight == 0 && plan.empty() && group.empty()) {
                            // nothing will free memory: drop pooled contexts of other shapes
                            evict_free();
                            c = acquire(j);
                            if (!c) {                    // the job alone exceeds the budget
                                pending.pop_front();
                                j->st = IMG_ENOMEM;
                                j->state = 2;
                                j->t_done = now_ms();
                                cv_done.notify_all();
                                continue;
                            }
                        }
                        if (!c) break;                   // wait for memory to free up
                        j->ctx = c;
                        j->state = 1;
                        j->t_start = now_ms();
                        pending.pop_front();
                        group.push_back(j);
                        ++inflight;
                    }
                    if (group.empty()) break;
                    sl->busy = true;                     // reserved for this plan
                    plan.emplace_back(sl, std::move(group));
                }
                const bool quiet = inflight == 0 && pending.empty() && plan.empty();
                if (stop && quiet) break;
                if (quiet) {
                    cv_work.wait(lk);
                    continue;
                }
            }
            for (auto &pg : plan) {
                img_status st = launch(*pg.first, pg.second);
                if (st != IMG_OK) {
                    std::lock_guard<std::mutex> lk(mu);
                    fatal = st;
                    for (SJob *j : pg.second) {
                        j->st = st;
                        j->state = 2;
                        j->t_done = now_ms();
                        if (j->ctx) release(j->ctx);
                        j->ctx = nullptr;
                        --inflight;
                    }
                    pg.first->busy = false;
                    pg.first->group.clear();
                    cv_done.notify_all();
                }
            }
            if (plan.empty() && done.empty()) {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait_for(lk, std::chrono::microseconds(200));
            }
        }
    }
};

extern "C" {

void img_server_params_default(img_server_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->hbm_budget_bytes = (size_t)8 << 30;
    p->max_inflight_jobs = 0;
    p->max_batch = 2;
    p->n_streams = 128;
    p->max_pixels = 65536;
}

img_status img_server_create(const img_server_params *prm, img_server **out) {
    if (!out || !prm) return IMG_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return IMG_ECUDA;
    img_server *s = new (std::nothrow) img_server();
    if (!s) return IMG_ENOMEM;
    s->prm = *prm;
    cudaGetDevice(&s->device);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->device);
    if (s->prm.max_inflight_jobs <= 0) s->prm.max_inflight_jobs = 2 * sms;
    if (s->prm.max_batch <= 0) s->prm.max_batch = 2;
    if (s->prm.n_streams <= 0) s->prm.n_streams = 128;
    if (s->prm.max_pixels <= 0) s->prm.max_pixels = 65536;
    s->slots.resize(s->prm.n_streams);
    const int mb = s->prm.max_batch;
    for (auto &sl : s->slots) {
        if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&sl.jobs, mb * sizeof(JobDev *)) != cudaSuccess ||
            cudaMalloc(&sl.infos, mb * sizeof(DevInfo)) != cudaSuccess ||
            cudaMallocHost(&sl.h_infos, mb * sizeof(DevInfo)) != cudaSuccess ||
            cudaMallocHost(&sl.h_stage, sl.stage_cap = (size_t)mb * (64 << 10) + (4 << 20)) != cudaSuccess ||
            cudaMallocHost(&sl.h_sigma, (sl.sigma_cap = (size_t)mb * s->prm.max_pixels) * sizeof(double)) !=
                cudaSuccess) {
            img_server_destroy(s);
            return IMG_ECUDA;
        }
    }
    s->th = std::thread([s] { s->loop(); });
    *out = s;
    return IMG_OK;
}

img_status img_server_reserve(img_server *s, const img_params *prm, int count) {
    if (!s || !prm || count < 0) return IMG_EINVAL;
    SJob probe;
    probe.prm = *prm;
    probe.ant.assign(prm->ant_xyz, prm->ant_xyz + 3 * prm->p);
    probe.l.assign(prm->l, prm->l + prm->n_l);
    probe.m.assign(prm->m, prm->m + prm->n_m);
    std::lock_guard<std::mutex> lk(s->mu);
    std::vector<img_ctx *> got;
    for (int k = 0; k < count; ++k) {
        img_ctx *c = s->acquire(&probe);
        if (!c) break;
        got.push_back(c);
    }
    for (img_ctx *c : got) s->release(c);
    return (int)got.size() == count ? IMG_OK : IMG_ENOMEM;
}

img_status img_server_submit(img_server *s, const img_params *prm, const void *R, int dtype, long long N,
                             long long *job_id) {
    if (!s || !prm || !R || !job_id) return IMG_EINVAL;
    if (dtype != IMG_C64 && dtype != IMG_C128) return IMG_EINVAL;
    if (N <= prm->p) return IMG_EINVAL;
    if ((long long)prm->n_l * prm->n_m > s->prm.max_pixels) return IMG_EINVAL;
    // validate by the same rules as img_create, without allocating
    if (prm->p < 2 || prm->p > kMaxP || prm->n_l < 1 || prm->n_m < 1 || !prm->ant_xyz || !prm->l ||
        !prm->m || !(prm->lambda > 0.0))
        return IMG_EINVAL;
    for (int k = 0; k < prm->p; ++k)
        if (prm->ant_xyz[3 * k + 2] != 0.0) return IMG_EINVAL;
    auto j = std::make_unique<SJob>();
    j->prm = *prm;
    j->ant.assign(prm->ant_xyz, prm->ant_xyz + 3 * prm->p);
    j->l.assign(prm->l, prm->l + prm->n_l);
    j->m.assign(prm->m, prm->m + prm->n_m);
    const size_t pp = (size_t)prm->p * prm->p;
    j->R.resize(2 * pp);
    if (dtype == IMG_C128) std::memcpy(j->R.data(), R, 2 * pp * sizeof(double));
    else
        for (size_t e = 0; e < 2 * pp; ++e) j->R[e] = static_cast<const float *>(R)[e];
    if (!finite_all(j->R.data(), j->R.size())) return IMG_EINVAL;
    j->N = N;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->fatal != IMG_OK) return s->fatal;
        j->id = s->next_id++;
        j->t_submit = now_ms();
        *job_id = j->id;
        s->pending.push_back(j.get());
        s->jobs.emplace(j->id, std::move(j));
    }
    s->cv_work.notify_all();
    return IMG_OK;
}

img_status img_server_wait(img_server *s, long long job_id, double *sigma, img_solve_info *info,
                           double timeout_ms, double *latency_ms) {
    if (!s) return IMG_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return IMG_EINVAL;
    SJob *j = it->second.get();
    const auto until = std::chrono::steady_clock::now() +
                       std::chrono::microseconds((long long)(std::max(0.0, timeout_ms) * 1000.0));
    while (j->state != 2) {
        if (s->cv_done.wait_until(lk, until) == std::cv_status::timeout && j->state != 2) return IMG_ETIMEOUT;
    }
    if (sigma) std::memcpy(sigma, j->sigma.data(), j->sigma.size() * sizeof(double));
    if (info) *info = j->info;
    if (latency_ms) *latency_ms = j->t_done - j->t_submit;
    const img_status st = j->st;
    s->jobs.erase(it);
    return st;
}

void img_server_destroy(img_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (auto &sl : s->slots) {
        if (sl.s) cudaStreamSynchronize(sl.s);
        if (sl.jobs) cudaFree(sl.jobs);
        if (sl.infos) cudaFree(sl.infos);
        if (sl.h_infos) cudaFreeHost(sl.h_infos);
        if (sl.h_stage) cudaFreeHost(sl.h_stage);
        if (sl.h_sigma) cudaFreeHost(sl.h_sigma);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.s) cudaStreamDestroy(sl.s);
    }
    for (img_ctx *c : s->all_ctx) img_destroy(c);
    delete s;
}

}  // extern "C"
