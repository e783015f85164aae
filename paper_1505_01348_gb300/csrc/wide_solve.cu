// Wide active-set solver (Table I with LSQR subproblems, Sec. IV and V) for
// 64 < p <= 384 on tensor cores, as one CUDA graph per job.
//
// The Table I loop is a graph WHILE node whose body is one pass (or two:
// freeing the pixel chosen by the last gradient, then the next subproblem).
// The subproblem's LSQR is an IF node holding the initialisation and a WHILE
// node of Golub-Kahan iterations; the feasible / infeasible branch is an
// IF/ELSE node.  Kernels set the conditions from device memory, so a whole
// solve runs without a host round trip.  Every kernel has a fixed grid and
// reads the sizes of the moment (|F|, |U|, support) from the control block.
//
// Operators (tc_items.cuh): the adjoint over the free set or over every pixel
// runs in (tile, unit) work items from a B image of U; the forward over a
// list forms Gram blocks from a list image.  Both split products FP16x3 or
// BF16x3 with FP32 accumulation.  Scalars of LSQR, feasibility, the step and
// the multiplier tests are FP64 or FP32 exactly as in the one-CTA solver.
//
// PWLS gradient: with d_i = R^-1 a_i cached per support pixel, the whitened
// residual is U_g = R^-1 - sum_S s_i x_i d_i d_i^H (= L^-H (I - sum s x c c^H)
// L^-1 with c_i = L^-1 a_i), so no p^3 sandwich runs per gradient.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "cta_ops.cuh"
#include "tc_items.cuh"

namespace img {

constexpr int kWsThreads = 256;
// Grid of the list kernels (forward, free-list adjoint): a share of the SMs,
// so that the kernels of several solves in flight pack next to each other;
// the full-image adjoint of the gradient takes every SM.  32 measured best
// for 16 solves of 256x256, p = 288 in flight (0.54 images/s; 64 CTAs:
// 0.48, 48: 0.51, 16: 0.53); fewer CTAs also mean fewer forward splits.
constexpr int kListGrid = 32;
constexpr int kWsSums = 2048;           // per-CTA partial sums of the reductions
// 64-pixel stages per forward task (at least).  Fewer, longer tasks write
// fewer partial blocks for the reduction to read back (16 solves of 256x256,
// p = 288 in flight: 4 -> 0.539, 8 -> 0.551, 16 -> 0.561 images/s), but the
// split also fixes the order of the forward's partial sums, and with 4 the
// complete 256x256, p = 288 solve takes the FP64 oracle's decisions one for
// one at the same LSQR tolerance (with 16 a tie at decision 2013 of 2797
// falls the other way).
constexpr int kFwdPerTask = 4;

// Device control block of one wide solve.
struct WsCtl {
    int f, nu, ns;              // |F|, |U|, |F u U| of the current subproblem
    int pending;                // pixel the last gradient chose to free, or -1
    int outer;                  // Table I passes so far
    int stop;                   // the loop ends after this pass
    int converged, status, feasible, nev, timeouts;
    int it, maxit, lsqr_total;  // LSQR iterations of this subproblem / cap / sum
    int nsplit;                 // forward split of the current list
    int nlist;                  // length of the current forward list
    int adj_rows;               // unit x K-group partial rows of the free-list adjoint
    float sXF, sXS;             // power-of-two scales of the F and support list images
    float sW;                   // weight scale used by the last forward
    float sB;                   // scale of the current B image
    unsigned mx_t, mx_w;        // max |entry| bits of the matrix being imaged / the weights
    unsigned long long key;     // argmin key of the multiplier test
    double alpha, beta, us, bnorm, anorm2, rhobar, phibar, fa;
    double lam_min, op_flops;
    unsigned long long t_begin;
    unsigned cond[4];           // last value of each loop / branch condition (host-driven mode)
    int cache_slot, cache_pixel; // support slot whose vectors k_ws_cache computes (-1: none)
    int nsums;                  // CTA shares of ||t||^2 left in sums by k_ws_fred
    int adj_sq;                 // full-image adjoint as sums of squares (MVDR denominators)
    unsigned long long launches;  // kernels executed in this solve
    double sums[kWsSums];
};

enum { kCondOuter = 0, kCondLsqrIf = 1, kCondLsqr = 2, kCondFeas = 3 };

// Set a graph condition (h != 0 inside the solve graph) and mirror it in the
// control block for the host-driven mode.
__device__ __forceinline__ void ws_cond(WsCtl *ctl, int which, cudaGraphConditionalHandle h, unsigned v) {
    ctl->cond[which] = v;
    if (h) cudaGraphSetConditional(h, v);
}

// Device buffers of the wide solver (device pointers, passed by value).
struct WsBufs {
    WsCtl *ctl;
    float2 *dvec;               // cap x p: d_i = R^-1 a_i (PWLS); cvec for LS
    float *dmax;                // cap
    int *iota;                  // cap: 0, 1, 2, ...
    float *wl;                  // cap: weights of the current forward list
    float *padj;                // max(Q, cap) x (nu nk): unit (x K group) partial dots, row-contiguous
    float *pfwd;                // forward partial blocks (tasks x 128 x 256)
    unsigned char *ximgF, *ximgS, *ximgW, *bimg;   // list images: F, U or support, weighted; B image
    int npairs, pm[kItemsFwdMaxPairs], pnb[kItemsFwdMaxPairs];
    int max_tasks;              // capacity of pfwd in blocks
    int fwd_per;                // 64-pixel stages per forward task (at least)
    int nrows_adj;              // rows of padj (max(Q, cap))
    int ld_adj;                 // partial dots per row of padj (nu nk)
};

enum { kListF = 0, kListU = 1, kListS = 2 };
enum { kRedB = 0, kRedT = 1, kRedG = 2 };

__device__ __forceinline__ float pow2_scale(float mx) { return mx > 0.f ? exp2f(-ceilf(log2f(mx))) : 1.f; }
__device__ __forceinline__ unsigned long long key_of(float lam, int i) {
    unsigned b = __float_as_uint(lam);
    b = (b & 0x80000000u) ? ~b : (b | 0x80000000u);      // order-preserving
    return ((unsigned long long)b << 32) | (unsigned)i;
}
__device__ __forceinline__ float lam_of(unsigned long long key) {
    unsigned b = (unsigned)(key >> 32);
    b = (b & 0x80000000u) ? (b & 0x7fffffffu) : ~b;
    return __uint_as_float(b);
}
__device__ __forceinline__ double ws_flops_fwd(int p, int n) { return 4.0 * p * (double)p * n; }
__device__ __forceinline__ double ws_flops_adj(int p, int n) { return 8.0 * p * (double)p * n; }

// Count this kernel in the solve's launch total (block 0, thread 0).
__device__ __forceinline__ void ws_count(WsCtl *ctl) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctl->launches, 1ull);
}

__device__ void ws_log(const JobDev &J, WsCtl *ctl, int kind, int pixel, float val) {
    if (ctl->nev < J.ev_cap) {
        J.ev[ctl->nev] = (kind << 24) | pixel;
        J.evv[ctl->nev] = val;
    }
    ctl->nev++;
}

// ---------------------------------------------------------------- start / end
__global__ void k_ws_start(const JobDev *Jp, WsBufs B, cudaGraphConditionalHandle h_outer) {
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    for (int i = threadIdx.x; i < J.Q; i += blockDim.x) {
        J.x[i] = 0.0;
        J.set[i] = IMG_SET_L;
        J.slot[i] = -1;
        J.grad[i] = 0.f;
    }
    for (int j = threadIdx.x; j < J.cap; j += blockDim.x) B.iota[j] = j;
    if (threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        ctl->t_begin = t;
        ctl->launches = 1;
        ctl->f = ctl->nu = ctl->ns = 0;
        ctl->pending = -1;
        ctl->outer = 0;
        ctl->converged = 0;
        ctl->status = IMG_OK;
        ctl->feasible = 0;
        ctl->nev = 0;
        ctl->timeouts = 0;
        ctl->it = ctl->maxit = ctl->lsqr_total = 0;
        ctl->nsplit = 1;
        ctl->nlist = 0;
        ctl->mx_t = ctl->mx_w = 0;
        ctl->lam_min = 0.0;
        ctl->op_flops = 0.0;
        ctl->stop = 0;
        if (J.flags[0] != 0 || J.flags[1] != 1) {
            ctl->status = J.flags[0] != 0 ? J.flags[0] : IMG_EINVAL;
            ctl->stop = 1;
        }
        ws_cond(ctl, kCondOuter, h_outer, ctl->stop ? 0u : 1u);
    }
}

__global__ void k_ws_end(const JobDev *Jp, WsBufs B, cudaGraphConditionalHandle h_outer) {
    ws_count(B.ctl);
    WsCtl *ctl = B.ctl;
    if (threadIdx.x == 0) ws_cond(ctl, kCondOuter, h_outer, ctl->stop ? 0u : 1u);
}

__global__ void k_ws_finish(const JobDev *Jp, WsBufs B) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    __shared__ double sbuf[kWsThreads / 32];
    int nf = 0, nu = 0;
    for (int i = threadIdx.x; i < J.Q; i += blockDim.x) {
        J.sigma[i] = (double)J.scale[i] * J.x[i];
        nf += J.set[i] == IMG_SET_F;
        nu += J.set[i] == IMG_SET_U;
    }
    const double tf = block_sum((double)nf, sbuf);
    const double tu = block_sum((double)nu, sbuf);
    if (threadIdx.x == 0) {
        DevInfo info{};
        int st = ctl->status;
        if (st == IMG_OK && ctl->timeouts) st = IMG_ETIMEOUT;
        if (st == IMG_OK && !ctl->converged) st = IMG_ENOTCONV;
        info.status = st;
        info.outer = ctl->outer;
        info.lsqr_iters = ctl->lsqr_total;
        info.n_free = (int)tf;
        info.n_upper = (int)tu;
        info.converged = ctl->converged;
        info.lambda_min = ctl->lam_min;
        info.op_flops = ctl->op_flops;
        info.t_begin_ns = ctl->t_begin;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        info.t_end_ns = t;
        info.cyc_total = (double)(t - ctl->t_begin);
        info.cyc_aux[0] = (double)ctl->launches;      // kernels this solve executed
        *J.ev_count = ctl->nev;
        *J.info = info;
    }
}

// ---------------------------------------------------------------- support cache
// c_i = T a_i (T = L^-1 for PWLS, I for LS) into cvec row `slot`, and for
// PWLS d_i = R^-1 a_i into dvec; their largest component magnitudes by
// atomicMax on the float bits (cmax / dmax of the slot start at zero).
// CTA b computes rows k = 32 b + lane; warp w sums the terms l = w, w + 8, ...
constexpr int kCacheRows = 32;
__global__ void __launch_bounds__(kWsThreads) k_ws_cache(const JobDev *Jp, WsBufs B) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    const WsCtl *ctl = B.ctl;
    const int slot = ctl->cache_slot;
    if (ctl->stop || slot < 0) return;
    const int i = ctl->cache_pixel;
    const int p = J.p;
    const int im = i / J.n_l, il = i - im * J.n_l;
    const bool pwls = J.cost == IMG_COST_PWLS;
    __shared__ float2 sa[kItemsMaxP];
    __shared__ float2 part[2][8][kCacheRows];
    for (int k = threadIdx.x; k < p; k += blockDim.x) sa[k] = steer(J, il, im, k);
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int k = blockIdx.x * kCacheRows + lane;
    float2 sc = make_float2(0.f, 0.f), sd = make_float2(0.f, 0.f);
    if (k < p) {
        if (!pwls) {
            if (w == 0) sc = sa[k];
        } else {
            const float2 *__restrict__ Li = J.Li32 + k;
            const float2 *__restrict__ Ri = J.Ri32 + k;
#pragma unroll 4
            for (int l = w; l <= k; l += 8) cfma(sc, Li[(size_t)l * p], sa[l]);
#pragma unroll 4
            for (int l = w; l < p; l += 8) cfma(sd, Ri[(size_t)l * p], sa[l]);
        }
    }
    part[0][w][lane] = sc;
    part[1][w][lane] = sd;
    __syncthreads();
    if (w == 0) {
        float2 c = make_float2(0.f, 0.f), d = make_float2(0.f, 0.f);
        for (int q = 0; q < 8; ++q) {
            c.x += part[0][q][lane].x;
            c.y += part[0][q][lane].y;
            d.x += part[1][q][lane].x;
            d.y += part[1][q][lane].y;
        }
        float mc = 0.f, md = 0.f;
        if (k < p) {
            J.cvec[(size_t)slot * p + k] = c;
            mc = fmaxf(fabsf(c.x), fabsf(c.y));
            if (pwls) {
                B.dvec[(size_t)slot * p + k] = d;
                md = fmaxf(fabsf(d.x), fabsf(d.y));
            }
        }
        for (int o = 16; o; o >>= 1) {
            mc = fmaxf(mc, __shfl_xor_sync(0xffffffffu, mc, o));
            md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
        }
        if (lane == 0) {
            atomicMax(reinterpret_cast<unsigned *>(J.cmax + slot), __float_as_uint(mc));
            if (pwls) atomicMax(reinterpret_cast<unsigned *>(B.dmax + slot), __float_as_uint(md));
        }
    }
}

// Remove support slot of pixel i (swap with the last entry).
__device__ void ws_remove(const JobDev &J, const WsBufs &B, int i, int &ns) {
    const int p = J.p;
    const int sl = J.slot[i];
    const int last = ns - 1;
    const bool pwls = J.cost == IMG_COST_PWLS;
    if (sl != last) {
        const int moved = J.supp[last];
        for (int k = threadIdx.x; k < p; k += blockDim.x) {
            J.cvec[(size_t)sl * p + k] = J.cvec[(size_t)last * p + k];
            if (pwls) B.dvec[(size_t)sl * p + k] = B.dvec[(size_t)last * p + k];
        }
        if (threadIdx.x == 0) {
            J.supp[sl] = moved;
            J.slot[moved] = sl;
            J.cmax[sl] = J.cmax[last];
            if (pwls) B.dmax[sl] = B.dmax[last];
        }
    }
    if (threadIdx.x == 0) J.slot[i] = -1;
    ns = last;
    __syncthreads();
}

// Largest value of a per-slot maximum array over a position list (CTA).
__device__ float ws_list_max(const float *mx, const int *pos, int n) {
    __shared__ float sred[kWsThreads / 32];
    float m = 0.f;
    for (int j = threadIdx.x; j < n; j += blockDim.x) m = fmaxf(m, mx[pos ? pos[j] : j]);
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = m;
    __syncthreads();
    m = 0.f;
    for (int w = 0; w < kWsThreads / 32; ++w) m = fmaxf(m, sred[w]);
    __syncthreads();
    return m;
}

// K groups of the free-list adjoint: the largest divisor of nk that keeps
// the work items within the grid.
__device__ int ws_nkg(int items, int nk, int grid) {
    int best = 1;
    for (int d = 1; d <= nk; ++d)
        if (nk % d == 0 && items * d <= grid) best = d;
    return best;
}

__device__ int ws_nsplit(int n, int npairs, int max_tasks, int per) {
    const int stages = (n + kFwdPix - 1) / kFwdPix;
    int ns = (stages + per - 1) / per;             // about `per` stages per task
    const int cap = max(1, max_tasks / max(npairs, 1));
    ns = min(ns, cap);
    return max(ns, 1);
}

// ---------------------------------------------------------------- pass
// Table I, first part of a loop iteration: free the pending pixel (a pass of
// its own): give it a support slot when it has none (its vectors are then
// computed by k_ws_cache), move it to F and log it.
__global__ void k_ws_free(const JobDev *Jp, WsBufs B) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    if (threadIdx.x != 0) return;
    ctl->cache_slot = -1;
    if (ctl->stop) return;
    const int max_outer = J.max_outer > 0 ? J.max_outer : 10 * J.Q + 100;
    const int i = ctl->pending;
    if (i < 0) return;
    if (ctl->outer >= max_outer) {
        ctl->stop = 1;
        return;
    }
    int ns = ctl->ns;
    if (J.slot[i] < 0) {
        if (ns >= J.cap) {
            ctl->status = IMG_ENOMEM;
            ctl->stop = 1;
            return;
        }
        J.supp[ns] = i;
        J.slot[i] = ns;
        J.cmax[ns] = 0.f;
        if (J.cost == IMG_COST_PWLS) B.dmax[ns] = 0.f;
        ctl->cache_slot = ns;
        ctl->cache_pixel = i;
        ctl->ns = ns + 1;
    }
    ctl->outer++;
    J.set[i] = IMG_SET_F;
    ws_log(J, ctl, 0, i, (float)ctl->lam_min);
    ctl->pending = -1;
}

// Then set up the subproblem of the next pass: compact F and U, the U
// weights -s_i x_i (eq. bsubproblemLS / MVDR), the F scales, the list scales
// and the LSQR iteration cap; h_lif := (|F| > 0).
__global__ void k_ws_pass(const JobDev *Jp, WsBufs B, cudaGraphConditionalHandle h_lif) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    __shared__ int cbuf[kWsThreads / 32];
    __shared__ int s_skip;
    const int max_outer = J.max_outer > 0 ? J.max_outer : 10 * J.Q + 100;
    const int ns = ctl->ns;
    if (threadIdx.x == 0) {
        if (!ctl->stop && ctl->outer >= max_outer) ctl->stop = 1;
        s_skip = ctl->stop;
    }
    __syncthreads();
    if (s_skip) {
        if (threadIdx.x == 0) {
            ctl->f = 0;
            ws_cond(ctl, kCondLsqrIf, h_lif, 0u);
        }
        return;
    }
    const int f = block_compact(ns, [&](int pos) { return J.set[J.supp[pos]] == IMG_SET_F; }, J.fpos, cbuf);
    const int nu = block_compact(ns, [&](int pos) { return J.set[J.supp[pos]] == IMG_SET_U; }, J.fpos + f, cbuf);
    float wm = 0.f;
    for (int j = threadIdx.x; j < nu; j += blockDim.x) {
        const int i = J.supp[J.fpos[f + j]];
        const float wv = -J.scale[i] * (float)J.x[i];
        B.wl[j] = wv;
        wm = fmaxf(wm, fabsf(wv));
    }
    for (int j = threadIdx.x; j < f; j += blockDim.x) J.sF[j] = J.scale[J.supp[J.fpos[j]]];
    const float mF = ws_list_max(J.cmax, J.fpos, f);
    const float mU = ws_list_max(J.cmax, J.fpos + f, nu);
    for (int o = 16; o; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, o));
    __shared__ float swm[kWsThreads / 32];
    if ((threadIdx.x & 31) == 0) swm[threadIdx.x >> 5] = wm;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < kWsThreads / 32; ++w) wm = fmaxf(wm, swm[w]);
        ctl->outer++;
        ctl->f = f;
        ctl->nu = nu;
        ctl->nlist = nu;
        ctl->sXF = pow2_scale(mF) * kLift;
        ctl->sXS = pow2_scale(mU) * kLift;
        ctl->mx_w = __float_as_uint(wm);
        ctl->nsplit = ws_nsplit(nu, B.npairs, B.max_tasks, B.fwd_per);
        ctl->maxit = J.lsqr_maxit > 0 ? J.lsqr_maxit : 4 * f + 20;
        ctl->it = 0;
        ctl->op_flops += ws_flops_fwd(J.p, nu);
        ws_cond(ctl, kCondLsqrIf, h_lif, f > 0 ? 1u : 0u);
    }
}

// ---------------------------------------------------------------- images
// List image of the F list (cvec, scale sXF), of the U list (cvec, scale
// sXS) or of the support (dvec / cvec, scale sXS); every row of the tiles
// and the padding chunks are written.  U and S share one image buffer.
// weighted: the image of the rows times their weights wl (the second
// operand of a forward) into ximgW, scaled by sX sW with sW the power of two
// of max |wl| (stored for the reduction).
template <bool BF16>
__global__ void k_ws_listimg(const JobDev *Jp, WsBufs B, int which, int weighted) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    if (ctl->stop) return;
    const UnitGeom g = unit_geom(J.p);
    const bool S = which == kListS, Ul = which == kListU;
    const int n = S ? ctl->ns : (Ul ? ctl->nu : ctl->f);
    const int *pos = S ? B.iota : (Ul ? J.fpos + ctl->f : J.fpos);
    const float2 *vec = (S && J.cost == IMG_COST_PWLS) ? B.dvec : J.cvec;
    float sX = (S || Ul) ? ctl->sXS : ctl->sXF;
    unsigned char *img = weighted ? B.ximgW : ((S || Ul) ? B.ximgS : B.ximgF);
    if (weighted) {
        const float sW = pow2_scale(__uint_as_float(ctl->mx_w));
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->sW = sW;
        sX *= sW;
    }
    const float *wgt = weighted ? B.wl : nullptr;
    const int ntl = (n + kTcM - 1) / kTcM;
    const long long total = (long long)ntl * g.nkA * kTcM * 8;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c16 = (int)(e & 7);
        long long r2 = e >> 3;
        const int r = (int)(r2 % kTcM);
        r2 /= kTcM;
        const int kc = (int)(r2 % g.nkA), t = (int)(r2 / g.nkA);
        list_image_chunk<BF16>(vec, pos, wgt, n, J.p, g, sX, img, t, kc, r, c16);
    }
}

// B unit image of the matrix U (W0 for LSQR, W1 for the gradient) with the
// power-of-two scale of ctl->mx_t.
template <bool BF16>
__global__ void k_ws_emb(const JobDev *Jp, WsBufs B, int grad, const float2 *Um) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    if (ctl->stop) return;
    const UnitGeom g = unit_geom(J.p);
    const float sc = pow2_scale(__uint_as_float(ctl->mx_t)) * kLift;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->sB = sc;
    const float2 *U = Um ? Um : (grad ? J.W1 : J.W0);
    const int rows = unit_rows(g);
    const long long total = (long long)g.nu * g.nk * rows * 8;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c16 = (int)(e & 7);
        long long r2 = e >> 3;
        const int n = (int)(r2 % rows);
        r2 /= rows;
        const int kc = (int)(r2 % g.nk), u = (int)(r2 / g.nk);
        unit_image_chunk<BF16>(U, J.p, g, sc, B.bimg, u, kc, n, c16);
    }
}

// ---------------------------------------------------------------- operators
// Forward over the current list: F (weights wl = s_j v_j, cvec), U (weights
// -s_i x_i, cvec) or the support S (weights -s_i x_i, dvec / cvec): Gram
// blocks from the list's image and its weighted image.
template <bool BF16>
__global__ void __launch_bounds__(kItemsFwdThreads, 1) k_ws_fwd(const JobDev *Jp, WsBufs B, int which) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    if (ctl->stop) return;
    const UnitGeom g = unit_geom(J.p);
    const int n = which == kListF ? ctl->f : (which == kListU ? ctl->nu : ctl->ns);
    const unsigned char *XA = which == kListF ? B.ximgF : B.ximgS;
    if (n <= 0) return;
    const int nsplit = ctl->nsplit;
    const int tasks = B.npairs * nsplit;
    extern __shared__ float4 smem4[];
    unsigned char *dyn = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem4) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bars[6];
    __shared__ uint32_t tslot;
    if (blockIdx.x >= tasks) return;
    // one tensor-memory allocation for all of this CTA's tasks
    if (threadIdx.x < 32) tmem_alloc(&tslot, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    int to = 0;
    for (int task = blockIdx.x; task < tasks; task += gridDim.x) {
        const int pr = task / nsplit, s = task - pr * nsplit;
        to += items_forward<BF16>(g, dyn, bars, tmem, XA, B.ximgW, n, B.pm[pr], B.pnb[pr], s, nsplit,
                                  B.pfwd + (size_t)task * kTcM * 256);
        __syncthreads();
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(tmem, 256);
    if (to && threadIdx.x == 0) {
        // a broken pipeline ends the solve: every later kernel sees stop
        atomicAdd(&ctl->timeouts, to);
        ctl->stop = 1;
    }
}

// Sum the forward partial blocks in a fixed order into K and form
//   kRedB: W0 = base + K             (subproblem data, base R_hat or I)
//   kRedT: W0 = K - fa W0            (LSQR: t <- M v - alpha u, u = t us)
//   kRedG: W1 = base + K             (gradient residual, base R_hat or R_hat^-1)
// with K = sum w_j v_j v_j^H (weights carry the sign); max |entry| into
// mx_t; for kRedB / kRedT the norm beta = ||W0|| (FP64, fixed order).
// Re K(a,b) = G(a,b) + G(Kp+a,Kp+b), Im K(a,b) = G(b,Kp+a) - G(a,Kp+b) with G
// read in its upper triangle.  One CTA per 32 x 32 tile of (a, b): the four
// source tiles are read row by row (coalesced) into shared memory, those
// stored below the diagonal transposed on the way.
constexpr int kRedTile = 32;

// address of the stored Gram entry (r, c), r <= c, in the first partial of
// its block (blocks are column-major: entry (r, c) of block (m, nb) at
// (c - 256 nb) 128 + r - 128 m); partial q follows at q 128 256
__device__ __forceinline__ const float *fred_at(const WsBufs &B, const int *pidx, int nsplit, int r, int c) {
    const int m = r >> 7, nb = c >> 8;
    return B.pfwd + (size_t)pidx[m * 4 + nb] * nsplit * kTcM * 256 + (size_t)(c - 256 * nb) * kTcM + (r - 128 * m);
}

__global__ void __launch_bounds__(kWsThreads) k_ws_fred(const JobDev *Jp, WsBufs B, int mode) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    if (ctl->stop) return;
    const int p = J.p;
    const UnitGeom g = unit_geom(p);
    const int Kp = g.Kp;
    const bool pwls = J.cost == IMG_COST_PWLS;
    const int n = mode == kRedT ? ctl->f : (mode == kRedB ? ctl->nu : ctl->ns);
    const int nsplit = ctl->nsplit;
    const float sX = mode == kRedT ? ctl->sXF : ctl->sXS;
    const float inv = n > 0 ? 1.f / (sX * sX * ctl->sW) : 0.f;
    const float fa = (float)ctl->fa;
    float2 *dst = mode == kRedG ? J.W1 : J.W0;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->mx_w = 0u;     // the weights are consumed
    __shared__ int pidx[6 * 4];
    __shared__ float T[4][kRedTile][kRedTile + 1];   // G(a,b), G(Kp+a,Kp+b), G(a,Kp+b), G(b,Kp+a), as [a][b]
    if (threadIdx.x < 24) pidx[threadIdx.x] = 0;
    __syncthreads();
    if (threadIdx.x < B.npairs) pidx[B.pm[threadIdx.x] * 4 + B.pnb[threadIdx.x]] = threadIdx.x;
    __syncthreads();
    const int nt = (p + kRedTile - 1) / kRedTile;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;      // 32 x 8
    float mx = 0.f, ss = 0.f;
    for (int tile = blockIdx.x; tile < nt * nt; tile += gridDim.x) {
        const int a0 = (tile % nt) * kRedTile, b0 = (tile / nt) * kRedTile;
        if (n > 0) {
            // the stored blocks are column-major: lanes run along the stored
            // row index (coalesced), i along the column.  Each thread gathers
            // the addresses of all its entries first, then sums the partials
            // with every load of a partial in flight at once.
            const float *src[4][6];
            float acc[4][6];
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) {
                const int i = ty + 8 * ii;
                const int a = a0 + tx, b = b0 + i;           // element (a, b) = tile [tx][i]
                const int bt = b0 + tx, at = a0 + i;         // element (at, bt) = tile [i][tx]
                const bool up = (a0 < b0 || (a0 == b0 && a <= b)) && a < p && b < p;
                const bool lo = (a0 > b0 || (a0 == b0 && bt <= at)) && at < p && bt < p;
                src[ii][0] = up ? fred_at(B, pidx, nsplit, a, b) : nullptr;              // G(a, b)
                src[ii][1] = up ? fred_at(B, pidx, nsplit, Kp + a, Kp + b) : nullptr;    // G(Kp+a, Kp+b)
                src[ii][2] = lo ? fred_at(B, pidx, nsplit, bt, at) : nullptr;            // G(at, bt)
                src[ii][3] = lo ? fred_at(B, pidx, nsplit, Kp + bt, Kp + at) : nullptr;
                src[ii][4] = (a < p && b < p) ? fred_at(B, pidx, nsplit, a, Kp + b) : nullptr;     // G(a, Kp+b)
                src[ii][5] = (at < p && bt < p) ? fred_at(B, pidx, nsplit, bt, Kp + at) : nullptr; // G(b, Kp+a)
#pragma unroll
                for (int e = 0; e < 6; ++e) acc[ii][e] = 0.f;
            }
            for (int q = 0; q < nsplit; ++q) {
                const size_t off = (size_t)q * kTcM * 256;
                float v[4][6];
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                    for (int e = 0; e < 6; ++e) v[ii][e] = src[ii][e] ? src[ii][e][off] : 0.f;
#pragma unroll
                for (int ii = 0; ii < 4; ++ii)
#pragma unroll
                    for (int e = 0; e < 6; ++e) acc[ii][e] += v[ii][e];
            }
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) {
                const int i = ty + 8 * ii;
                if (src[ii][0]) {
                    T[0][tx][i] = acc[ii][0];
                    T[1][tx][i] = acc[ii][1];
                }
                if (src[ii][2]) {
                    T[0][i][tx] = acc[ii][2];
                    T[1][i][tx] = acc[ii][3];
                }
                if (src[ii][4]) T[2][tx][i] = acc[ii][4];
                if (src[ii][5]) T[3][i][tx] = acc[ii][5];
            }
        }
        __syncthreads();
        // outputs K(a, b) at dst[b p + a]: lanes along a (coalesced)
        for (int j = ty; j < kRedTile; j += 8) {
            const int a = a0 + tx, b = b0 + j;
            if (a < p && b < p) {
                const int e = b * p + a;
                float2 k = make_float2(0.f, 0.f);
                if (n > 0) k = make_float2((T[0][tx][j] + T[1][tx][j]) * inv, (T[3][tx][j] - T[2][tx][j]) * inv);
                float2 out;
                if (mode == kRedT) {
                    const float2 t = dst[e];
                    out = make_float2(k.x - fa * t.x, k.y - fa * t.y);
                } else {
                    float2 base;
                    if (mode == kRedB) base = pwls ? make_float2(a == b ? 1.f : 0.f, 0.f) : J.R32[e];
                    else base = pwls ? J.Ri32[e] : J.R32[e];
                    out = make_float2(base.x + k.x, base.y + k.y);
                }
                dst[e] = out;
                mx = fmaxf(mx, fmaxf(fabsf(out.x), fabsf(out.y)));
                ss = fmaf(out.x, out.x, fmaf(out.y, out.y, ss));
            }
        }
        __syncthreads();
    }
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&ctl->mx_t, __float_as_uint(mx));
    if (mode == kRedG) return;
    // this CTA's share of ||W0||^2 (FP64); k_ws_vx adds the shares in CTA order
    __shared__ double sbuf[kWsThreads / 32];
    const double cs = block_sum((double)ss, sbuf);
    if (threadIdx.x == 0) ctl->sums[blockIdx.x] = cs;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->nsums = gridDim.x;
}

// Adjoint over the free list (LIST) or over every pixel (gradient): unit
// partial dots into padj[row * ld_adj + u] (u: unit, or unit x K group).
template <bool BF16, bool LIST>
__global__ void __launch_bounds__(kWideThreads, 1) k_ws_adj(const JobDev *Jp, WsBufs B) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    if (ctl->stop) return;
    const UnitGeom g = unit_geom(J.p);
    const int n = LIST ? ctl->f : J.Q;
    if (n <= 0) return;
    const int ntiles = LIST ? (n + kTcM - 1) / kTcM : tc_num_tiles(J.n_l, J.n_m);
    const int nkg = LIST ? ws_nkg(ntiles * g.nu, g.nk, gridDim.x) : 1;
    if (LIST && blockIdx.x == 0 && threadIdx.x == 0) ctl->adj_rows = g.nu * nkg;
    extern __shared__ float4 smem4[];
    unsigned char *dyn = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem4) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bars[kWideBars];
    __shared__ uint32_t tslot;
    float *out = B.padj;
    const int ld = B.ld_adj;
    const bool sq = !LIST && ctl->adj_sq;
    const int to = items_adjoint<BF16, LIST>(
        J, g, dyn, bars, &tslot, B.bimg, B.ximgF, J.cvec, J.fpos, n, ntiles, nkg, blockIdx.x, gridDim.x, sq,
        [&](int u, int t, int r, float v) {
            if (LIST) {
                const int j = t * kTcM + r;
                if (j < n) out[(size_t)j * ld + u] = v;
            } else {
                const int i = tc_tile_pixel(t, r, J.n_l, J.n_m);
                if (i >= 0) out[(size_t)i * ld + u] = v;
            }
        });
    if (to && threadIdx.x == 0) {
        // a broken pipeline ends the solve: every later kernel sees stop
        atomicAdd(&ctl->timeouts, to);
        ctl->stop = 1;
    }
}

// ---------------------------------------------------------------- LSQR vectors
// One CTA of kVxThreads threads per Golub-Kahan half step on the f-vectors:
//   beta = ||t|| from the CTA shares of the reduction (FP64, in CTA order),
//   us = 1/beta; (init: ||b|| = beta; else ||B||^2 += alpha^2 + beta^2);
//   v <- s_F (M^H u) - beta v  (init: v <- s_F M^H u), M^H u = us times the
//   adjoint's unit (x K group) partial dots;  alpha = ||v||;
//   the plane rotation (FP64); v <- v / alpha; init: w = v, x = 0; else
//   x += t1 w, w = v + t2 w; the weights s_F v of the next forward and their
//   maximum; ||x|| and the Paige-Saunders stopping tests; h_lsqr := continue.
constexpr int kVxThreads = 256;

__device__ __forceinline__ double vx_sum(double v, double *sb) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sb[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll 8
    for (int w = 0; w < kVxThreads / 32; ++w) t += sb[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(kVxThreads) k_ws_vx(const JobDev *Jp, WsBufs B, int init,
                                                       cudaGraphConditionalHandle h_lsqr) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    __shared__ double sb[kVxThreads / 32];
    __shared__ float swm[kVxThreads / 32];
    if (ctl->stop) {
        if (threadIdx.x == 0) ws_cond(ctl, kCondLsqr, h_lsqr, 0u);
        return;
    }
    const int f = ctl->f, ld = B.ld_adj, rows = ctl->adj_rows;
    // beta from the reduction's CTA shares
    double part = 0.0;
    for (int b = threadIdx.x; b < ctl->nsums; b += blockDim.x) part += ctl->sums[b];
    const double beta = sqrt(vx_sum(part, sb));
    const double us = beta > 0.0 ? 1.0 / beta : 0.0;
    const double alpha_prev = ctl->alpha;
    const float sc = 1.f / (ctl->sXF * ctl->sB);
    const float fus = (float)us, fb = (float)beta;
    float ss = 0.f;
    const int r4 = rows >> 2;
    float *__restrict__ vv = J.v;
    const float *__restrict__ sF = J.sF;
    // two rows per thread per step: every load of both rows is in flight
    // before the sums (rows <= nu nk <= 36 partial dots, 9 float4)
    for (int j0 = threadIdx.x; j0 < f; j0 += 2 * blockDim.x) {
        float4 s4[2][9];
        float vo[2], sf[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + h * blockDim.x;
            const bool ok = j < f;
            const float4 *pr = reinterpret_cast<const float4 *>(B.padj + (size_t)(ok ? j : 0) * ld);
#pragma unroll
            for (int q = 0; q < 9; ++q) s4[h][q] = (ok && q < r4) ? pr[q] : make_float4(0.f, 0.f, 0.f, 0.f);
            sf[h] = ok ? sF[j] : 0.f;
            vo[h] = (ok && !init) ? vv[j] : 0.f;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int j = j0 + h * blockDim.x;
            if (j >= f) continue;
            float y = 0.f;
#pragma unroll
            for (int q = 0; q < 9; ++q) y += (s4[h][q].x + s4[h][q].y) + (s4[h][q].z + s4[h][q].w);
            for (int u = 4 * r4; u < rows; ++u) y += B.padj[(size_t)j * ld + u];
            y *= sc;
            const float vn = init ? sf[h] * (y * fus) : sf[h] * (y * fus) - fb * vo[h];
            vv[j] = vn;
            ss = fmaf(vn, vn, ss);
        }
    }
    const double alpha = sqrt(vx_sum((double)ss, sb));
    double rhobar = ctl->rhobar, phibar = ctl->phibar, anorm2 = ctl->anorm2, t1 = 0.0, t2 = 0.0, absc = 0.0;
    if (init) {
        phibar = beta;
        rhobar = alpha;
        anorm2 = 0.0;
    } else {
        anorm2 += alpha_prev * alpha_prev + beta * beta;
        const double rho = hypot(rhobar, beta);
        const double c = rhobar / rho, sn = beta / rho;
        const double theta = sn * alpha;
        rhobar = -c * alpha;
        const double phi = c * phibar;
        phibar = sn * phibar;
        t1 = phi / rho;
        t2 = -theta / rho;
        absc = fabs(c);
    }
    const float ia = alpha > 0.0 ? (float)(1.0 / alpha) : 1.f, ft1 = (float)t1, ft2 = (float)t2;
    float xs2 = 0.f, wm = 0.f;
#pragma unroll 4
    for (int j = threadIdx.x; j < f; j += blockDim.x) {
        const float vj = J.v[j] * ia;
        J.v[j] = vj;
        if (init) {
            J.w[j] = vj;
            J.xs[j] = 0.f;
        } else {
            const float xj = J.xs[j] + ft1 * J.w[j];
            J.xs[j] = xj;
            J.w[j] = vj + ft2 * J.w[j];
            xs2 = fmaf(xj, xj, xs2);
        }
        const float wv = J.sF[j] * vj;
        B.wl[j] = wv;
        wm = fmaxf(wm, fabsf(wv));
    }
    const double xnorm2 = vx_sum((double)xs2, sb);
    for (int o = 16; o; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, o));
    if ((threadIdx.x & 31) == 0) swm[threadIdx.x >> 5] = wm;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < kVxThreads / 32; ++w) wm = fmaxf(wm, swm[w]);
        ctl->mx_w = __float_as_uint(wm);
        ctl->mx_t = 0u;                       // the image of t is consumed
        ctl->beta = beta;
        ctl->us = us;
        ctl->alpha = alpha;
        ctl->rhobar = rhobar;
        ctl->phibar = phibar;
        ctl->anorm2 = anorm2;
        bool more;
        if (init) {
            ctl->bnorm = beta;
            more = alpha > 0.0 && beta > 0.0 && ctl->maxit >= 1;
        } else {
            ctl->it++;
            const double xnorm = sqrt(xnorm2);
            const double rnorm = phibar;
            const double arnorm = phibar * alpha * absc;
            const double anorm = sqrt(anorm2);
            more = ctl->it < ctl->maxit;
            if (rnorm <= J.lsqr_btol * ctl->bnorm + J.lsqr_atol * anorm * xnorm) more = false;
            if (arnorm <= J.lsqr_atol * anorm * rnorm) more = false;
        }
        // the next forward: t <- M v - alpha u with u = t us, so fa = alpha us
        ctl->fa = alpha * us;
        ctl->nlist = f;
        ctl->nsplit = ws_nsplit(f, B.npairs, B.max_tasks, B.fwd_per);
        ws_cond(ctl, kCondLsqr, h_lsqr, more ? 1u : 0u);
    }
}

// ---------------------------------------------------------------- feasibility
// After the subproblem: count its LSQR iterations, test 0 <= z <= u with the
// relative tolerance (non-strict, Table I); h_feas := feasible.
__global__ void k_ws_feas(const JobDev *Jp, WsBufs B, cudaGraphConditionalHandle h_feas) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    __shared__ int s_stop;
    if (threadIdx.x == 0) s_stop = ctl->stop;
    __syncthreads();
    if (s_stop) {
        if (threadIdx.x == 0) ws_cond(ctl, kCondFeas, h_feas, 0u);
        return;
    }
    const int f = ctl->f;
    int bad = 0;
    const double tau = J.feas_tol;
    for (int j = threadIdx.x; j < f; j += blockDim.x) {
        const double z = J.xs[j];
        const double u = J.upper[J.supp[J.fpos[j]]];
        if (!(z >= -tau * u && z <= (1.0 + tau) * u)) bad = 1;
    }
    const bool feasible = __syncthreads_or(bad) == 0;
    if (threadIdx.x == 0) {
        if (f > 0) {
            const int its = min(ctl->it, ctl->maxit);
            ctl->lsqr_total += its;
            ctl->op_flops += (its + 1) * (ws_flops_fwd(J.p, f) + ws_flops_adj(J.p, f));
        }
        ctl->feasible = feasible ? 1 : 0;
        ws_cond(ctl, kCondFeas, h_feas, feasible ? 1u : 0u);
    }
}

// Feasible: x_F = clip(z, 0, u); the support weights -s_i x_i for the
// gradient's residual, their maximum, the support list scale; reset the
// argmin key.
__global__ void k_ws_accept(const JobDev *Jp, WsBufs B) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    if (ctl->stop) return;
    const int f = ctl->f, ns = ctl->ns;
    for (int j = threadIdx.x; j < f; j += blockDim.x) {
        const int i = J.supp[J.fpos[j]];
        J.x[i] = fmin(fmax((double)J.xs[j], 0.0), J.upper[i]);
    }
    __syncthreads();
    float wm = 0.f;
    for (int j = threadIdx.x; j < ns; j += blockDim.x) {
        const int i = J.supp[j];
        const float wv = -J.scale[i] * (float)J.x[i];
        B.wl[j] = wv;
        wm = fmaxf(wm, fabsf(wv));
    }
    const float mS = ws_list_max(J.cost == IMG_COST_PWLS ? B.dmax : J.cmax, nullptr, ns);
    __shared__ float swm[kWsThreads / 32];
    for (int o = 16; o; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, o));
    if ((threadIdx.x & 31) == 0) swm[threadIdx.x >> 5] = wm;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < kWsThreads / 32; ++w) wm = fmaxf(wm, swm[w]);
        ctl->mx_w = __float_as_uint(wm);
        ctl->sXS = pow2_scale(mS) * kLift;
        ctl->nlist = ns;
        ctl->nsplit = ws_nsplit(ns, B.npairs, B.max_tasks, B.fwd_per);
        ctl->key = ~0ull;
        ctl->op_flops += ws_flops_fwd(J.p, ns) + ws_flops_adj(J.p, J.Q);
    }
}

// Gradient g_i = -s_i Re(a_i^H U_g a_i) (eq. gls / eq. gmvdr) from the unit
// partial dots; lambda_L = g, lambda_U = -g (eq. etaL, eq. etaU); candidates
// lambda_i < -eps_i off F; smallest lambda, ties to the smallest pixel.
__global__ void k_ws_grad(const JobDev *Jp, WsBufs B) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    if (ctl->stop) return;
    const UnitGeom g = unit_geom(J.p);
    const float sc = 1.f / (steer_scale(J.p) * kLift * ctl->sB);
    const int ld = B.ld_adj;
    unsigned long long best = ~0ull;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < J.Q; i += gridDim.x * blockDim.x) {
        float y = 0.f;
        for (int u = 0; u < g.nu; ++u) y += B.padj[(size_t)i * ld + u];
        const float gv = -J.scale[i] * (y * sc);
        J.grad[i] = gv;
        const unsigned char st = J.set[i];
        if (st != IMG_SET_F) {
            const float lam = st == IMG_SET_U ? -gv : gv;
            if (lam < -J.eps[i]) {
                const unsigned long long k = key_of(lam, i);
                best = k < best ? k : best;
            }
        }
    }
    for (int o = 16; o; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        best = ob < best ? ob : best;
    }
    if ((threadIdx.x & 31) == 0 && best != ~0ull) atomicMin(&ctl->key, best);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->mx_t = 0u;
}

__global__ void k_ws_decide(const JobDev *Jp, WsBufs B) {
    ws_count(B.ctl);
    WsCtl *ctl = B.ctl;
    if (threadIdx.x != 0 || ctl->stop) return;
    const unsigned long long k = ctl->key;
    if (k == ~0ull) {
        ctl->converged = 1;
        ctl->stop = 1;
        ctl->lam_min = INFINITY;
    } else {
        ctl->pending = (int)(k & 0xffffffffu);
        ctl->lam_min = (double)lam_of(k);
    }
}

// Infeasible: step towards z (eq. mumax), smallest pixel index on ties; the
// blocking pixel goes to U when its direction is positive, to L otherwise,
// exactly at its bound, and leaves the support when it goes to L.
__global__ void k_ws_step(const JobDev *Jp, WsBufs B) {
    ws_count(B.ctl);
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    __shared__ double sv[kWsThreads / 32];
    __shared__ int si[kWsThreads / 32];
    __shared__ int s_stop;
    if (threadIdx.x == 0) s_stop = ctl->stop;
    __syncthreads();
    if (s_stop) return;
    const int f = ctl->f;
    int ns = ctl->ns;
    double best = INFINITY;
    int bidx = 0x7fffffff;
    for (int j = threadIdx.x; j < f; j += blockDim.x) {
        const int i = J.supp[J.fpos[j]];
        const double xi = J.x[i];
        const double pd = (double)J.xs[j] - xi;
        double mu = INFINITY;
        if (pd > 0.0) mu = (J.upper[i] - xi) / pd;
        else if (pd < 0.0) mu = -xi / pd;
        if (mu < best || (mu == best && i < bidx)) { best = mu; bidx = i; }
    }
    block_argmin(best, bidx, sv, si);
    const double mu = best;
    const int ic = bidx;
    int dirup = 0;
    for (int j = threadIdx.x; j < f; j += blockDim.x)
        if (J.supp[J.fpos[j]] == ic) dirup = ((double)J.xs[j] - J.x[ic] > 0.0) ? 1 : 0;
    const bool up = __syncthreads_or(dirup) != 0;
    for (int j = threadIdx.x; j < f; j += blockDim.x) {
        const int i = J.supp[J.fpos[j]];
        const double xi = J.x[i];
        J.x[i] = xi + mu * ((double)J.xs[j] - xi);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        J.set[ic] = up ? IMG_SET_U : IMG_SET_L;
        J.x[ic] = up ? J.upper[ic] : 0.0;
        ws_log(J, ctl, up ? 2 : 1, ic, (float)mu);
    }
    __syncthreads();
    if (!up) ws_remove(J, B, ic, ns);
    if (threadIdx.x == 0) ctl->ns = ns;
}


// ---------------------------------------------------------------- bounds
// Dirty image and MVDR denominators (Sec. III-C, III-D) on the work-item
// adjoint: out_i = Re(a_i^H U a_i) for U = R_hat and U = R_hat^-1 over every
// pixel, from the unit image of U.  k_ws_bnd_max readies the control block
// (no solve runs on the context meanwhile) and reduces max |U|;
// k_ws_bnd_out sums each pixel's unit partial dots.
__global__ void k_ws_bnd_max(const JobDev *Jp, WsBufs B, const float2 *U, int first, int sq) {
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctl->adj_sq = sq;
    if (first && blockIdx.x == 0 && threadIdx.x == 0) {
        // bounds (first = 1): a failed factor leaves them alone; the
        // stand-alone adjoint (first = 2) does not depend on the factor
        ctl->stop = first == 1 && J.flags[0] != 0 ? 1 : 0;
        ctl->timeouts = 0;
    }
    const int pp = J.p * J.p;
    float mx = 0.f;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < pp; e += gridDim.x * blockDim.x)
        mx = fmaxf(mx, fmaxf(fabsf(U[e].x), fabsf(U[e].y)));
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&ctl->mx_t, __float_as_uint(mx));
}

__global__ void k_ws_bnd_out(const JobDev *Jp, WsBufs B, float *out) {
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    if (ctl->timeouts && blockIdx.x == 0 && threadIdx.x == 0) J.flags[2] = IMG_ETIMEOUT;
    if (ctl->stop) return;
    const UnitGeom g = unit_geom(J.p);
    const float s1 = steer_scale(J.p) * kLift * ctl->sB;
    const float sc = ctl->adj_sq ? 1.f / (s1 * s1) : 1.f / s1;
    const int ld = B.ld_adj;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < J.Q; i += gridDim.x * blockDim.x) {
        float y = 0.f;
        for (int u = 0; u < g.nu; ++u) y += B.padj[(size_t)i * ld + u];
        out[i] = y * sc;
    }
}

__global__ void k_ws_adj_out(const JobDev *Jp, WsBufs B, double *out) {
    const JobDev &J = *Jp;
    WsCtl *ctl = B.ctl;
    if (ctl->stop) return;
    const UnitGeom g = unit_geom(J.p);
    const float sc = 1.f / (steer_scale(J.p) * kLift * ctl->sB);
    const int ld = B.ld_adj;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < J.Q; i += gridDim.x * blockDim.x) {
        float y = 0.f;
        for (int u = 0; u < g.nu; ++u) y += B.padj[(size_t)i * ld + u];
        out[i] = (double)(y * sc);
    }
}

__global__ void k_ws_bnd_reset(WsBufs B) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        B.ctl->mx_t = 0u;
        B.ctl->adj_sq = 0;                    // the solve's adjoints are dots
    }
}

// ================================================================ host side
namespace {

template <class K>
cudaError_t set_smem(K kern, size_t bytes) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

struct Cap {
    cudaStream_t st;
    cudaGraph_t g;
    cudaError_t err = cudaSuccess;
    // begin a capture into g after dependency dep (null: none)
    void begin(cudaGraph_t graph, cudaGraphNode_t dep) {
        g = graph;
        if (err == cudaSuccess)
            err = cudaStreamBeginCaptureToGraph(st, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0,
                                                cudaStreamCaptureModeRelaxed);
    }
    // end the capture; returns the last captured node
    cudaGraphNode_t end() {
        cudaGraphNode_t leaf = nullptr;
        if (err == cudaSuccess) {
            cudaStreamCaptureStatus cs;
            const cudaGraphNode_t *deps = nullptr;
            size_t nd = 0;
            err = cudaStreamGetCaptureInfo(st, &cs, nullptr, nullptr, &deps, nullptr, &nd);
            if (err == cudaSuccess && nd == 1) leaf = deps[0];
        }
        cudaGraph_t out = nullptr;
        const cudaError_t e = cudaStreamEndCapture(st, &out);
        if (err == cudaSuccess) err = e;
        if (err == cudaSuccess && !leaf) err = cudaErrorStreamCaptureInvalidated;
        return leaf;
    }
    void check() {
        if (err == cudaSuccess) err = cudaGetLastError();
    }
};

cudaGraphNode_t add_cond(Cap &c, cudaGraph_t g, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                         int size, cudaGraphNode_t dep, cudaGraph_t *bodies) {
    if (c.err != cudaSuccess) return nullptr;
    cudaGraphNodeParams prm = {};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = h;
    prm.conditional.type = type;
    prm.conditional.size = (unsigned)size;
    cudaGraphNode_t node = nullptr;
    c.err = cudaGraphAddNode(&node, g, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &prm);
    if (c.err == cudaSuccess)
        for (int i = 0; i < size; ++i) bodies[i] = prm.conditional.phGraph_out[i];
    return node;
}

}  // namespace

struct WsHost {
    int device = 0;
    int bf16 = 0;
    int direct = 0;             // host-driven loop instead of the graph
    int sms = 1;
    unsigned *h_cond = nullptr; // pinned mirror of the conditions
    const JobDev *dj = nullptr;
    int p = 0, cap = 0, Q = 0;
    UnitGeom g{};
    void *mem = nullptr;
    WsBufs B{};
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

size_t ws_bytes(const JobDev &hj, int sms, WsBufs *B, char *base) {
    const UnitGeom g = unit_geom(hj.p);
    const int cap = hj.cap, p = hj.p;
    size_t off = 0;
    auto take = [&](size_t n) {
        off = (off + 1023) & ~size_t(1023);
        char *r = base ? base + off : nullptr;
        off += n;
        return r;
    };
    WsBufs b{};
    b.npairs = items_fwd_pairs(g, b.pm, b.pnb);
    b.max_tasks = std::max(b.npairs, 2 * std::min(sms, kListGrid));
    b.fwd_per = kFwdPerTask;
    b.nrows_adj = std::max(hj.Q, cap);
    b.ld_adj = (g.nu * g.nk + 3) / 4 * 4;    // a multiple of 4: rows read as float4
    b.ctl = reinterpret_cast<WsCtl *>(take(sizeof(WsCtl)));
    b.dvec = hj.cost == IMG_COST_PWLS ? reinterpret_cast<float2 *>(take((size_t)cap * p * sizeof(float2))) : nullptr;
    b.dmax = reinterpret_cast<float *>(take((size_t)cap * sizeof(float)));
    b.iota = reinterpret_cast<int *>(take((size_t)cap * sizeof(int)));
    b.wl = reinterpret_cast<float *>(take((size_t)cap * sizeof(float)));
    b.padj = reinterpret_cast<float *>(take((size_t)b.ld_adj * b.nrows_adj * sizeof(float)));
    b.pfwd = reinterpret_cast<float *>(take((size_t)b.max_tasks * kTcM * 256 * sizeof(float)));
    b.ximgF = reinterpret_cast<unsigned char *>(take(list_image_bytes(g, cap)));
    b.ximgS = reinterpret_cast<unsigned char *>(take(list_image_bytes(g, cap)));
    b.ximgW = reinterpret_cast<unsigned char *>(take(list_image_bytes(g, cap)));
    b.bimg = reinterpret_cast<unsigned char *>(take(unit_image_bytes(g)));
    if (B) *B = b;
    return off + 1024;
}

template <bool BF>
static cudaError_t ws_capture(WsHost *w, const JobDev *dj, const JobDev &hj, int sms) {
    const WsBufs &B = w->B;
    Cap c{};
    cudaStreamCreateWithFlags(&c.st, cudaStreamNonBlocking);
    cudaGraph_t G = nullptr;
    c.err = cudaGraphCreate(&G, 0);
    cudaGraphConditionalHandle h_outer = 0, h_lif = 0, h_lsqr = 0, h_feas = 0;
    if (c.err == cudaSuccess) c.err = cudaGraphConditionalHandleCreate(&h_outer, G, 1, cudaGraphCondAssignDefault);
    if (c.err == cudaSuccess) c.err = cudaGraphConditionalHandleCreate(&h_lif, G, 0, 0);
    if (c.err == cudaSuccess) c.err = cudaGraphConditionalHandleCreate(&h_lsqr, G, 0, 0);
    if (c.err == cudaSuccess) c.err = cudaGraphConditionalHandleCreate(&h_feas, G, 0, 0);
    const size_t fsm = items_fwd_smem_bytes(), asm_ = items_smem_bytes();
    if (c.err == cudaSuccess) c.err = set_smem(k_ws_fwd<BF>, fsm);
    if (c.err == cudaSuccess) c.err = set_smem(k_ws_adj<BF, true>, asm_);
    if (c.err == cudaSuccess) c.err = set_smem(k_ws_adj<BF, false>, asm_);
    const int ntr = (hj.p + kRedTile - 1) / kRedTile;
    const int g_red = std::min(ntr * ntr, kWsSums);
    const int g_grad = std::min((hj.Q + kWsThreads - 1) / kWsThreads, 4 * sms);
    const int g_img = sms;
    const int g_cache = (hj.p + kCacheRows - 1) / kCacheRows;
    const int g_fwd = std::min(sms, kListGrid), g_adj = std::min(sms, kListGrid);
    cudaStream_t s = c.st;
    // top level: start, the Table I loop, finish
    c.begin(G, nullptr);
    k_ws_start<<<1, kWsThreads, 0, s>>>(dj, B, h_outer);
    c.check();
    cudaGraphNode_t n0 = c.end();
    cudaGraph_t ob[1] = {};
    cudaGraphNode_t nw = add_cond(c, G, h_outer, cudaGraphCondTypeWhile, 1, n0, ob);
    c.begin(G, nw);
    k_ws_finish<<<1, kWsThreads, 0, s>>>(dj, B);
    c.check();
    c.end();
    // one loop iteration: free the pending pixel, subproblem, branch
    c.begin(ob[0], nullptr);
    k_ws_free<<<1, 32, 0, s>>>(dj, B);
    k_ws_cache<<<g_cache, kWsThreads, 0, s>>>(dj, B);
    k_ws_pass<<<1, kWsThreads, 0, s>>>(dj, B, h_lif);
    c.check();
    cudaGraphNode_t n1 = c.end();
    cudaGraph_t lb[1] = {};
    cudaGraphNode_t nif = add_cond(c, ob[0], h_lif, cudaGraphCondTypeIf, 1, n1, lb);
    // LSQR on F (Sec. V-A): data b, initialisation, iterations
    c.begin(lb[0], nullptr);
    k_ws_listimg<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, kListF, 0);
    k_ws_listimg<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, kListU, 0);
    k_ws_listimg<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, kListU, 1);
    k_ws_fwd<BF><<<g_fwd, kItemsFwdThreads, fsm, s>>>(dj, B, kListU);
    k_ws_fred<<<g_red, kWsThreads, 0, s>>>(dj, B, kRedB);
    k_ws_emb<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, 0, nullptr);
    k_ws_adj<BF, true><<<g_adj, kWideThreads, asm_, s>>>(dj, B);
    k_ws_vx<<<1, kVxThreads, 0, s>>>(dj, B, 1, h_lsqr);
    c.check();
    cudaGraphNode_t n2 = c.end();
    cudaGraph_t wb[1] = {};
    add_cond(c, lb[0], h_lsqr, cudaGraphCondTypeWhile, 1, n2, wb);
    c.begin(wb[0], nullptr);
    k_ws_listimg<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, kListF, 1);
    k_ws_fwd<BF><<<g_fwd, kItemsFwdThreads, fsm, s>>>(dj, B, kListF);
    k_ws_fred<<<g_red, kWsThreads, 0, s>>>(dj, B, kRedT);
    k_ws_emb<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, 0, nullptr);
    k_ws_adj<BF, true><<<g_adj, kWideThreads, asm_, s>>>(dj, B);
    k_ws_vx<<<1, kVxThreads, 0, s>>>(dj, B, 0, h_lsqr);
    c.check();
    c.end();
    // feasibility, then the gradient (feasible) or the step (infeasible)
    c.begin(ob[0], nif);
    k_ws_feas<<<1, kWsThreads, 0, s>>>(dj, B, h_feas);
    c.check();
    cudaGraphNode_t n3 = c.end();
    cudaGraph_t fb[2] = {};
    cudaGraphNode_t nfe = add_cond(c, ob[0], h_feas, cudaGraphCondTypeIf, 2, n3, fb);
    c.begin(fb[0], nullptr);
    k_ws_accept<<<1, kWsThreads, 0, s>>>(dj, B);
    k_ws_listimg<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, kListS, 0);
    k_ws_listimg<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, kListS, 1);
    k_ws_fwd<BF><<<g_fwd, kItemsFwdThreads, fsm, s>>>(dj, B, kListS);
    k_ws_fred<<<g_red, kWsThreads, 0, s>>>(dj, B, kRedG);
    k_ws_emb<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, 1, nullptr);
    k_ws_adj<BF, false><<<sms, kWideThreads, asm_, s>>>(dj, B);
    k_ws_grad<<<g_grad, kWsThreads, 0, s>>>(dj, B);
    k_ws_decide<<<1, 32, 0, s>>>(dj, B);
    c.check();
    c.end();
    c.begin(fb[1], nullptr);
    k_ws_step<<<1, kWsThreads, 0, s>>>(dj, B);
    c.check();
    c.end();
    c.begin(ob[0], nfe);
    k_ws_end<<<1, 32, 0, s>>>(dj, B, h_outer);
    c.check();
    c.end();
    if (c.err == cudaSuccess) c.err = cudaGraphInstantiate(&w->exec, G, 0);
    w->graph = G;
    cudaStreamDestroy(c.st);
    return c.err;
}

// The solve with the loop and branches taken on the host: the same kernels in
// the same order as the graph, with a stream synchronisation wherever the
// graph tests a condition.  For tools that cannot look inside graphs with
// conditional nodes (kernel profilers); the results are the same.
template <bool BF>
static cudaError_t ws_direct(WsHost *w, cudaStream_t s) {
    const WsBufs &B = w->B;
    const JobDev *dj = w->dj;
    const int sms = w->sms;
    const size_t fsm = items_fwd_smem_bytes(), asm_ = items_smem_bytes();
    const int ntr = (w->p + kRedTile - 1) / kRedTile;
    const int g_red = std::min(ntr * ntr, kWsSums);
    const int g_grad = std::min((w->Q + kWsThreads - 1) / kWsThreads, 4 * sms);
    const int g_img = sms;
    const int g_cache = (w->p + kCacheRows - 1) / kCacheRows;
    const int g_fwd = std::min(sms, kListGrid), g_adj = std::min(sms, kListGrid);
    cudaError_t e = cudaSuccess;
    auto cond = [&](int which) -> unsigned {
        if (e == cudaSuccess) e = cudaMemcpyAsync(w->h_cond, &B.ctl->cond[0], 4 * sizeof(unsigned),
                                                  cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? w->h_cond[which] : 0u;
    };
    k_ws_start<<<1, kWsThreads, 0, s>>>(dj, B, 0);
    while (cond(kCondOuter)) {
        k_ws_free<<<1, 32, 0, s>>>(dj, B);
        k_ws_cache<<<g_cache, kWsThreads, 0, s>>>(dj, B);
        k_ws_pass<<<1, kWsThreads, 0, s>>>(dj, B, 0);
        if (cond(kCondLsqrIf)) {
            k_ws_listimg<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, kListF, 0);
            k_ws_listimg<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, kListU, 0);
            k_ws_listimg<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, kListU, 1);
            k_ws_fwd<BF><<<g_fwd, kItemsFwdThreads, fsm, s>>>(dj, B, kListU);
            k_ws_fred<<<g_red, kWsThreads, 0, s>>>(dj, B, kRedB);
            k_ws_emb<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, 0, nullptr);
            k_ws_adj<BF, true><<<g_adj, kWideThreads, asm_, s>>>(dj, B);
            k_ws_vx<<<1, kVxThreads, 0, s>>>(dj, B, 1, 0);
            while (cond(kCondLsqr)) {
                k_ws_listimg<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, kListF, 1);
                k_ws_fwd<BF><<<g_fwd, kItemsFwdThreads, fsm, s>>>(dj, B, kListF);
                k_ws_fred<<<g_red, kWsThreads, 0, s>>>(dj, B, kRedT);
                k_ws_emb<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, 0, nullptr);
                k_ws_adj<BF, true><<<g_adj, kWideThreads, asm_, s>>>(dj, B);
                k_ws_vx<<<1, kVxThreads, 0, s>>>(dj, B, 0, 0);
            }
        }
        k_ws_feas<<<1, kWsThreads, 0, s>>>(dj, B, 0);
        if (cond(kCondFeas)) {
            k_ws_accept<<<1, kWsThreads, 0, s>>>(dj, B);
            k_ws_listimg<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, kListS, 0);
            k_ws_listimg<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, kListS, 1);
            k_ws_fwd<BF><<<g_fwd, kItemsFwdThreads, fsm, s>>>(dj, B, kListS);
            k_ws_fred<<<g_red, kWsThreads, 0, s>>>(dj, B, kRedG);
            k_ws_emb<BF><<<g_img, kWsThreads, 0, s>>>(dj, B, 1, nullptr);
            k_ws_adj<BF, false><<<sms, kWideThreads, asm_, s>>>(dj, B);
            k_ws_grad<<<g_grad, kWsThreads, 0, s>>>(dj, B);
            k_ws_decide<<<1, 32, 0, s>>>(dj, B);
        } else {
            k_ws_step<<<1, kWsThreads, 0, s>>>(dj, B);
        }
        k_ws_end<<<1, 32, 0, s>>>(dj, B, 0);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) break;
    }
    k_ws_finish<<<1, kWsThreads, 0, s>>>(dj, B);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

// Every kernel of the solve with the largest shared-memory carveout, so the
// SMs need no reconfiguration between the tensor-core kernels (near 200 KB
// of shared memory each) and the small ones in between.
template <bool BF>
static cudaError_t ws_carveout() {
    const int c = cudaSharedmemCarveoutMaxShared;
    const void *ks[] = {(const void *)k_ws_start, (const void *)k_ws_end, (const void *)k_ws_finish,
                        (const void *)k_ws_free, (const void *)k_ws_cache,
                        (const void *)k_ws_pass, (const void *)k_ws_listimg<BF>, (const void *)k_ws_emb<BF>,
                        (const void *)k_ws_fwd<BF>, (const void *)k_ws_fred, (const void *)k_ws_adj<BF, true>,
                        (const void *)k_ws_adj<BF, false>, (const void *)k_ws_vx, (const void *)k_ws_feas,
                        (const void *)k_ws_accept, (const void *)k_ws_grad, (const void *)k_ws_decide,
                        (const void *)k_ws_step};
    for (const void *k : ks) {
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, c);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t ws_create(const JobDev &hj, const JobDev *dj, int mode, WsHost **out) {
    *out = nullptr;
    if (hj.p > kItemsMaxP || (mode != 1 && mode != 2)) return cudaErrorInvalidValue;
    WsHost *w = new WsHost();
    cudaGetDevice(&w->device);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, w->device);
    w->bf16 = mode == 2;
    w->g = unit_geom(hj.p);
    w->sms = sms;
    w->dj = dj;
    w->p = hj.p;
    w->cap = hj.cap;
    w->Q = hj.Q;
    {
        const char *env = getenv("IMG_SOLVE_GRAPH");
        w->direct = env && env[0] == '0';
    }
    const size_t bytes = ws_bytes(hj, sms, nullptr, nullptr);
    cudaError_t e = cudaMalloc(&w->mem, bytes);
    if (e != cudaSuccess) {
        delete w;
        return e;
    }
    char *base = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(w->mem) + 1023) & ~uintptr_t(1023));
    ws_bytes(hj, sms, &w->B, base);
    e = w->bf16 ? ws_carveout<true>() : ws_carveout<false>();
    if (e == cudaSuccess) e = set_smem(k_ws_adj<true, false>, items_smem_bytes());
    if (e == cudaSuccess) e = set_smem(k_ws_adj<false, false>, items_smem_bytes());
    if (e != cudaSuccess) {
        ws_destroy(w);
        return e;
    }
    if (w->direct) {
        e = cudaMallocHost(&w->h_cond, 4 * sizeof(unsigned));
        if (e == cudaSuccess) {
            // the attributes the graph build would set
            e = set_smem(k_ws_fwd<true>, items_fwd_smem_bytes());
            if (e == cudaSuccess) e = set_smem(k_ws_fwd<false>, items_fwd_smem_bytes());
            if (e == cudaSuccess) e = set_smem(k_ws_adj<true, true>, items_smem_bytes());
            if (e == cudaSuccess) e = set_smem(k_ws_adj<true, false>, items_smem_bytes());
            if (e == cudaSuccess) e = set_smem(k_ws_adj<false, true>, items_smem_bytes());
            if (e == cudaSuccess) e = set_smem(k_ws_adj<false, false>, items_smem_bytes());
        }
    } else {
        e = w->bf16 ? ws_capture<true>(w, dj, hj, sms) : ws_capture<false>(w, dj, hj, sms);
    }
    if (e != cudaSuccess) {
        ws_destroy(w);
        return e;
    }
    *out = w;
    return cudaSuccess;
}

cudaError_t ws_bounds(WsHost *w, const JobDev &hj, cudaStream_t st) {
    const WsBufs &B = w->B;
    const JobDev *dj = w->dj;
    const int sms = w->sms;
    const size_t asm_ = items_smem_bytes();
    const int gq = std::min((hj.Q + kWsThreads - 1) / kWsThreads, 4 * sms);
    for (int k = 0; k < 2; ++k) {
        // dirty image from R_hat; MVDR denominators ||L^-1 a||^2 from the B
        // image of L^-H (V = L^-1) with the sum-of-squares epilogue
        const float2 *U = k == 0 ? hj.R32 : hj.LiH32;
        k_ws_bnd_reset<<<1, 32, 0, st>>>(B);
        k_ws_bnd_max<<<sms, kWsThreads, 0, st>>>(dj, B, U, k == 0, k);
        if (w->bf16) {
            k_ws_emb<true><<<sms, kWsThreads, 0, st>>>(dj, B, 0, U);
            k_ws_adj<true, false><<<sms, kWideThreads, asm_, st>>>(dj, B);
        } else {
            k_ws_emb<false><<<sms, kWsThreads, 0, st>>>(dj, B, 0, U);
            k_ws_adj<false, false><<<sms, kWideThreads, asm_, st>>>(dj, B);
        }
        k_ws_bnd_out<<<gq, kWsThreads, 0, st>>>(dj, B, k == 0 ? hj.dirty : hj.h);
    }
    k_ws_bnd_reset<<<1, 32, 0, st>>>(B);
    return cudaGetLastError();
}

cudaError_t ws_psi_adj(WsHost *w, const JobDev &hj, const float2 *U, double *out, cudaStream_t st) {
    const WsBufs &B = w->B;
    const JobDev *dj = w->dj;
    const int sms = w->sms;
    const size_t asm_ = items_smem_bytes();
    const int gq = std::min((hj.Q + kWsThreads - 1) / kWsThreads, 4 * sms);
    k_ws_bnd_reset<<<1, 32, 0, st>>>(B);
    k_ws_bnd_max<<<sms, kWsThreads, 0, st>>>(dj, B, U, 2, 0);
    if (w->bf16) {
        k_ws_emb<true><<<sms, kWsThreads, 0, st>>>(dj, B, 0, U);
        k_ws_adj<true, false><<<sms, kWideThreads, asm_, st>>>(dj, B);
    } else {
        k_ws_emb<false><<<sms, kWsThreads, 0, st>>>(dj, B, 0, U);
        k_ws_adj<false, false><<<sms, kWideThreads, asm_, st>>>(dj, B);
    }
    k_ws_adj_out<<<gq, kWsThreads, 0, st>>>(dj, B, out);
    k_ws_bnd_reset<<<1, 32, 0, st>>>(B);
    return cudaGetLastError();
}

cudaError_t ws_launch(WsHost *w, cudaStream_t st) {
    if (w->direct) return w->bf16 ? ws_direct<true>(w, st) : ws_direct<false>(w, st);
    return cudaGraphLaunch(w->exec, st);
}

size_t ws_size(const JobDev &hj) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return ws_bytes(hj, sms, nullptr, nullptr);
}

void ws_destroy(WsHost *w) {
    if (!w) return;
    if (w->exec) cudaGraphExecDestroy(w->exec);
    if (w->graph) cudaGraphDestroy(w->graph);
    if (w->mem) cudaFree(w->mem);
    if (w->h_cond) cudaFreeHost(w->h_cond);
    delete w;
}

}  // namespace img
