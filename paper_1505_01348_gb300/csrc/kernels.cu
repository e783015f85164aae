// Kernels of the bounded least-squares imager (SIMT FP32 operator path).
//
//   k_tables    separable steering tables (FP64 phase reduction + sincospi)
//   k_factor    Cholesky R = L L^H, L^-1 and R^-1 in FP64 (one CTA per job)
//   k_bounds    dirty image a^H R a and a^H R^-1 a over all pixels (many CTAs
//               per job), the adjoint operator with U = R_hat and R_hat^-1
//   k_finalize  MVDR bound, D, thresholds (Sec. III-D, Appendix A)
//   k_solve     persistent active-set + LSQR driver, one CTA per job
//               (Table I, Sec. V-A, Sec. V-B)
#include "cta_ops.cuh"
#include "tc_ops.cuh"
#include "tc_wide.cuh"

#include <mutex>
#include <unordered_map>
#include "../../include/img.h"

namespace img {

// ---------------------------------------------------------------- tables
// El[il*p+k] = p^{-1/2} exp(-j 2 pi x_k l_il / lam), Em[im*p+k] = exp(-j 2 pi y_k m_im / lam).
// The phase argument t is reduced to r = t - rint(t) in FP64 before sincospi,
// so phases of hundreds of turns keep full accuracy.
// Tables of one job by the threads [t0, t0 + nt) of the grid dimension used.
__device__ void tables_job(const JobDev &J, int t0, int nt) {
    const int p = J.p;
    const int total = p * (J.n_l + J.n_m);
    const double sc = rsqrt((double)p);
    for (int e = t0; e < total; e += nt) {
        const bool isl = e < p * J.n_l;
        const int e2 = isl ? e : e - p * J.n_l;
        const int g = e2 / p, k = e2 - g * p;
        const double coord = isl ? J.ant[3 * k + 0] : J.ant[3 * k + 1];
        const double dir = isl ? J.lg[g] : J.mg[g];
        const double t = coord * dir / J.lam;
        const double r = t - rint(t);
        double s, c;
        sincospi(2.0 * r, &s, &c);
        if (isl) J.El[e2] = make_float2((float)(c * sc), (float)(-s * sc));
        else J.Em[e2] = make_float2((float)c, (float)(-s));
    }
}

__global__ void k_tables(JobDev *const *jobs) {
    tables_job(*jobs[blockIdx.y], blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------- factor
// Right-looking Cholesky in FP64, then L^-1 by forward substitution (one
// column per thread) and R^-1 = L^-H L^-1.  Status 0 ok, IMG_ENOTPD else.
__device__ void factor_job(const JobDev &J) {
    const int p = J.p;
    double2 *L = J.L64;
    __shared__ int bad;
    if (threadIdx.x == 0) {
        bad = 0;
        if (J.Bmax) J.Bmax[0] = J.Bmax[1] = 0u;   // max |R|, |R^-1| of the wide bounds start at zero
    }
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) L[e] = J.R64[e];
    __syncthreads();
    for (int j = 0; j < p; ++j) {
        // every thread reads the pivot itself; bad is written only by thread 0
        const double d = L[(size_t)j * p + j].x;
        const bool ok = d > 0.0 && isfinite(d);
        if (!ok) {
            if (threadIdx.x == 0) bad = 1;
            break;
        }
        const double dj = sqrt(d);
        const double inv = 1.0 / dj;
        __syncthreads();
        if (threadIdx.x == 0) L[(size_t)j * p + j] = make_double2(dj, 0.0);
        for (int i = j + 1 + threadIdx.x; i < p; i += blockDim.x) {
            double2 v = L[(size_t)j * p + i];
            L[(size_t)j * p + i] = make_double2(v.x * inv, v.y * inv);
        }
        __syncthreads();
        // trailing update of the lower triangle: L[i,k] -= L[i,j] conj(L[k,j]), j < k <= i
        const int m = p - j - 1;
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            const int k = j + 1 + t / m, i = j + 1 + t % m;
            if (i < k) continue;
            const double2 prod = zmulc(L[(size_t)j * p + i], L[(size_t)j * p + k]);
            const double2 v = L[(size_t)k * p + i];
            L[(size_t)k * p + i] = make_double2(v.x - prod.x, v.y - prod.y);
        }
        __syncthreads();
    }
    __syncthreads();
    if (bad) {
        if (threadIdx.x == 0) J.flags[0] = IMG_ENOTPD;
        return;
    }
    // zero the strict upper triangle
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const int col = e / p, row = e - col * p;
        if (row < col) L[e] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    // X = L^-1, column c by one thread
    double2 *X = J.Li64;
    for (int c = threadIdx.x; c < p; c += blockDim.x) {
        for (int i = 0; i < c; ++i) X[(size_t)c * p + i] = make_double2(0.0, 0.0);
        for (int i = c; i < p; ++i) {
            double2 s = make_double2(i == c ? 1.0 : 0.0, 0.0);
            for (int k = c; k < i; ++k) {
                const double2 t = zmul(L[(size_t)k * p + i], X[(size_t)c * p + k]);
                s.x -= t.x;
                s.y -= t.y;
            }
            const double lii = L[(size_t)i * p + i].x;
            X[(size_t)c * p + i] = make_double2(s.x / lii, s.y / lii);
        }
    }
    __syncthreads();
    // R^-1[a,b] = sum_k conj(X[k,a]) X[k,b], k >= max(a,b); FP32 copies
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const int b = e / p, a = e - b * p;
        double2 s = make_double2(0.0, 0.0);
        for (int k = max(a, b); k < p; ++k) {
            const double2 t = zmulc(X[(size_t)b * p + k], X[(size_t)a * p + k]);
            s.x += t.x;
            s.y += t.y;
        }
        J.Ri32[e] = make_float2((float)s.x, (float)s.y);
        J.Li32[e] = make_float2((float)X[e].x, (float)X[e].y);
        const double2 xt = X[(size_t)a * p + b];               // L^-1(b, a)
        J.LiH32[e] = make_float2((float)xt.x, (float)-xt.y);
        J.R32[e] = make_float2((float)J.R64[e].x, (float)J.R64[e].y);
    }
    if (threadIdx.x == 0) J.flags[0] = 0;
}

__global__ void k_factor(JobDev *const *jobs) { factor_job(*jobs[blockIdx.x]); }

// ---------------------------------------------------------------- bounds
// dirty_i = Re(a_i^H R a_i) and h_i = a_i^H R^-1 a_i = ||L^-1 a_i||^2 for
// all pixels (eq. mfdimg and the MVDR denominator, the latter in whitened
// form: a sum of squares keeps its rounding error relative to h_i, where the
// quadratic form's error is relative to |a|^T |R^-1| |a|, far larger than h_i
// at a bright source), blockIdx.y = job.
__global__ void k_bounds(JobDev *const *jobs) {
    const JobDev &J = *jobs[blockIdx.y];
    if (J.flags[0] != 0) return;
    extern __shared__ float4 smem4[];
    float2 *A = reinterpret_cast<float2 *>(smem4);
    float *red = reinterpret_cast<float *>(A + J.p * kTile);
    const int ntiles = (J.Q + kTile - 1) / kTile;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int pix0 = t * kTile;
        const int np = min(kTile, J.Q - pix0);
        fill_steer_adj(J, pix0, np, A);
        __syncthreads();
        adj_chunk(J.R32, J.p, A, red);
        if (threadIdx.x < np) J.dirty[pix0 + threadIdx.x] = red[threadIdx.x];
        __syncthreads();
        adj_chunk<true>(J.Li32, J.p, A, red);
        if (threadIdx.x < np) J.h[pix0 + threadIdx.x] = red[threadIdx.x];
        __syncthreads();
    }
}

// Tensor-core form of k_bounds: pass 1 with B = R_hat (dirty image), pass 2
// with B from V = L^-1 and the sum-of-squares epilogue (MVDR denominators
// ||L^-1 a_i||^2), over 128-pixel tiles.
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) k_bounds_tc(JobDev *const *jobs) {
    const JobDev &J = *jobs[blockIdx.y];
    if (J.flags[0] != 0) return;
    constexpr bool BF = MODE == 2;
    extern __shared__ float4 smem4[];
    unsigned char *dyn = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem4) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bars[2];
    __shared__ uint32_t slot;
    __shared__ double dbuf[kThreads / 32];
    __shared__ float red[2 * kTcM];
    TcWork T{};
    tc_carve(T, dyn, J.p);
    tc_setup(T, bars, &slot, J.p);
    const float sX = tc_steer_scale(J.p);
    const uint32_t idesc = idesc_f16(2 * T.Kp, BF ? 1 : 0);
    const int ntiles = tc_num_tiles(J.n_l, J.n_m);
    const int mine = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    for (int pass = 0; pass < 2; ++pass) {
        const float sB = tc_build_B<BF>(pass == 0 ? J.R32 : J.LiH32, J.p, T, dbuf);
        const float inv = pass == 0 ? 1.f / (sX * sX * sB) : 1.f / ((sX * sB) * (sX * sB));
        float *dst = pass == 0 ? J.dirty : J.h;
        tc_run_tiles(
            T, mine, idesc,
            [&](int t, int b) { tc_gen_X_steer<BF>(J, T, b, blockIdx.x + t * gridDim.x, sX); },
            [&](int t, int b) {
                if (pass == 0) tc_epilogue<BF>(T, b, red);
                else tc_epilogue<BF, true>(T, b, red);
                if (threadIdx.x < kTcM) {
                    const int i = tc_tile_pixel(blockIdx.x + t * gridDim.x, threadIdx.x, J.n_l, J.n_m);
                    if (i >= 0) dst[i] = red[threadIdx.x] * inv;
                }
                __syncthreads();
            });
    }
    if (T.timeouts && threadIdx.x == 0) J.flags[2] = IMG_ETIMEOUT;
    tc_teardown(T, J.p);
}

// Tensor-core Psi^H vect(U) over all pixels of one job.
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) k_psi_adj_tc(const JobDev *Jp, const float2 *U,
                                                           double *out) {
    const JobDev &J = *Jp;
    constexpr bool BF = MODE == 2;
    extern __shared__ float4 smem4[];
    unsigned char *dyn = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem4) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bars[2];
    __shared__ uint32_t slot;
    __shared__ double dbuf[kThreads / 32];
    __shared__ float red[2 * kTcM];
    TcWork T{};
    tc_carve(T, dyn, J.p);
    tc_setup(T, bars, &slot, J.p);
    const float sX = tc_steer_scale(J.p);
    const uint32_t idesc = idesc_f16(2 * T.Kp, BF ? 1 : 0);
    const float sB = tc_build_B<BF>(U, J.p, T, dbuf);
    const float inv = 1.f / (sX * sX * sB);
    const int ntiles = tc_num_tiles(J.n_l, J.n_m);
    const int mine = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    tc_run_tiles(
        T, mine, idesc,
        [&](int t, int b) { tc_gen_X_steer<BF>(J, T, b, blockIdx.x + t * gridDim.x, sX); },
        [&](int t, int b) {
            tc_epilogue<BF>(T, b, red);
            if (threadIdx.x < kTcM) {
                const int i = tc_tile_pixel(blockIdx.x + t * gridDim.x, threadIdx.x, J.n_l, J.n_m);
                if (i >= 0) out[i] = red[threadIdx.x] * inv;
            }
            __syncthreads();
        });
    tc_teardown(T, J.p);
}

// max |entry| of R_hat (blockIdx.y = 0) and L^-H (1) per job, 8 blocks
// each (J.Bmax was zeroed by the factor kernel).
__global__ void k_emb_max_bounds(JobDev *const *jobs) {
    const JobDev &J = *jobs[blockIdx.x];
    if (J.flags[0] != 0) return;
    const int w = blockIdx.y;
    emb_absmax(w ? J.LiH32 : J.R32, J.p, blockIdx.z, gridDim.z, J.Bmax + w);
}

// Chunked B images of R_hat (blockIdx.y = 0) and L^-H (1) per job; one
// CTA per (64-column chunk, block of kEmbRows rows): blockIdx.z = chunk *
// (512 / kEmbRows) + row block.
template <int MODE>
__global__ void k_emb_bounds(JobDev *const *jobs) {
    const JobDev &J = *jobs[blockIdx.x];
    constexpr int kRB = 2 * kWideMaxP / kEmbRows;
    const int kc = blockIdx.z / kRB, rb = blockIdx.z - kc * kRB;
    if (J.flags[0] != 0 || kc >= wide_nk(J.p) || rb * kEmbRows >= 2 * wide_kp(J.p)) return;
    const int w = blockIdx.y;
    emb_B_chunk<MODE == 2>(w ? J.LiH32 : J.R32, J.p, J.Bimg + (size_t)w * wide_B_bytes(J.p), J.Bmax[w],
                           J.Bscale + w, kc, rb);
}

// Wide tensor-core bounds for 64 < p <= 256: dirty image (B = R_hat) and
// a^H R^-1 a = ||L^-1 a||^2 (B from V = L^-1, sum of squares) in one
// warp-specialised pass over the tiles.
template <int MODE>
__global__ void __launch_bounds__(kWideThreads, 1) k_bounds_wide(JobDev *const *jobs) {
    const JobDev &J = *jobs[blockIdx.y];
    if (J.flags[0] != 0) return;
    extern __shared__ float4 smem4[];
    unsigned char *dyn = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem4) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bars[kWideBars];
    __shared__ uint32_t slot;
    const int ntiles = tc_num_tiles(J.n_l, J.n_m);
    const int mine = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    float *dirty = J.dirty, *h = J.h;
    const int to = wide_adjoint<MODE == 2>(J, dyn, bars, &slot, J.Bimg, J.Bimg + wide_B_bytes(J.p), J.Bscale, 2,
                                           blockIdx.x, gridDim.x, mine, 2,
                                           [&](int s, int i, float v) { (s == 0 ? dirty : h)[i] = v; });
    if (to && threadIdx.x == 0) J.flags[2] = IMG_ETIMEOUT;
}

// max |entry| of one operator U (Jp->Bmax[0] zeroed before), and its B
// image for k_psi_adj_wide (grid: chunks x row blocks).
template <class TC>
__global__ void k_emb_max_one(const JobDev *Jp, const TC *U) {
    emb_absmax(U, Jp->p, blockIdx.x, gridDim.x, Jp->Bmax);
}
template <int MODE, class TC>
__global__ void k_emb_one(const JobDev *Jp, const TC *U) {
    emb_B_chunk<MODE == 2>(U, Jp->p, Jp->Bimg, Jp->Bmax[0], Jp->Bscale, blockIdx.x, blockIdx.y);
}

// Wide tensor-core Psi^H vect(U) over all pixels of one job.
template <int MODE>
__global__ void __launch_bounds__(kWideThreads, 1) k_psi_adj_wide(const JobDev *Jp, double *out) {
    const JobDev &J = *Jp;
    extern __shared__ float4 smem4[];
    unsigned char *dyn = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem4) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bars[kWideBars];
    __shared__ uint32_t slot;
    const int ntiles = tc_num_tiles(J.n_l, J.n_m);
    const int mine = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    wide_adjoint<MODE == 2>(J, dyn, bars, &slot, J.Bimg, J.Bimg, J.Bscale, 1, blockIdx.x, gridDim.x, mine, 0,
                            [&](int, int i, float v) { out[i] = v; });
}

// ---------------------------------------------------------------- wide forward
// Blocks of G formed by k_fwd_wide, in fwd_pairs order, and the index of
// block (m, nb) in that order (-1: not formed).
struct FwdMap {
    int np;
    int m[16], nb[16];
    int idx[6][3];      // 2 Kp <= 768 features: 6 row blocks of 128, 3 column blocks of 256
};

__global__ void k_fwd_wmax(const float *w, int Q, unsigned *wbits) { fwd_wmax(w, Q, wbits); }

template <int MODE>
__global__ void __launch_bounds__(kFwdThreads, 1) k_fwd_wide(const JobDev *Jp, const float *w, const unsigned *wbits,
                                                            FwdMap map, float *part) {
    const JobDev &J = *Jp;
    extern __shared__ float4 smem4[];
    unsigned char *dyn = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem4) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bars[5];
    __shared__ uint32_t slot;
    const int pr = blockIdx.y, S = gridDim.x;
    wide_forward<MODE == 2>(J, dyn, bars, &slot, w, *wbits, map.m[pr], map.nb[pr], blockIdx.x, S,
                            part + ((size_t)pr * S + blockIdx.x) * (kTcM * 256));
}

// Sum of the S partials of every formed block, in a fixed order: 4 groups
// of threads take s = g, g + 4, ... for 64 consecutive entries, then the 4
// group sums are added in group order.  Ub: np blocks of 128 x 256 doubles.
__global__ void k_fwd_reduce(const float *part, int S, int nent, double *Ub) {
    __shared__ double red[4][64];
    const int j = threadIdx.x & 63, g = threadIdx.x >> 6;
    const int e = blockIdx.x * 64 + j;
    constexpr size_t kBlk = (size_t)kTcM * 256;
    double acc = 0.0;
    if (e < nent) {
        const int pr = e / (int)kBlk, off = e - pr * (int)kBlk;
        const float *q = part + (size_t)pr * S * kBlk + off;
#pragma unroll 4
        for (int s = g; s < S; s += 4) acc += q[(size_t)s * kBlk];
    }
    red[g][j] = acc;
    __syncthreads();
    if (g == 0 && e < nent) Ub[e] = ((red[0][j] + red[1][j]) + red[2][j]) + red[3][j];
}

// K (p x p complex128, column-major) from the summed blocks: entries of G on
// or above the diagonal, U(a, b); K_kl = U(k,l) + U(Kp+k,Kp+l) + j (U(l,Kp+k)
// - U(k,Kp+l)) for k <= l, scaled back by 1 / (sX^2 sW); K_lk = conj(K_kl).
__global__ void k_fwd_assemble(int p, const double *Ub, FwdMap map, const unsigned *wbits, double2 *K) {
    const int Kp = wide_kp(p);
    const float sX = steer_scale(p);
    const double inv = 1.0 / ((double)sX * sX * emb_scale_of(*wbits));
    constexpr size_t kBlk = (size_t)kTcM * 256;
    auto U = [&](int a, int b) {
        const int m = a >> 7, nb = b >> 8, pr = map.idx[m][nb];
        return Ub[(size_t)pr * kBlk + (size_t)(a - 128 * m) * 256 + (b - 256 * nb)];
    };
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p * p; e += gridDim.x * blockDim.x) {
        const int l = e / p, k = e - l * p;
        if (k > l) continue;
        const double re = (U(k, l) + U(Kp + k, Kp + l)) * inv;
        const double im = k == l ? 0.0 : (U(l, Kp + k) - U(k, Kp + l)) * inv;
        K[(size_t)l * p + k] = make_double2(re, im);
        K[(size_t)k * p + l] = make_double2(re, -im);
    }
}

// ---------------------------------------------------------------- full-image LSQR
// Unconstrained LS / WLS image with every pixel free: LSQR (Sec. V-A) on
// M = Psi (CLS) or W Psi D^-1 (PWLS, W = conj(L^-1) kron L^-1), b = vect(R_hat)
// or W vect(R_hat) = vect(I).  The bidiagonalisation runs as a stream of
// kernels: the operators above, complex p x p products for the whitening,
// one-CTA reductions in a fixed order, and a one-thread kernel for the FP64
// scalar recurrences, whose results later kernels read from device memory.

// out = sum of squares of n floats (complex: 2n floats), one CTA, fixed order.
__global__ void k_sumsq(const float *x, int n, double *out) {
    __shared__ double red[32];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fma((double)x[i], (double)x[i], acc);
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *out = s;
    }
}

// FP64 scalars (one thread).  phase 0: beta of b; 1: alpha of the first v;
// 2: beta of an iteration; 3: alpha, rotation and update coefficients.
__global__ void k_ls_scalar(double *sc, int phase) {
    if (threadIdx.x != 0) return;
    if (phase == 0) {
        const double beta = sqrt(sc[kLsSsU]);
        sc[kLsBeta] = beta;
        sc[kLsBnorm] = beta;
        sc[kLsUs] = beta > 0.0 ? 1.0 / beta : 0.0;
    } else if (phase == 1) {
        const double alpha = sqrt(sc[kLsSsV]);
        sc[kLsAlpha] = alpha;
        sc[kLsIa] = alpha > 0.0 ? 1.0 / alpha : 1.0;
        sc[kLsPhibar] = sc[kLsBeta];
        sc[kLsRhobar] = alpha;
        sc[kLsAnorm2] = 0.0;
        sc[kLsRnorm] = sc[kLsBeta];
        sc[kLsArnorm] = alpha * sc[kLsBeta];
    } else if (phase == 2) {
        const double beta = sqrt(sc[kLsSsU]), alpha = sc[kLsAlpha];
        sc[kLsBeta] = beta;
        sc[kLsUs] = beta > 0.0 ? 1.0 / beta : 0.0;
        sc[kLsAnorm2] += alpha * alpha + beta * beta;
    } else {
        const double alpha = sqrt(sc[kLsSsV]), beta = sc[kLsBeta];
        const double rhobar = sc[kLsRhobar], phibar = sc[kLsPhibar];
        const double rho = hypot(rhobar, beta);
        const double c = rhobar / rho, s = beta / rho;
        const double theta = s * alpha, phi = c * phibar;
        sc[kLsAlpha] = alpha;
        sc[kLsIa] = alpha > 0.0 ? 1.0 / alpha : 1.0;
        sc[kLsRhobar] = -c * alpha;
        sc[kLsPhibar] = s * phibar;
        sc[kLsT1] = phi / rho;
        sc[kLsT2] = -theta / rho;
        sc[kLsRnorm] = s * phibar;
        sc[kLsArnorm] = s * phibar * alpha * fabs(c);
    }
}

// u = b: vect(R_hat) (CLS) or vect(I) (PWLS, W vect(R_hat) = vect(L^-1 R L^-H)).
__global__ void k_ls_init_u(const float2 *R32, int p, int pwls, float2 *u) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < p * p; e += gridDim.x * blockDim.x) {
        const int j = e / p, i = e - j * p;
        u[e] = pwls ? make_float2(i == j ? 1.f : 0.f, 0.f) : R32[e];
    }
}
// u *= us (u = t / beta).
__global__ void k_ls_scale_u(float2 *u, int pp, const double *sc) {
    const float us = (float)sc[kLsUs];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < pp; e += gridDim.x * blockDim.x)
        u[e] = make_float2(u[e].x * us, u[e].y * us);
}
// u = Mv - alpha u.
__global__ void k_ls_u(float2 *u, const float2 *Mv, int pp, const double *sc) {
    const float a = (float)sc[kLsAlpha];
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < pp; e += gridDim.x * blockDim.x) {
        const float2 m = Mv[e], o = u[e];
        u[e] = make_float2(m.x - a * o.x, m.y - a * o.y);
    }
}
// wx = scale o v (the forward's pixel weights, D^-1 v for PWLS).
__global__ void k_ls_weights(const float *scale, const float *v, float *wx, int Q) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q; i += gridDim.x * blockDim.x) wx[i] = scale[i] * v[i];
}
// v = scale o y - beta v (first = true: v = scale o y).
__global__ void k_ls_v(float *v, const double *y, const float *scale, int Q, const double *sc, int first) {
    const float b = first ? 0.f : (float)sc[kLsBeta];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q; i += gridDim.x * blockDim.x)
        v[i] = scale[i] * (float)y[i] - (first ? 0.f : b * v[i]);
}
// v /= alpha; first: w = v, x = 0; else x += t1 w, w = v + t2 w.
__global__ void k_ls_xw(float *x, float *w, float *v, int Q, const double *sc, int first) {
    const float ia = (float)sc[kLsIa], t1 = (float)sc[kLsT1], t2 = (float)sc[kLsT2];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q; i += gridDim.x * blockDim.x) {
        const float vi = v[i] * ia;
        v[i] = vi;
        if (first) {
            w[i] = vi;
            x[i] = 0.f;
        } else {
            const float wi = w[i];
            x[i] += t1 * wi;
            w[i] = vi + t2 * wi;
        }
    }
}
__global__ void k_ls_sigma(const float *x, const float *scale, double *sigma, int Q) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q; i += gridDim.x * blockDim.x)
        sigma[i] = (double)scale[i] * (double)x[i];
}
__global__ void k_d2c(const double2 *src, float2 *dst, int n) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        dst[e] = make_float2((float)src[e].x, (float)src[e].y);
}

// C = op(A) op(B), p x p complex FP32 column-major; op 0: as is, 1: conjugate
// transpose.  32 x 32 output tiles, 256 threads (2 x 2 outputs each).
__global__ void k_cgemm(int p, const float2 *A, int opA, const float2 *B, int opB, float2 *C) {
    __shared__ float2 As[32][33], Bs[32][33];
    const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float2 acc[2][2] = {};
    for (int k0 = 0; k0 < p; k0 += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
            const int r = e & 31, c = e >> 5;           // As[r][c] = op(A)[i0 + r, k0 + c]
            const int i = i0 + r, k = k0 + c;
            float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
            if (i < p && k < p) {
                a = opA ? A[(size_t)i * p + k] : A[(size_t)k * p + i];
                if (opA) a.y = -a.y;
            }
            As[r][c] = a;
            const int kk = k0 + r, j = j0 + c;          // Bs[r][c] = op(B)[k0 + r, j0 + c]
            if (kk < p && j < p) {
                b = opB ? B[(size_t)kk * p + j] : B[(size_t)j * p + kk];
                if (opB) b.y = -b.y;
            }
            Bs[r][c] = b;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) cfma(acc[a][b], As[2 * ty + a][kk], Bs[kk][2 * tx + b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = i0 + 2 * ty + a, j = j0 + 2 * tx + b;
            if (i < p && j < p) C[(size_t)j * p + i] = acc[a][b];
        }
}

// ---------------------------------------------------------------- failure detection
// Self-test of the bounded waits every tensor-core kernel uses: one CTA
// allocates tensor memory, waits on an mbarrier that receives an arrival only
// when `arrive` is set, gives up after `polls` polls, frees the tensor memory
// on its normal exit path and reports through *status (IMG_OK or
// IMG_ETIMEOUT).  No fault, trap or endless loop is involved.
__global__ void k_wait_selftest(unsigned polls, int arrive, int *status) {
    __shared__ uint64_t bar;
    __shared__ uint32_t slot;
    __shared__ int timed_out;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        timed_out = 0;
    }
    if (threadIdx.x < 32) tmem_alloc(&slot, 32);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (arrive && threadIdx.x == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
    if (!mbar_wait(&bar, 0u, polls)) atomicOr(&timed_out, 1);
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(slot, 32);
    if (threadIdx.x == 0) *status = timed_out ? IMG_ETIMEOUT : IMG_OK;
}

cudaError_t launch_wait_selftest(unsigned polls, int arrive, int *status, cudaStream_t st) {
    k_wait_selftest<<<1, 64, 0, st>>>(polls, arrive, status);
    return cudaGetLastError();
}

// Bounds, preconditioner and thresholds (one CTA per job):
//   C = N/(N-p) or 1; mvdr = C/h; D = h^2/C; std_MF = dirty/sqrt(N);
//   std_MVDR = mvdr/sqrt(N-p-1); gamma = chosen image, optionally inflated;
//   PWLS: x = D sigma (scale 1/D, upper D gamma); eps = kappa std with a floor.
__device__ void finalize_job(const JobDev &J) {
    __shared__ double sbuf[kThreads / 32];
    const double C = J.bias_c ? (double)J.N / (double)(J.N - J.p) : 1.0;
    const double sqN = sqrt((double)J.N);
    const double dof = (double)(J.N - J.p - 1);
    const bool pwls = J.cost == IMG_COST_PWLS;
    double mx = 0.0;
    for (int i = threadIdx.x; i < J.Q; i += blockDim.x) {
        const double h = J.h[i];
        const double d = J.dirty[i];
        const double mv = C / h;
        const double base = J.bound == IMG_BOUND_MF ? d : mv;
        const double sd = J.bound == IMG_BOUND_MF ? d / sqN : (dof > 0 ? mv / sqrt(dof) : INFINITY);
        double g = base;
        if (J.inflate == IMG_INFLATE_RATIO) g = (1.0 + J.alpha) * base;
        else if (J.inflate == IMG_INFLATE_STD) g = base + J.alpha * sd;
        const double D = h * h / C;
        double mb = mv;
        if (J.inflate == IMG_INFLATE_RATIO) mb = (1.0 + J.alpha) * mv;
        else if (J.inflate == IMG_INFLATE_STD) mb = mv + J.alpha * (dof > 0 ? mv / sqrt(dof) : INFINITY);
        J.mvb[i] = mb;
        J.gamma[i] = g;
        J.upper[i] = pwls ? D * g : g;
        J.scale[i] = pwls ? (float)(1.0 / D) : 1.0f;
        const double sdc = pwls ? (dof > 0 ? mv / sqrt(dof) : INFINITY) : d / sqN;
        J.eps[i] = (float)(J.kappa * sdc);
        mx = fmax(mx, pwls ? mv : d);
    }
    // max over the CTA (all values positive)
    for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) mx = fmax(mx, sbuf[w]);
    const float fl = (float)(J.eps_floor * mx);
    for (int i = threadIdx.x; i < J.Q; i += blockDim.x) J.eps[i] = fmaxf(J.eps[i], fl);
    if (threadIdx.x == 0) J.flags[1] = 1;
    __syncthreads();
}

__global__ void k_finalize(JobDev *const *jobs, int *batch_status) {
    const JobDev &J = *jobs[blockIdx.x];
    if (batch_status && threadIdx.x == 0) batch_status[blockIdx.x] = J.flags[0];
    if (J.flags[0] != 0) return;
    finalize_job(J);
}

// ---------------------------------------------------------------- solver
struct SolveShared {
    double dbuf[kThreads / 32];
    double vbuf[kThreads / 32];
    int ibuf[kThreads / 32];
    int cbuf[kThreads / 32];
    float wsm[kTile];
    float red[kTile + 16 * kTile];
};

// c = T a_i for the support cache (T = L^-1 for PWLS, identity for LS), and
// its largest component magnitude (for the tensor-core operand scaling).
__device__ void cache_vector(const JobDev &J, int i, int slot, double *sbuf) {
    const int p = J.p;
    const int im = i / J.n_l, il = i - im * J.n_l;
    float2 *c = J.cvec + (size_t)slot * p;
    const bool pwls = J.cost == IMG_COST_PWLS;
    float mx = 0.f;
    for (int k = threadIdx.x; k < p; k += blockDim.x) {
        float2 s = make_float2(0.f, 0.f);
        if (!pwls) {
            s = steer(J, il, im, k);
        } else {
            for (int l = 0; l <= k; ++l) cfma(s, J.Li32[(size_t)l * p + k], steer(J, il, im, l));
        }
        c[k] = s;
        mx = fmaxf(mx, fmaxf(fabsf(s.x), fabsf(s.y)));
    }
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) m = fmaxf(m, (float)sbuf[w]);
        J.cmax[slot] = m;
    }
    __syncthreads();
}

// Power-of-two scale for the cached vectors of a list (max |entry| <= 1),
// lifted by kLift (the tiles' split parts stay normal FP16 numbers).
__device__ float list_scale(const JobDev &J, const int *pos, int n, double *sbuf) {
    float mx = 0.f;
    for (int j = threadIdx.x; j < n; j += blockDim.x) mx = fmaxf(mx, J.cmax[pos ? pos[j] : j]);
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) mx = fmaxf(mx, (float)sbuf[w]);
    __syncthreads();
    return (mx > 0.f ? exp2f(-ceilf(log2f(mx))) : 1.f) * kLift;
}

// K = base + sum_j wt[j] c_j c_j^H over a list of cached vectors, on tensor
// cores when MODE != 0 and Kp = 64, else on CUDA cores.
template <int MODE>
__device__ void forward_cache(const JobDev &J, TcWork &T, const int *pos, const float *wt, int n,
                              const float2 *base, bool base_identity, float2 *K, float2 *A,
                              float *wsm, double *dbuf) {
    if constexpr (MODE != 0) {
        if (T.Kp == 64) {
            constexpr bool BF = MODE == 2;
            const float sX = list_scale(J, pos, n, dbuf);
            tc_forward<BF>(T, J.p, n, wt, sX,
                           [&](int t, int np) { tc_gen_X_cache<BF>(J, T, 0, pos, t * kTcM, np, sX); },
                           base, base_identity, K, dbuf);
            return;
        }
    }
    forward_list(J, pos, wt, n, false, base, base_identity, K, A, wsm);
}

// Adjoint over a list of cached vectors: t_j = Re(c_j^H U c_j), handed to
// epi(j, t_j) on threads < tile size.  MODE 0: CUDA cores (FP32); 1/2:
// tensor cores with split FP16 / BF16 operands.
template <int MODE, class Epi>
__device__ void adjoint_list(const JobDev &J, const float2 *U, const int *pos, int n, float2 *A,
                             TcWork &T, float *red, double *dbuf, Epi epi) {
    if constexpr (MODE == 0) {
        for (int j0 = 0; j0 < n; j0 += kTile) {
            const int np = min(kTile, n - j0);
            fill_cache_adj(J, pos, j0, np, A);
            __syncthreads();
            adj_chunk(U, J.p, A, red);
            if (threadIdx.x < np) epi(j0 + threadIdx.x, red[threadIdx.x]);
            __syncthreads();
        }
    } else {
        constexpr bool BF = MODE == 2;
        const float sB = tc_build_B<BF>(U, J.p, T, dbuf);
        const float sXl = list_scale(J, pos, n, dbuf);
        const uint32_t idesc = idesc_f16(2 * T.Kp, BF ? 1 : 0);
        tc_run_tiles(
            T, (n + kTcM - 1) / kTcM, idesc,
            [&](int t, int b) {
                const int j0 = t * kTcM;
                tc_gen_X_cache<BF>(J, T, b, pos, j0, min(kTcM, n - j0), sXl);
                T.sX[b] = sXl;
            },
            [&](int t, int b) {
                const int j0 = t * kTcM;
                const int np = min(kTcM, n - j0);
                tc_epilogue<BF>(T, b, red);
                const float inv = 1.f / (T.sX[b] * T.sX[b] * sB);
                if (threadIdx.x < np) epi(j0 + threadIdx.x, red[threadIdx.x] * inv);
                __syncthreads();
            });
    }
}

// Full-image adjoint with generated steering vectors: epi(i, Re(a_i^H U a_i))
// for every pixel, on one thread per pixel.  SQ: epi(i, ||V a_i||^2) with V
// = U on CUDA cores (U column-major) and V = U^H on tensor cores (the B
// operand's convention), i.e. U = L^-1 resp. L^-H for the whitened MVDR
// denominator.
template <int MODE, bool SQ = false, class Epi, class Pre>
__device__ void adjoint_full(const JobDev &J, const float2 *U, float2 *A, TcWork &T, float *red,
                             double *dbuf, Epi epi, Pre pre) {
    const int Q = J.Q;
    if constexpr (MODE == 0) {
        const int ntiles = (Q + kTile - 1) / kTile;
        for (int t = 0; t < ntiles; ++t) {
            const int pix0 = t * kTile;
            const int np = min(kTile, Q - pix0);
            fill_steer_adj(J, pix0, np, A);
            __syncthreads();
            adj_chunk<SQ>(U, J.p, A, red);
            if (threadIdx.x < np) {
                pre(pix0 + threadIdx.x);
                epi(pix0 + threadIdx.x, red[threadIdx.x]);
            }
            __syncthreads();
        }
    } else {
        constexpr bool BF = MODE == 2;
        const float sB = tc_build_B<BF>(U, J.p, T, dbuf);
        const float sX = tc_steer_scale(J.p);
        const float inv = SQ ? 1.f / ((sX * sB) * (sX * sB)) : 1.f / (sX * sX * sB);
        const uint32_t idesc = idesc_f16(2 * T.Kp, BF ? 1 : 0);
        tc_run_tiles(
            T, tc_num_tiles(J.n_l, J.n_m), idesc,
            [&](int t, int b) { tc_gen_X_steer<BF>(J, T, b, t, sX); },
            [&](int t, int b) {
                tc_epilogue<BF, SQ>(T, b, red);
                if (threadIdx.x < kTcM) {
                    const int i = tc_tile_pixel(t, threadIdx.x, J.n_l, J.n_m);
                    if (i >= 0) epi(i, red[threadIdx.x] * inv);
                }
                __syncthreads();
            },
            [&](int t) {
                if (threadIdx.x < kTcM) {
                    const int i = tc_tile_pixel(t, threadIdx.x, J.n_l, J.n_m);
                    if (i >= 0) pre(i);
                }
            });
    }
}

template <int MODE, bool SQ = false, class Epi>
__device__ void adjoint_full(const JobDev &J, const float2 *U, float2 *A, TcWork &T, float *red,
                             double *dbuf, Epi epi) {
    adjoint_full<MODE, SQ>(J, U, A, T, red, dbuf, epi, [](int) {});
}

// LSQR (Paige-Saunders) on the free set: min || b - M_F x ||, with
// M_F x = vect(sum_j s_j x_j c_j c_j^H) and (M_F^H u)_j = s_j Re(c_j^H U c_j).
// b is in J.W0 on entry.  The bidiagonalisation follows eq. initbeta ..
// eq. lanczos; rotations and stopping tests as in the FP64 oracle, scalars in
// FP64.  The u-space vector is kept unnormalised: W0 holds t with u = t * us
// (us = 1/beta), which saves a normalisation pass per iteration.  Returns the
// iteration count; the solution is in J.xs[0..f).
template <int MODE>
__device__ int lsqr_cta(const JobDev &J, int f, float2 *A, TcWork &T, SolveShared &S, DevInfo &info) {
    constexpr bool BF = MODE == 2;
    const int p = J.p, pp = p * p;
    const int *__restrict__ fpos = J.fpos;
    float2 *__restrict__ t = J.W0;
    // free-set tiles resident in shared memory for the whole solve (tensor
    // cores, Kp = 64, at most two 128-pixel tiles); the f-vectors then live
    // in shared memory too
    bool resident = false;
    float sXr = 1.f;
    unsigned char *stage = nullptr;
    float *v = J.v, *w = J.w, *xs = J.xs, *sF = J.sF, *wt = J.xs + J.cap;
    if constexpr (MODE != 0) {
        resident = T.Kp == 64 && f <= 2 * kTcM;
        if (resident) {
            stage = T.Blo + (T.Blo - T.Bhi);
            float *fv = reinterpret_cast<float *>(stage + tc_stage_bytes(p));
            v = fv;
            w = fv + 2 * kTcM;
            xs = fv + 4 * kTcM;
            sF = fv + 6 * kTcM;
            wt = fv + 8 * kTcM;
            sXr = list_scale(J, fpos, f, S.dbuf);
            tc_gen_X_cache<BF>(J, T, 0, fpos, 0, min(kTcM, f), sXr);
            if (f > kTcM) tc_gen_X_cache<BF>(J, T, 1, fpos, kTcM, f - kTcM, sXr);
        }
    }
    {
        const int *__restrict__ supp = J.supp;
        const float *__restrict__ scale = J.scale;
        for (int j = threadIdx.x; j < f; j += blockDim.x) sF[j] = scale[supp[fpos[j]]];
    }
    float acc = 0.f;     // per-thread partial (<= 16 terms), reduced in FP64
    for (int e = threadIdx.x; e < pp; e += blockDim.x) acc = fmaf(t[e].x, t[e].x, fmaf(t[e].y, t[e].y, acc));
    double beta = sqrt(block_sum((double)acc, S.dbuf));
    const double bnorm = beta;
    for (int j = threadIdx.x; j < f; j += blockDim.x) xs[j] = 0.f;
    if (beta == 0.0) {
        for (int j = threadIdx.x; j < f; j += blockDim.x) J.xs[j] = 0.f;
        __syncthreads();
        return 0;
    }
    double us = 1.0 / beta;
    auto adjoint = [&](auto epi) {
        if constexpr (MODE != 0) {
            if (resident) {
                tc_adjoint_resident<BF>(T, t, p, f, sXr, S.red, S.dbuf, epi, info.cyc_aux);
                return;
            }
        }
        adjoint_list<MODE>(J, t, fpos, f, A, T, S.red, S.dbuf, epi);
    };
    {
        const float fus = (float)us;
        adjoint([&](int j, float y) { v[j] = sF[j] * (y * fus); });
    }
    acc = 0.f;
    for (int j = threadIdx.x; j < f; j += blockDim.x) acc = fmaf(v[j], v[j], acc);
    double alpha = sqrt(block_sum((double)acc, S.dbuf));
    int it = 0;
    if (alpha == 0.0) {
        for (int j = threadIdx.x; j < f; j += blockDim.x) J.xs[j] = 0.f;
        __syncthreads();
        return 0;
    }
    {
        const float ia = (float)(1.0 / alpha);
        for (int j = threadIdx.x; j < f; j += blockDim.x) {
            v[j] *= ia;
            w[j] = v[j];
        }
    }
    __syncthreads();
    double phibar = beta, rhobar = alpha, anorm2 = 0.0;
    const int maxit = J.lsqr_maxit > 0 ? J.lsqr_maxit : 4 * f + 20;
    const double atol = J.lsqr_atol, btol = J.lsqr_btol;
    for (it = 1; it <= maxit; ++it) {
        // t <- M v - alpha u  (u = t * us), beta = ||t||
        for (int j = threadIdx.x; j < f; j += blockDim.x) wt[j] = sF[j] * v[j];
        __syncthreads();
        long long tc0 = clock64();
        const float fa = (float)(alpha * us);
        acc = 0.f;
        bool done = false;
        if constexpr (MODE != 0) {
            if (resident) {
                float inv;
                const float *G = tc_forward_resident<BF>(T, stage, f, wt, sXr, &inv, S.dbuf, info.cyc_aux);
                const long long cu = clock64();
                for (int e = threadIdx.x; e < pp; e += blockDim.x) {
                    const int bcol = e / p, a = e - bcol * p;
                    float2 kv = G ? tc_k_entry(G, T.Kp, a, bcol) : make_float2(0.f, 0.f);
                    const float2 to = t[e];
                    const float2 tn = make_float2(kv.x * inv - fa * to.x, kv.y * inv - fa * to.y);
                    t[e] = tn;
                    acc = fmaf(tn.x, tn.x, fmaf(tn.y, tn.y, acc));
                }
                info.cyc_aux[2] += (double)(clock64() - cu);
                done = true;
            }
        }
        if (!done) {
            forward_cache<MODE>(J, T, fpos, wt, f, nullptr, false, J.W1, A, S.wsm, S.dbuf);
            const float2 *__restrict__ W1 = J.W1;
            for (int e = threadIdx.x; e < pp; e += blockDim.x) {
                const float2 mv = W1[e];
                const float2 to = t[e];
                const float2 tn = make_float2(mv.x - fa * to.x, mv.y - fa * to.y);
                t[e] = tn;
                acc = fmaf(tn.x, tn.x, fmaf(tn.y, tn.y, acc));
            }
        }
        info.cyc_lsqr_fwd += (double)(clock64() - tc0);
        beta = sqrt(block_sum((double)acc, S.dbuf));
        us = beta > 0.0 ? 1.0 / beta : 0.0;
        anorm2 += alpha * alpha + beta * beta;
        // v <- M^H u - beta v
        const float fb = (float)beta, fus = (float)us;
        tc0 = clock64();
        adjoint([&](int j, float y) { v[j] = sF[j] * (y * fus) - fb * v[j]; });
        info.cyc_lsqr_adj += (double)(clock64() - tc0);
        acc = 0.f;
        for (int j = threadIdx.x; j < f; j += blockDim.x) acc = fmaf(v[j], v[j], acc);
        alpha = sqrt(block_sum((double)acc, S.dbuf));
        // plane rotation (scalars in FP64, the same in every thread)
        const double rho = hypot(rhobar, beta);
        const double c = rhobar / rho, s = beta / rho;
        const double theta = s * alpha;
        rhobar = -c * alpha;
        const double phi = c * phibar;
        phibar = s * phibar;
        const float t1 = (float)(phi / rho), t2 = (float)(-theta / rho);
        const float ia = alpha > 0.0 ? (float)(1.0 / alpha) : 1.f;
        acc = 0.f;
        for (int j = threadIdx.x; j < f; j += blockDim.x) {
            const float vj = v[j] * ia;                 // v <- v / alpha
            v[j] = vj;
            const float xj = xs[j] + t1 * w[j];
            xs[j] = xj;
            w[j] = vj + t2 * w[j];
            acc = fmaf(xj, xj, acc);
        }
        const double xnorm = sqrt(block_sum((double)acc, S.dbuf));
        const double rnorm = phibar;
        const double arnorm = phibar * alpha * fabs(c);
        const double anorm = sqrt(anorm2);
        if (rnorm <= btol * bnorm + atol * anorm * xnorm) break;
        if (arnorm <= atol * anorm * rnorm) break;
    }
    if (xs != J.xs)
        for (int j = threadIdx.x; j < f; j += blockDim.x) J.xs[j] = xs[j];
    __syncthreads();
    return min(it, maxit);
}

__device__ __forceinline__ double flops_fwd(int p, int n) { return 4.0 * p * (double)p * n; }
__device__ __forceinline__ double flops_adj(int p, int n) { return 8.0 * p * (double)p * n; }

// Remove support slot sl (pixel i) by moving the last entry into it.
__device__ void supp_remove(const JobDev &J, int i, int &ns) {
    const int p = J.p;
    const int sl = J.slot[i];
    const int last = ns - 1;
    if (sl != last) {
        const int moved = J.supp[last];
        for (int k = threadIdx.x; k < p; k += blockDim.x)
            J.cvec[(size_t)sl * p + k] = J.cvec[(size_t)last * p + k];
        if (threadIdx.x == 0) {
            J.supp[sl] = moved;
            J.slot[moved] = sl;
            J.cmax[sl] = J.cmax[last];
        }
    }
    if (threadIdx.x == 0) J.slot[i] = -1;
    ns = last;
    __syncthreads();
}

// Persistent active-set driver (Table I), one CTA per job.  MODE selects the
// adjoint's arithmetic (0 CUDA cores FP32, 1 tensor cores FP16x3, 2 BF16x3).
template <int MODE, bool PREP>
__global__ void __launch_bounds__(kThreads, 1)
k_solve(JobDev *const *jobs, DevInfo *batch_info, double *const *sigma_out) {
    const JobDev &J = *jobs[blockIdx.x];
    extern __shared__ float4 smem4[];
    // one 1024-aligned region serves the CUDA-core chunk or the tensor tiles
    unsigned char *dyn = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem4) + 1023) & ~uintptr_t(1023));
    float2 *A = reinterpret_cast<float2 *>(dyn);
    __shared__ SolveShared S;
    __shared__ uint64_t tc_bar[2];
    __shared__ uint32_t tc_slot;
    DevInfo info{};
    info.status = IMG_OK;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(info.t_begin_ns));
    const int p = J.p, Q = J.Q;
    const bool pwls = J.cost == IMG_COST_PWLS;
    // tensor memory is allocated once per CTA (the permit is relinquished)
    TcWork T{};
    if constexpr (MODE != 0) {
        tc_carve(T, dyn, p);
        tc_setup(T, tc_bar, &tc_slot, p);
    }
    if constexpr (PREP) {
        // the whole job in this CTA: steering tables, factor, dirty image and
        // MVDR denominators (the adjoint of k_bounds), bounds and thresholds
        tables_job(J, threadIdx.x, blockDim.x);
        __syncthreads();
        factor_job(J);
        __syncthreads();
        if (J.flags[0] == 0) {
            adjoint_full<MODE>(J, J.R32, A, T, S.red, S.dbuf, [&](int i, float v) { J.dirty[i] = v; });
            adjoint_full<MODE, true>(J, MODE == 0 ? J.Li32 : J.LiH32, A, T, S.red, S.dbuf,
                                     [&](int i, float v) { J.h[i] = v; });
            finalize_job(J);
        }
        __syncthreads();
    }
    if (J.flags[0] != 0 || J.flags[1] != 1) {
        info.status = J.flags[0] != 0 ? J.flags[0] : IMG_EINVAL;
        if (threadIdx.x == 0) {
            *J.info = info;
            if (batch_info) batch_info[blockIdx.x] = info;
        }
        if constexpr (MODE != 0) tc_teardown(T, p);
        return;
    }
    for (int i = threadIdx.x; i < Q; i += blockDim.x) {
        J.x[i] = 0.0;
        J.set[i] = IMG_SET_L;
        J.slot[i] = -1;
        J.grad[i] = 0.f;
    }
    __syncthreads();
    const long long t_start = clock64();
    int nev = 0;          // decisions so far
    auto log_event = [&](int kind, int pixel, float val) {
        if (threadIdx.x == 0 && nev < J.ev_cap) {
            J.ev[nev] = (kind << 24) | pixel;
            J.evv[nev] = val;
        }
        ++nev;
    };
    int ns = 0;           // support size |F u U|
    bool flag = true;     // Freegradient-isnotzero
    int imin = -1;
    double lam_min = 0.0;
    const int max_outer = J.max_outer > 0 ? J.max_outer : 10 * Q + 100;
    int outer = 0;
    bool converged = false;
    float *wt = J.xs + J.cap;
    while (outer < max_outer) {
        ++outer;
        if (flag) {
            const int f = block_compact(ns, [&](int pos) { return J.set[J.supp[pos]] == IMG_SET_F; },
                                        J.fpos, S.cbuf);
            bool feasible = true;
            if (f > 0) {
                // b = B0 - sum_{U} s_i x_i c_i c_i^H   (eq. bsubproblemLS / MVDR)
                const int nu = block_compact(ns, [&](int pos) { return J.set[J.supp[pos]] == IMG_SET_U; },
                                             J.fpos + f, S.cbuf);
                for (int j = threadIdx.x; j < nu; j += blockDim.x) {
                    const int i = J.supp[J.fpos[f + j]];
                    wt[j] = -J.scale[i] * (float)J.x[i];
                }
                __syncthreads();
                forward_cache<MODE>(J, T, J.fpos + f, wt, nu, pwls ? nullptr : J.R32, pwls, J.W0, A, S.wsm,
                                    S.dbuf);
                info.op_flops += flops_fwd(p, nu);
                const long long t0 = clock64();
                const int its = lsqr_cta<MODE>(J, f, A, T, S, info);
                info.cyc_lsqr += (double)(clock64() - t0);
                info.lsqr_iters += its;
                info.op_flops += (its + 1) * (flops_fwd(p, f) + flops_adj(p, f));
                // feasibility with the relative tolerance tau, non-strict
                int bad = 0;
                const double tau = J.feas_tol;
                for (int j = threadIdx.x; j < f; j += blockDim.x) {
                    const double z = J.xs[j];
                    const double u = J.upper[J.supp[J.fpos[j]]];
                    if (!(z >= -tau * u && z <= (1.0 + tau) * u)) bad = 1;
                }
                feasible = __syncthreads_or(bad) == 0;
            }
            if (feasible) {
                for (int j = threadIdx.x; j < f; j += blockDim.x) {
                    const int i = J.supp[J.fpos[j]];
                    J.x[i] = fmin(fmax((double)J.xs[j], 0.0), J.upper[i]);
                }
                flag = false;
                __syncthreads();
                // gradient: E = B0 - sum_S s_i x_i c_i c_i^H, U_g = T^H E T
                for (int j = threadIdx.x; j < ns; j += blockDim.x) {
                    const int i = J.supp[j];
                    wt[j] = -J.scale[i] * (float)J.x[i];
                }
                __syncthreads();
                forward_cache<MODE>(J, T, nullptr, wt, ns, pwls ? nullptr : J.R32, pwls, J.W1, A, S.wsm,
                                    S.dbuf);
                info.op_flops += flops_fwd(p, ns);
                const float2 *Ug = J.W1;
                if (pwls) {
                    cgemm_pp(p, J.W1, false, J.Li32, J.W2);
                    cgemm_pp(p, J.Li32, true, J.W2, J.W0);
                    Ug = J.W0;
                }
                const long long tg = clock64();
                double best = INFINITY;
                int bidx = 0x7fffffff;
                float bestf = INFINITY;
                {
                    const float *__restrict__ scale = J.scale;
                    const float *__restrict__ eps = J.eps;
                    const unsigned char *__restrict__ set = J.set;
                    float *__restrict__ grad = J.grad;
                    // this thread's pixel of the tile: its scale, threshold and set
                    // are loaded before the tile's MMA is awaited
                    float pscale = 0.f, peps = 0.f;
                    unsigned char pset = 0;
                    adjoint_full<MODE>(
                        J, Ug, A, T, S.red, S.dbuf,
                        [&](int i, float val) {
                            // lambda_L = g, lambda_U = -g (eq. etaL, eq. etaU); g and eps are FP32
                            const float g = -pscale * val;
                            grad[i] = g;
                            if (pset != IMG_SET_F) {
                                const float lam = pset == IMG_SET_U ? -g : g;
                                if (lam < -peps && (lam < bestf || (lam == bestf && i < bidx))) {
                                    bestf = lam;
                                    bidx = i;
                                }
                            }
                        },
                        [&](int i) {
                            pscale = scale[i];
                            peps = eps[i];
                            pset = set[i];
                        });
                }
                best = bestf;
                info.op_flops += flops_adj(p, Q);
                block_argmin(best, bidx, S.vbuf, S.ibuf);
                info.cyc_gradient += (double)(clock64() - tg);
                lam_min = best;
                if (bidx == 0x7fffffff) {
                    converged = true;
                    break;
                }
                imin = bidx;
            } else {
                // step towards z: mu_i per eq. mumax, smallest index on ties
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
                block_argmin(best, bidx, S.vbuf, S.ibuf);
                const double mu = best;
                const int ic = bidx;
                // the blocking pixel moves to U when its direction is positive
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
                }
                log_event(up ? 2 : 1, ic, (float)mu);
                __syncthreads();
                if (!up) supp_remove(J, ic, ns);
                flag = true;
            }
        } else {
            // delete a constraint: pixel imin joins F at its current value
            const int i = imin;
            if (J.slot[i] < 0) {
                if (ns >= J.cap) {
                    info.status = IMG_ENOMEM;
                    break;
                }
                cache_vector(J, i, ns, S.dbuf);
                if (threadIdx.x == 0) {
                    J.supp[ns] = i;
                    J.slot[i] = ns;
                }
                ++ns;
            }
            if (threadIdx.x == 0) J.set[i] = IMG_SET_F;
            log_event(0, i, (float)lam_min);
            __syncthreads();
            flag = true;
        }
    }
    if (!converged && info.status == IMG_OK) info.status = IMG_ENOTCONV;
    if constexpr (MODE != 0) {
        if (T.timeouts && info.status == IMG_OK) info.status = IMG_ETIMEOUT;
        tc_teardown(T, p);
    }
    double *out = sigma_out ? sigma_out[blockIdx.x] : nullptr;
    int nf = 0, nu = 0;
    for (int i = threadIdx.x; i < Q; i += blockDim.x) {
        const double s = (double)J.scale[i] * J.x[i];
        J.sigma[i] = s;
        if (out) out[i] = s;
        nf += J.set[i] == IMG_SET_F;
        nu += J.set[i] == IMG_SET_U;
    }
    const double tf = block_sum((double)nf, S.dbuf);
    const double tu = block_sum((double)nu, S.dbuf);
    if (threadIdx.x == 0) {
        info.outer = outer;
        info.n_free = (int)tf;
        info.n_upper = (int)tu;
        info.converged = converged ? 1 : 0;
        info.lambda_min = lam_min;
        info.cyc_total = (double)(clock64() - t_start);
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(info.t_end_ns));
        *J.ev_count = nev;
        *J.info = info;
        if (batch_info) batch_info[blockIdx.x] = info;
    }
}

// ---------------------------------------------------------------- operators
// K = sum_i x_i a_i a_i^H over all pixels, split over CTAs into partial
// matrices part[b] (p x p each), then summed in order by k_psi_reduce.
__global__ void k_psi_partial(const JobDev *Jp, const float *wx, float2 *part, int per_cta) {
    extern __shared__ float4 smem4[];
    float2 *C = reinterpret_cast<float2 *>(smem4);
    __shared__ float wsm[kTile];
    const JobDev &J = *Jp;
    const int i0 = blockIdx.x * per_cta;
    const int n = max(0, min(per_cta, J.Q - i0));
    const int p = J.p;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float2 *K = part + (size_t)blockIdx.x * p * p;
    for (int mt = 0; mt < p; mt += kTile) {
        for (int nt = 0; nt < p; nt += kTile) {
            const int r0 = mt + ty * 4, c0 = nt + tx * 4;
            float2 acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
            for (int j0 = 0; j0 < n; j0 += kTile) {
                const int np = min(kTile, n - j0);
                for (int e = threadIdx.x; e < kTile * p; e += kThreads) {
                    const int j = e / p, k = e - j * p;
                    float2 c = make_float2(0.f, 0.f);
                    if (j < np) {
                        const int i = i0 + j0 + j;
                        const int im = i / J.n_l, il = i - im * J.n_l;
                        c = steer(J, il, im, k);
                    }
                    C[e] = c;
                }
                if (threadIdx.x < kTile) wsm[threadIdx.x] = threadIdx.x < np ? wx[i0 + j0 + threadIdx.x] : 0.f;
                __syncthreads();
                if (r0 < p && c0 < p) {
                    for (int j = 0; j < np; ++j) {
                        const float wj = wsm[j];
                        const float2 *cj = C + j * p;
                        float2 ck[4], cl[4];
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const float2 t = (r0 + r < p) ? cj[r0 + r] : make_float2(0.f, 0.f);
                            ck[r] = make_float2(wj * t.x, wj * t.y);
                        }
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            const float2 t = (c0 + c < p) ? cj[c0 + c] : make_float2(0.f, 0.f);
                            cl[c] = make_float2(t.x, -t.y);
                        }
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int c = 0; c < 4; ++c) cfma(acc[r][c], ck[r], cl[c]);
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int k = r0 + r, l = c0 + c;
                    if (k < p && l < p) K[(size_t)l * p + k] = acc[r][c];
                }
        }
    }
}

// Tensor-core Psi x: CTA b accumulates pixels [b*per, (b+1)*per) into its
// partial matrix part[b] (Kp = 64).
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) k_psi_partial_tc(const JobDev *Jp, const float *wx, float2 *part,
                                                               int per) {
    const JobDev &J = *Jp;
    constexpr bool BF = MODE == 2;
    extern __shared__ float4 smem4[];
    unsigned char *dyn = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem4) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bars[2];
    __shared__ uint32_t slot;
    __shared__ double dbuf[kThreads / 32];
    TcWork T{};
    tc_carve(T, dyn, J.p);
    tc_setup(T, bars, &slot, J.p);
    const int i0 = blockIdx.x * per;
    const int n = max(0, min(per, J.Q - i0));
    const float sX = tc_steer_scale(J.p);
    tc_forward<BF>(T, J.p, n, wx + i0, sX,
                   [&](int t, int np) { tc_gen_X_range<BF>(J, T, 0, i0 + t * kTcM, np, sX); },
                   nullptr, false, part + (size_t)blockIdx.x * J.p * J.p, dbuf);
    tc_teardown(T, J.p);
}

__global__ void k_psi_reduce(const float2 *part, int nparts, int pp, double2 *Kout) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < pp; e += gridDim.x * blockDim.x) {
        double sx = 0.0, sy = 0.0;
        for (int b = 0; b < nparts; ++b) {
            const float2 v = part[(size_t)b * pp + e];
            sx += v.x;
            sy += v.y;
        }
        Kout[e] = make_double2(sx, sy);
    }
}

__global__ void k_psi_adj(const JobDev *J, const float2 *U, double *out) {
    // out_i = Re(a_i^H U a_i) over all pixels (Psi^H vect(U))
    extern __shared__ float4 smem4[];
    float2 *A = reinterpret_cast<float2 *>(smem4);
    float *red = reinterpret_cast<float *>(A + J->p * kTile);
    const int ntiles = (J->Q + kTile - 1) / kTile;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int pix0 = t * kTile;
        const int np = min(kTile, J->Q - pix0);
        fill_steer_adj(*J, pix0, np, A);
        __syncthreads();
        adj_chunk(U, J->p, A, red);
        if (threadIdx.x < np) out[pix0 + threadIdx.x] = red[threadIdx.x];
        __syncthreads();
    }
}

__global__ void k_to_double(const float *src, double *dst, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

__global__ void k_z2c(const double2 *src, float2 *dst, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

__global__ void k_c2z(const float2 *src, double2 *dst, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = make_double2(src[i].x, src[i].y);
}

__global__ void k_d2f(const double *src, float *dst, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = (float)src[i];
}

// ---------------------------------------------------------------- launchers
size_t solve_smem_bytes(int p, int mode) {
    size_t b = (size_t)p * kTile * sizeof(float2);
    // tensor tiles + forward staging + five LSQR f-vectors of 256 floats
    const size_t tc = tc_smem_bytes(p) + tc_stage_bytes(p) + 10 * kTcM * sizeof(float);
    if (mode != 0) b = b > tc ? b : tc;
    return b + 1024;
}
size_t bounds_smem_bytes(int p) {
    return (size_t)p * kTile * sizeof(float2) + (kTile + 16 * kTile) * sizeof(float);
}

// Raise a kernel's dynamic shared-memory limit (and prefer the maximum
// shared-memory carve-out) only when a launch needs more than any before:
// changing a function's attributes while instances of it run can hold the
// launch back, which serialised independent launches on separate streams.
static std::mutex g_attr_mu;
static std::unordered_map<const void *, size_t> g_attr;

static cudaError_t ensure_smem(const void *func, size_t bytes) {
    std::lock_guard<std::mutex> lock(g_attr_mu);
    auto it = g_attr.find(func);
    if (it != g_attr.end() && it->second >= bytes) return cudaSuccess;
    const size_t want = bytes < 48 * 1024 ? 48 * 1024 : bytes;
    cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)want);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    g_attr[func] = want;
    return cudaSuccess;
}

static int g_num_sms = 0;
static int num_sms() {
    if (!g_num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

cudaError_t launch_tables(JobDev *const *jobs, int n, cudaStream_t st) {
    k_tables<<<dim3(16, n), kThreads, 0, st>>>(jobs);
    return cudaGetLastError();
}

cudaError_t launch_factor(JobDev *const *jobs, int n, cudaStream_t st) {
    k_factor<<<n, kThreads, 0, st>>>(jobs);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_bounds_tc_t(JobDev *const *jobs, int n, int max_tiles, int max_p, cudaStream_t st) {
    const size_t sm = tc_smem_bytes(max_p) + 1024;
    cudaError_t e = ensure_smem((const void *)k_bounds_tc<MODE>, sm);
    if (e != cudaSuccess) return e;
    int per_job = (num_sms() + n - 1) / n;
    per_job = max(1, min(per_job, max_tiles));
    k_bounds_tc<MODE><<<dim3(per_job, n), kThreads, sm, st>>>(jobs);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_bounds_wide_t(JobDev *const *jobs, int n, int max_tiles, int max_p, cudaStream_t st) {
    k_emb_max_bounds<<<dim3(n, 2, 8), kThreads, 0, st>>>(jobs);
    k_emb_bounds<MODE><<<dim3(n, 2, wide_nk(max_p) * (2 * kWideMaxP / kEmbRows)), kThreads, 0, st>>>(jobs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t sm = wide_smem_bytes(max_p);
    e = ensure_smem((const void *)k_bounds_wide<MODE>, sm);
    if (e != cudaSuccess) return e;
    int per_job = (num_sms() + n - 1) / n;
    per_job = max(1, min(per_job, max_tiles));
    k_bounds_wide<MODE><<<dim3(per_job, n), kWideThreads, sm, st>>>(jobs);
    return cudaGetLastError();
}

cudaError_t launch_bounds(JobDev *const *jobs, int n, int max_tiles, int max_p, int mode, cudaStream_t st) {
    if (mode != 0 && max_p > kMaxTcP) {
        if (mode == 1) return launch_bounds_wide_t<1>(jobs, n, max_tiles, max_p, st);
        return launch_bounds_wide_t<2>(jobs, n, max_tiles, max_p, st);
    }
    if (mode == 1) return launch_bounds_tc_t<1>(jobs, n, (max_tiles + 1) / 2, max_p, st);
    if (mode == 2) return launch_bounds_tc_t<2>(jobs, n, (max_tiles + 1) / 2, max_p, st);
    const size_t sm = bounds_smem_bytes(max_p);
    cudaError_t e = ensure_smem((const void *)k_bounds, sm);
    if (e != cudaSuccess) return e;
    int per_job = (2 * num_sms() + n - 1) / n;
    per_job = max(1, min(per_job, max_tiles));
    k_bounds<<<dim3(per_job, n), kThreads, sm, st>>>(jobs);
    return cudaGetLastError();
}

cudaError_t launch_finalize(JobDev *const *jobs, int n, cudaStream_t st, int *batch_status) {
    k_finalize<<<n, kThreads, 0, st>>>(jobs, batch_status);
    return cudaGetLastError();
}

template <int MODE, bool PREP>
static cudaError_t launch_solve_t(JobDev *const *jobs, int n, size_t sm, DevInfo *batch_info,
                                  double *const *sigma_out, cudaStream_t st) {
    cudaError_t e = ensure_smem((const void *)k_solve<MODE, PREP>, sm);
    if (e != cudaSuccess) return e;
    k_solve<MODE, PREP><<<n, kThreads, sm, st>>>(jobs, batch_info, sigma_out);
    return cudaGetLastError();
}

cudaError_t launch_solve(JobDev *const *jobs, int n, int max_p, int mode, DevInfo *batch_info,
                         double *const *sigma_out, cudaStream_t st) {
    const size_t sm = solve_smem_bytes(max_p, mode);
    if (mode == 1) return launch_solve_t<1, false>(jobs, n, sm, batch_info, sigma_out, st);
    if (mode == 2) return launch_solve_t<2, false>(jobs, n, sm, batch_info, sigma_out, st);
    return launch_solve_t<0, false>(jobs, n, sm, batch_info, sigma_out, st);
}

cudaError_t launch_job(JobDev *const *jobs, int n, int max_p, int mode, DevInfo *batch_info,
                       double *const *sigma_out, cudaStream_t st) {
    size_t sm = solve_smem_bytes(max_p, mode);
    if (mode == 0) {
        const size_t b = bounds_smem_bytes(max_p);
        sm = sm > b ? sm : b;
    }
    if (mode == 1) return launch_solve_t<1, true>(jobs, n, sm, batch_info, sigma_out, st);
    if (mode == 2) return launch_solve_t<2, true>(jobs, n, sm, batch_info, sigma_out, st);
    return launch_solve_t<0, true>(jobs, n, sm, batch_info, sigma_out, st);
}

// Psi x over all pixels: nparts CTAs write partial p x p sums into `part`
// (nparts * p * p float2 of scratch), reduced in a fixed order in FP64.
template <int MODE>
static cudaError_t launch_psi_tc_t(const JobDev *job_dev, const float *wx, float2 *part, int nparts, int Q,
                                   int p, double2 *Kout, cudaStream_t st) {
    const size_t sm = tc_smem_bytes(p) + 1024;
    cudaError_t e = ensure_smem((const void *)k_psi_partial_tc<MODE>, sm);
    if (e != cudaSuccess) return e;
    int per = (Q + nparts - 1) / nparts;
    per = ((per + kTcM - 1) / kTcM) * kTcM;
    const int used = (Q + per - 1) / per;
    k_psi_partial_tc<MODE><<<used, kThreads, sm, st>>>(job_dev, wx, part, per);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_psi_reduce<<<(p * p + 255) / 256, 256, 0, st>>>(part, used, p * p, Kout);
    return cudaGetLastError();
}

cudaError_t launch_psi(const JobDev *job_dev, const float *wx, float2 *part, int nparts, int Q,
                       int p, int mode, double2 *Kout, cudaStream_t st) {
    const int Kp = (p + 31) / 32 * 32;
    if (mode == 1 && Kp == 64) return launch_psi_tc_t<1>(job_dev, wx, part, nparts, Q, p, Kout, st);
    if (mode == 2 && Kp == 64) return launch_psi_tc_t<2>(job_dev, wx, part, nparts, Q, p, Kout, st);
    const size_t sm = (size_t)p * kTile * sizeof(float2);
    cudaError_t e = ensure_smem((const void *)k_psi_partial, sm);
    if (e != cudaSuccess) return e;
    int per = (Q + nparts - 1) / nparts;
    per = ((per + kTile - 1) / kTile) * kTile;
    const int used = (Q + per - 1) / per;
    k_psi_partial<<<used, kThreads, sm, st>>>(job_dev, wx, part, per);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_psi_reduce<<<(p * p + 255) / 256, 256, 0, st>>>(part, used, p * p, Kout);
    return cudaGetLastError();
}

// Partial blocks (one per CTA, at most one CTA per SM) followed by the
// summed blocks (at most 12 at Kp = 384, in doubles; room for 16).
size_t psi_wide_part_floats(int sms) { return (size_t)sms * kTcM * 256 + (size_t)2 * 16 * kTcM * 256; }

cudaError_t launch_psi_wide(const JobDev *job_dev, unsigned *wbits, const float *wx, float *part, int Q, int p,
                            int n_l, int n_m, int mode, double2 *Kout, cudaStream_t st) {
    if (p < 1 || p > kMaxWideFwdP || (mode != 1 && mode != 2)) return cudaErrorInvalidValue;
    if (fwd_pairs(p, nullptr, nullptr) > 16) return cudaErrorInvalidValue;
    FwdMap map{};
    map.np = fwd_pairs(p, map.m, map.nb);
    for (int a = 0; a < 6; ++a)
        for (int b = 0; b < 3; ++b) map.idx[a][b] = -1;
    for (int q = 0; q < map.np; ++q) map.idx[map.m[q]][map.nb[q]] = q;
    const int sms = num_sms();
    const int nblk = fwd_nblocks(n_l, n_m);
    const int S = max(1, min(nblk, sms / map.np));
    cudaError_t e = cudaMemsetAsync(wbits, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    k_fwd_wmax<<<max(1, min(2 * sms, (Q + 4 * kThreads - 1) / (4 * kThreads))), kThreads, 0, st>>>(wx, Q, wbits);
    const size_t sm = fwd_smem_bytes();
    e = (mode == 1) ? ensure_smem((const void *)k_fwd_wide<1>, sm) : ensure_smem((const void *)k_fwd_wide<2>, sm);
    if (e != cudaSuccess) return e;
    if (mode == 1)
        k_fwd_wide<1><<<dim3(S, map.np), kFwdThreads, sm, st>>>(job_dev, wx, wbits, map, part);
    else
        k_fwd_wide<2><<<dim3(S, map.np), kFwdThreads, sm, st>>>(job_dev, wx, wbits, map, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double *Ub = reinterpret_cast<double *>(part + (size_t)sms * kTcM * 256);
    const int nent = map.np * kTcM * 256;
    k_fwd_reduce<<<(nent + 63) / 64, 256, 0, st>>>(part, S, nent, Ub);
    k_fwd_assemble<<<(p * p + kThreads - 1) / kThreads, kThreads, 0, st>>>(p, Ub, map, wbits, Kout);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- full-image LSQR launchers
static inline int ls_grid(int n) { return max(1, min(4 * num_sms(), (n + kThreads - 1) / kThreads)); }

cudaError_t ls_forward(const JobDev *jd, const JobDev &hj, LsBufs &b, int mode, float *fwd_part, float2 *part,
                       int nparts, cudaStream_t st) {
    const int Q = hj.Q, p = hj.p, pp = p * p;
    k_ls_weights<<<ls_grid(Q), kThreads, 0, st>>>(hj.scale, b.v, b.wx, Q);
    cudaError_t e = mode != 0 ? launch_psi_wide(jd, hj.Bmax + 1, b.wx, fwd_part, Q, p, hj.n_l, hj.n_m, mode, b.Kd, st)
                              : launch_psi(jd, b.wx, part, nparts, Q, p, 0, b.Kd, st);
    if (e != cudaSuccess) return e;
    k_d2c<<<ls_grid(pp), kThreads, 0, st>>>(b.Kd, b.Mv, pp);
    if (hj.cost == IMG_COST_PWLS) {
        // W vect(K) = vect(L^-1 K L^-H)
        const dim3 g((p + 31) / 32, (p + 31) / 32);
        k_cgemm<<<g, kThreads, 0, st>>>(p, b.Mv, 0, hj.Li32, 1, b.T1);
        k_cgemm<<<g, kThreads, 0, st>>>(p, hj.Li32, 0, b.T1, 0, b.Mv);
    }
    return cudaGetLastError();
}

cudaError_t ls_adjoint(const JobDev *jd, const JobDev &hj, LsBufs &b, int mode, cudaStream_t st) {
    const int Q = hj.Q, p = hj.p;
    const float2 *U = b.u;
    if (hj.cost == IMG_COST_PWLS) {
        // W^H vect(u) = vect(L^-H u L^-1)
        const dim3 g((p + 31) / 32, (p + 31) / 32);
        k_cgemm<<<g, kThreads, 0, st>>>(p, b.u, 0, hj.Li32, 0, b.T1);
        k_cgemm<<<g, kThreads, 0, st>>>(p, hj.Li32, 1, b.T1, 0, b.Uw);
        U = b.Uw;
    }
    cudaError_t e = mode != 0 ? launch_psi_adj_wide(jd, hj.Bmax, U, false, b.y, Q, p, mode, st)
                              : launch_psi_adj(jd, U, b.y, Q, p, 0, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t ls_begin(const JobDev *jd, const JobDev &hj, LsBufs &b, int mode, cudaStream_t st) {
    const int Q = hj.Q, p = hj.p, pp = p * p;
    k_ls_init_u<<<ls_grid(pp), kThreads, 0, st>>>(hj.R32, p, hj.cost == IMG_COST_PWLS, b.u);
    k_sumsq<<<1, 1024, 0, st>>>(reinterpret_cast<const float *>(b.u), 2 * pp, b.sc + kLsSsU);
    k_ls_scalar<<<1, 32, 0, st>>>(b.sc, 0);
    k_ls_scale_u<<<ls_grid(pp), kThreads, 0, st>>>(b.u, pp, b.sc);
    cudaError_t e = ls_adjoint(jd, hj, b, mode, st);
    if (e != cudaSuccess) return e;
    k_ls_v<<<ls_grid(Q), kThreads, 0, st>>>(b.v, b.y, hj.scale, Q, b.sc, 1);
    k_sumsq<<<1, 1024, 0, st>>>(b.v, Q, b.sc + kLsSsV);
    k_ls_scalar<<<1, 32, 0, st>>>(b.sc, 1);
    k_ls_xw<<<ls_grid(Q), kThreads, 0, st>>>(b.x, b.w, b.v, Q, b.sc, 1);
    return cudaGetLastError();
}

cudaError_t ls_iterate(const JobDev *jd, const JobDev &hj, LsBufs &b, int mode, float *fwd_part, float2 *part,
                       int nparts, cudaStream_t st) {
    const int Q = hj.Q, pp = hj.p * hj.p;
    // u <- M v - alpha u, beta = ||u||, u <- u / beta
    cudaError_t e = ls_forward(jd, hj, b, mode, fwd_part, part, nparts, st);
    if (e != cudaSuccess) return e;
    k_ls_u<<<ls_grid(pp), kThreads, 0, st>>>(b.u, b.Mv, pp, b.sc);
    k_sumsq<<<1, 1024, 0, st>>>(reinterpret_cast<const float *>(b.u), 2 * pp, b.sc + kLsSsU);
    k_ls_scalar<<<1, 32, 0, st>>>(b.sc, 2);
    k_ls_scale_u<<<ls_grid(pp), kThreads, 0, st>>>(b.u, pp, b.sc);
    // v <- M^H u - beta v, alpha = ||v||, rotation, x and w updates
    e = ls_adjoint(jd, hj, b, mode, st);
    if (e != cudaSuccess) return e;
    k_ls_v<<<ls_grid(Q), kThreads, 0, st>>>(b.v, b.y, hj.scale, Q, b.sc, 0);
    k_sumsq<<<1, 1024, 0, st>>>(b.v, Q, b.sc + kLsSsV);
    k_ls_scalar<<<1, 32, 0, st>>>(b.sc, 3);
    k_ls_xw<<<ls_grid(Q), kThreads, 0, st>>>(b.x, b.w, b.v, Q, b.sc, 0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- K-snapshot full-image LSQR
// y = first ? yk : y + yk (the snapshot sum of M^H u, snapshot order fixed).
__global__ void k_ls_accum(double *y, const double *yk, int Q, int first) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q; i += gridDim.x * blockDim.x)
        y[i] = first ? yk[i] : y[i] + yk[i];
}

// Pixel scale of the K-snapshot solver variable: 1/D with
// D = (sum_k h_k)^2 / (K C) for PWLS (eq. D), 1 for CLS.
__global__ void k_snap_scale(SnapPtrs sp, int K, int Q, int pwls, double C, float *scale) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q; i += gridDim.x * blockDim.x) {
        double hs = 0.0;
        for (int k = 0; k < K; ++k) hs += (double)sp.h[k][i];
        scale[i] = pwls ? (float)(1.0 / ((hs * hs) / ((double)K * C))) : 1.0f;
    }
}

cudaError_t launch_snap_scale(const SnapPtrs &sp, int K, int Q, int pwls, double C, float *scale, cudaStream_t st) {
    k_snap_scale<<<ls_grid(Q), kThreads, 0, st>>>(sp, K, Q, pwls, C, scale);
    return cudaGetLastError();
}

// Buffers of snapshot k: its block of u and M v, the shared scratch, and the
// per-snapshot adjoint output yk.
static LsBufs snap_bufs(const LsSnap &s, const LsBufs &b, int k) {
    LsBufs bk = b;
    const size_t pp = (size_t)s.hj[0].p * s.hj[0].p;
    bk.u = b.u + (size_t)k * pp;
    bk.Mv = b.Mv + (size_t)k * pp;
    bk.y = s.yk;
    return bk;
}

// y = sum_k M_k^H u_k.
static cudaError_t snap_adjoint(const LsSnap &s, LsBufs &b, cudaStream_t st) {
    const int Q = s.hj[0].Q;
    for (int k = 0; k < s.K; ++k) {
        LsBufs bk = snap_bufs(s, b, k);
        cudaError_t e = ls_adjoint(s.jd[k], s.hj[k], bk, s.mode[k], st);
        if (e != cudaSuccess) return e;
        k_ls_accum<<<ls_grid(Q), kThreads, 0, st>>>(b.y, s.yk, Q, k == 0);
    }
    return cudaGetLastError();
}

// M_k v into block k of b.Mv for every snapshot.
static cudaError_t snap_forward(const LsSnap &s, LsBufs &b, cudaStream_t st) {
    for (int k = 0; k < s.K; ++k) {
        LsBufs bk = snap_bufs(s, b, k);
        cudaError_t e = ls_forward(s.jd[k], s.hj[k], bk, s.mode[k], s.fwd_part[k], s.part[k], s.nparts[k], st);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

cudaError_t ls_snap_begin(const LsSnap &s, LsBufs &b, cudaStream_t st) {
    const int Q = s.hj[0].Q, p = s.hj[0].p, pp = p * p, n = s.K * pp;
    const int pwls = s.hj[0].cost == IMG_COST_PWLS;
    for (int k = 0; k < s.K; ++k)
        k_ls_init_u<<<ls_grid(pp), kThreads, 0, st>>>(s.hj[k].R32, p, pwls, b.u + (size_t)k * pp);
    k_sumsq<<<1, 1024, 0, st>>>(reinterpret_cast<const float *>(b.u), 2 * n, b.sc + kLsSsU);
    k_ls_scalar<<<1, 32, 0, st>>>(b.sc, 0);
    k_ls_scale_u<<<ls_grid(n), kThreads, 0, st>>>(b.u, n, b.sc);
    cudaError_t e = snap_adjoint(s, b, st);
    if (e != cudaSuccess) return e;
    k_ls_v<<<ls_grid(Q), kThreads, 0, st>>>(b.v, b.y, s.hj[0].scale, Q, b.sc, 1);
    k_sumsq<<<1, 1024, 0, st>>>(b.v, Q, b.sc + kLsSsV);
    k_ls_scalar<<<1, 32, 0, st>>>(b.sc, 1);
    k_ls_xw<<<ls_grid(Q), kThreads, 0, st>>>(b.x, b.w, b.v, Q, b.sc, 1);
    return cudaGetLastError();
}

cudaError_t ls_snap_iterate(const LsSnap &s, LsBufs &b, cudaStream_t st) {
    const int Q = s.hj[0].Q, pp = s.hj[0].p * s.hj[0].p, n = s.K * pp;
    cudaError_t e = snap_forward(s, b, st);
    if (e != cudaSuccess) return e;
    k_ls_u<<<ls_grid(n), kThreads, 0, st>>>(b.u, b.Mv, n, b.sc);
    k_sumsq<<<1, 1024, 0, st>>>(reinterpret_cast<const float *>(b.u), 2 * n, b.sc + kLsSsU);
    k_ls_scalar<<<1, 32, 0, st>>>(b.sc, 2);
    k_ls_scale_u<<<ls_grid(n), kThreads, 0, st>>>(b.u, n, b.sc);
    e = snap_adjoint(s, b, st);
    if (e != cudaSuccess) return e;
    k_ls_v<<<ls_grid(Q), kThreads, 0, st>>>(b.v, b.y, s.hj[0].scale, Q, b.sc, 0);
    k_sumsq<<<1, 1024, 0, st>>>(b.v, Q, b.sc + kLsSsV);
    k_ls_scalar<<<1, 32, 0, st>>>(b.sc, 3);
    k_ls_xw<<<ls_grid(Q), kThreads, 0, st>>>(b.x, b.w, b.v, Q, b.sc, 0);
    return cudaGetLastError();
}

cudaError_t ls_finish(const JobDev &hj, LsBufs &b, double *sigma, double *xnorm2, cudaStream_t st) {
    k_ls_sigma<<<ls_grid(hj.Q), kThreads, 0, st>>>(b.x, hj.scale, sigma, hj.Q);
    if (xnorm2) k_sumsq<<<1, 1024, 0, st>>>(b.x, hj.Q, xnorm2);
    return cudaGetLastError();
}

cudaError_t ls_xnorm2(const JobDev &hj, LsBufs &b, double *out, cudaStream_t st) {
    k_sumsq<<<1, 1024, 0, st>>>(b.x, hj.Q, out);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_psi_adj_tc_t(const JobDev *job_dev, const float2 *U, double *out, int Q, int p,
                                       cudaStream_t st) {
    const size_t sm = tc_smem_bytes(p) + 1024;
    cudaError_t e = ensure_smem((const void *)k_psi_adj_tc<MODE>, sm);
    if (e != cudaSuccess) return e;
    const int ntiles = (Q + kTcM - 1) / kTcM;
    k_psi_adj_tc<MODE><<<min(ntiles, num_sms()), kThreads, sm, st>>>(job_dev, U, out);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_psi_adj_wide_t(const JobDev *job_dev, unsigned *bmax, const void *U, bool u64,
                                         double *out, int Q, int p, cudaStream_t st) {
    const dim3 eg(wide_nk(p), 2 * wide_kp(p) / kEmbRows);
    cudaError_t e = cudaMemsetAsync(bmax, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const int nmax = min(16, (p * p + kThreads - 1) / kThreads);
    if (u64) {
        k_emb_max_one<double2><<<nmax, kThreads, 0, st>>>(job_dev, static_cast<const double2 *>(U));
        k_emb_one<MODE, double2><<<eg, kThreads, 0, st>>>(job_dev, static_cast<const double2 *>(U));
    } else {
        k_emb_max_one<float2><<<nmax, kThreads, 0, st>>>(job_dev, static_cast<const float2 *>(U));
        k_emb_one<MODE, float2><<<eg, kThreads, 0, st>>>(job_dev, static_cast<const float2 *>(U));
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t sm = wide_smem_bytes(p);
    e = ensure_smem((const void *)k_psi_adj_wide<MODE>, sm);
    if (e != cudaSuccess) return e;
    const int ntiles = (Q + kTcM - 1) / kTcM + 64;   // >= 2-D tiles of any grid
    k_psi_adj_wide<MODE><<<min(ntiles, num_sms()), kWideThreads, sm, st>>>(job_dev, out);
    return cudaGetLastError();
}

cudaError_t launch_psi_adj_wide(const JobDev *job_dev, unsigned *bmax, const void *U, bool u64, double *out,
                                int Q, int p, int mode, cudaStream_t st) {
    if (p < 1 || p > kMaxWideP || (mode != 1 && mode != 2)) return cudaErrorInvalidValue;
    if (mode == 1) return launch_psi_adj_wide_t<1>(job_dev, bmax, U, u64, out, Q, p, st);
    return launch_psi_adj_wide_t<2>(job_dev, bmax, U, u64, out, Q, p, st);
}

cudaError_t launch_psi_adj(const JobDev *job_dev, const float2 *U, double *out, int Q, int p, int mode,
                           cudaStream_t st) {
    if (mode != 0 && p > kMaxTcP) return cudaErrorInvalidValue;   // wide arrays: launch_psi_adj_wide
    if (mode == 1) return launch_psi_adj_tc_t<1>(job_dev, U, out, Q, p, st);
    if (mode == 2) return launch_psi_adj_tc_t<2>(job_dev, U, out, Q, p, st);
    const size_t sm = bounds_smem_bytes(p);
    cudaError_t e = ensure_smem((const void *)k_psi_adj, sm);
    if (e != cudaSuccess) return e;
    const int ntiles = (Q + kTile - 1) / kTile;
    k_psi_adj<<<min(ntiles, 2 * num_sms()), kThreads, sm, st>>>(job_dev, U, out);
    return cudaGetLastError();
}

cudaError_t launch_z2c(const double2 *src, float2 *dst, int n, cudaStream_t st) {
    k_z2c<<<min(1024, (n + 255) / 256 + 1), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_c2z(const float2 *src, double2 *dst, int n, cudaStream_t st) {
    k_c2z<<<min(1024, (n + 255) / 256 + 1), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

cudaError_t launch_d2f(const double *src, float *dst, int n, cudaStream_t st) {
    k_d2f<<<min(1024, (n + 255) / 256 + 1), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

// Dirty images over K snapshots from each snapshot's MF image d_k and MVDR
// denominator h_k = a_{i,k}^H R_k^-1 a_{i,k} (Sec. III-C, Sec. III-D,
// eq. ASSC0): MF (1/K) sum d_k, MVDR C K / sum h_k, ASSC C / max h_k.
// FP64, snapshot order fixed.
__global__ void k_snapshot_image(SnapPtrs sp, int K, int Q, int kind, double C, double *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q; i += gridDim.x * blockDim.x) {
        double acc = 0.0;
        if (kind == IMG_SNAP_MF) {
            for (int k = 0; k < K; ++k) acc += (double)sp.d[k][i];
            out[i] = acc / (double)K;
        } else if (kind == IMG_SNAP_MVDR) {
            for (int k = 0; k < K; ++k) acc += (double)sp.h[k][i];
            out[i] = (C * (double)K) / acc;
        } else {
            for (int k = 0; k < K; ++k) acc = fmax(acc, (double)sp.h[k][i]);
            out[i] = C / acc;
        }
    }
}

cudaError_t launch_snapshot_image(const SnapPtrs &sp, int K, int Q, int kind, double C, double *out,
                                  cudaStream_t st) {
    k_snapshot_image<<<min(1024, (Q + 255) / 256), 256, 0, st>>>(sp, K, Q, kind, C, out);
    return cudaGetLastError();
}

cudaError_t launch_to_double(const float *src, double *dst, int n, cudaStream_t st) {
    k_to_double<<<min(1024, (n + 255) / 256 + 1), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

}  // namespace img
