// CTA-level building blocks: complex helpers, block reductions, and the
// Khatri-Rao operator pair on CUDA cores (FP32, 256 threads, 64-pixel chunks).
//
//   adjoint  out_j = Re(c_j^H U c_j)                 (Psi^H vect(U), Sec. V-B)
//   forward  K = base + sum_j w_j c_j c_j^H          (Psi w = vect(A diag(w) A^H))
//
// The vectors c_j are either steering vectors generated from the separable
// tables or cached (whitened) steering vectors of the support set.
#pragma once
#include "img_internal.cuh"

namespace img {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zmulc(double2 a, double2 b) {  // a * conj(b)
    return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Steering vector element a_{k,i} from the separable tables.
__device__ __forceinline__ float2 steer(const JobDev &J, int il, int im, int k) {
    return cmul(J.El[il * J.p + k], J.Em[im * J.p + k]);
}

// ---------------------------------------------------------------- reductions
// Sum over the CTA; every thread receives the same value (fixed order).
__device__ __forceinline__ double block_sum(double v, double *sbuf) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) sbuf[warp] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) t += sbuf[w];
    __syncthreads();
    return t;
}

// Lexicographic (value, index) minimum over the CTA; ties go to the smaller
// index.  Every thread receives the result.
__device__ __forceinline__ void block_argmin(double &v, int &idx, double *sv, int *si) {
    for (int o = 16; o; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, idx, o);
        if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) { sv[warp] = v; si[warp] = idx; }
    __syncthreads();
    v = sv[0];
    idx = si[0];
#pragma unroll
    for (int w = 1; w < kThreads / 32; ++w) {
        if (sv[w] < v || (sv[w] == v && si[w] < idx)) { v = sv[w]; idx = si[w]; }
    }
    __syncthreads();
}

// Ordered compaction: out[k] = the k-th position in [0, n) whose predicate
// holds.  Returns the count (same in every thread).
template <class Pred>
__device__ int block_compact(int n, Pred pred, int *out, int *sbuf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int total = 0;
    for (int base = 0; base < n; base += kThreads) {
        const int pos = base + threadIdx.x;
        const bool p = pos < n && pred(pos);
        const unsigned m = __ballot_sync(0xffffffffu, p);
        if (lane == 0) sbuf[warp] = __popc(m);
        __syncthreads();
        int off = total;
        for (int w = 0; w < warp; ++w) off += sbuf[w];
        int chunk_total = 0;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) chunk_total += sbuf[w];
        if (p) out[off + __popc(m & ((1u << lane) - 1u))] = pos;
        total += chunk_total;
        __syncthreads();
    }
    return total;
}

// ---------------------------------------------------------------- adjoint
// Shared-memory chunk for the adjoint: A[k * kTile + j], k < p, j < kTile.
// Computes part_j = sum_k Re(conj(A[k][j]) (U A)[k][j]) and leaves the
// per-pixel sums in red[0..kTile) (valid after the call, before the next
// __syncthreads of the caller).  U is p x p column-major in global memory.
// SQ: part_j = ||(U A)[:][j]||^2 instead (with U = L^-1: the whitened MVDR
// denominator ||L^-1 a_j||^2, whose rounding error is relative to itself).
template <bool SQ = false>
__device__ __forceinline__ void adj_chunk(const float2 *U, int p,
                                          const float2 *A, float *red) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float part[4] = {0.f, 0.f, 0.f, 0.f};
    for (int mt = 0; mt < p; mt += kTile) {
        const int r0 = mt + ty * 4;
        if (r0 < p) {
            float2 y[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) y[r][c] = make_float2(0.f, 0.f);
            const int nr = min(4, p - r0);
            for (int l = 0; l < p; ++l) {
                const float4 *ap = reinterpret_cast<const float4 *>(A + l * kTile + tx * 4);
                const float4 a01 = ap[0], a23 = ap[1];
                const float2 a[4] = {make_float2(a01.x, a01.y), make_float2(a01.z, a01.w),
                                     make_float2(a23.x, a23.y), make_float2(a23.z, a23.w)};
                const float2 *up = U + (size_t)l * p + r0;
                float2 u[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) u[r] = (r < nr) ? up[r] : make_float2(0.f, 0.f);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) cfma(y[r][c], u[r], a[c]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                if (r < nr) {
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        if (SQ) {
                            part[c] = fmaf(y[r][c].x, y[r][c].x, fmaf(y[r][c].y, y[r][c].y, part[c]));
                        } else {
                            const float2 a = A[(r0 + r) * kTile + tx * 4 + c];
                            part[c] = fmaf(a.x, y[r][c].x, fmaf(a.y, y[r][c].y, part[c]));
                        }
                    }
                }
            }
        }
    }
    // red2[ty][j] then column sums into red[j]
    float *red2 = red + kTile;
#pragma unroll
    for (int c = 0; c < 4; ++c) red2[ty * kTile + tx * 4 + c] = part[c];
    __syncthreads();
    if (threadIdx.x < kTile) {
        float s = 0.f;
#pragma unroll
        for (int t = 0; t < 16; ++t) s += red2[t * kTile + threadIdx.x];
        red[threadIdx.x] = s;
    }
    __syncthreads();
}

// Fill the adjoint chunk with steering vectors of pixels pix0 .. pix0+np-1.
__device__ __forceinline__ void fill_steer_adj(const JobDev &J, int pix0, int np, float2 *A) {
    const int p = J.p;
    for (int e = threadIdx.x; e < p * kTile; e += kThreads) {
        const int k = e / kTile, j = e - k * kTile;
        float2 a = make_float2(0.f, 0.f);
        if (j < np) {
            const int i = pix0 + j;
            const int im = i / J.n_l, il = i - im * J.n_l;
            a = steer(J, il, im, k);
        }
        A[e] = a;
    }
}

// Fill the adjoint chunk with cached vectors cvec[pos[j]] (pos == nullptr:
// positions j0 + j).
__device__ __forceinline__ void fill_cache_adj(const JobDev &J, const int *pos, int j0, int np,
                                               float2 *A) {
    const int p = J.p;
    for (int e = threadIdx.x; e < p * kTile; e += kThreads) {
        const int j = e / p, k = e - j * p;
        float2 a = make_float2(0.f, 0.f);
        if (j < np) {
            const int sl = pos ? pos[j0 + j] : j0 + j;
            a = J.cvec[(size_t)sl * p + k];
        }
        A[k * kTile + j] = a;
    }
}

// ---------------------------------------------------------------- forward
// K = base_scale * base + sum_j wt[j] c_j c_j^H for list entries j < n.
// base == nullptr and base_identity: base is the identity matrix.
// Entries come from the support cache (pos[j] or j) or, when gen != 0, are
// steering vectors of pixels j (pos ignored, weights wt[j] per pixel).
// C: shared chunk of kTile * p float2 laid out [j][k]; wsm: kTile floats.
__device__ inline void forward_list(const JobDev &J, const int *pos, const float *wt, int n, bool gen,
                             const float2 *base, bool base_identity, float2 *K, float2 *C,
                             float *wsm) {
    const int p = J.p;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
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
                        if (gen) {
                            const int i = j0 + j;
                            const int im = i / J.n_l, il = i - im * J.n_l;
                            c = steer(J, il, im, k);
                        } else {
                            const int sl = pos ? pos[j0 + j] : j0 + j;
                            c = J.cvec[(size_t)sl * p + k];
                        }
                    }
                    C[e] = c;
                }
                if (threadIdx.x < kTile) wsm[threadIdx.x] = threadIdx.x < np ? wt[j0 + threadIdx.x] : 0.f;
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
            for (int r = 0; r < 4; ++r) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int k = r0 + r, l = c0 + c;
                    if (k < p && l < p) {
                        float2 b = make_float2(0.f, 0.f);
                        if (base) b = base[(size_t)l * p + k];
                        else if (base_identity && k == l) b = make_float2(1.f, 0.f);
                        K[(size_t)l * p + k] = make_float2(b.x + acc[r][c].x, b.y + acc[r][c].y);
                    }
                }
            }
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- small GEMM
// C = op(A) * B for p x p complex column-major matrices in global memory
// (plain loads: the operands may have been written earlier in the same kernel).
// op(A) = A (conjA = false) or A^H (conjA = true).  C must not alias A or B.
__device__ inline void cgemm_pp(int p, const float2 *A, bool conjA, const float2 *B, float2 *Cm) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    for (int mt = 0; mt < p; mt += kTile) {
        for (int nt = 0; nt < p; nt += kTile) {
            const int r0 = mt + ty * 4, c0 = nt + tx * 4;
            if (r0 >= p || c0 >= p) continue;
            float2 acc[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
            for (int k = 0; k < p; ++k) {
                float2 a[4], b[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int i = r0 + r;
                    if (i < p) {
                        if (conjA) {
                            const float2 t = A[(size_t)i * p + k];
                            a[r] = make_float2(t.x, -t.y);
                        } else {
                            a[r] = A[(size_t)k * p + i];
                        }
                    } else {
                        a[r] = make_float2(0.f, 0.f);
                    }
                }
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int j = c0 + c;
                    b[c] = (j < p) ? B[(size_t)j * p + k] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) cfma(acc[r][c], a[r], b[c]);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int i = r0 + r, j = c0 + c;
                    if (i < p && j < p) Cm[(size_t)j * p + i] = acc[r][c];
                }
        }
    }
    __syncthreads();
}

}  // namespace img
