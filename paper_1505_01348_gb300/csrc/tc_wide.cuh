// Tensor-core adjoint Psi^H for wide arrays, 64 < p <= 256 (Kp = p rounded
// up to 32, N = K = 2Kp <= 512): out_i = x_i^T B x_i as in tc_ops.cuh, but
// the 2Kp x 2Kp operand B no longer fits in shared memory.  k_emb_B writes B
// once per operator to global memory as K-chunks of 64 columns, each the
// exact shared-memory image of a swizzled K-major tile (hi part then lo part),
// and the operator kernel streams chunk c into shared memory with a bulk TMA
// copy (cp.async.bulk, completion counted in bytes on an mbarrier) while the
// CTA generates the matching 64-column chunk of the steering tile; chunks are
// double-buffered so copies and generation overlap the MMAs of the previous
// chunk.  The FP32 accumulator (2Kp columns of tensor memory) sums the chunks;
// the epilogue rebuilds x_i from the steering tables.
#pragma once
#include "tc_ops.cuh"

namespace img {

constexpr int kWideMaxP = 256;
constexpr int kChunkK = 64;                 // K columns per streamed chunk

__host__ __device__ inline int wide_kp(int p) { return (p + 31) / 32 * 32; }
// Bytes of one global B chunk (hi + lo): N rows x 128 bytes, twice.
__host__ __device__ inline size_t wide_chunk_bytes(int p) { return (size_t)2 * (2 * wide_kp(p)) * 128; }
// Bytes of the whole chunked B image.
__host__ __device__ inline size_t wide_B_bytes(int p) {
    return wide_chunk_bytes(p) * (2 * wide_kp(p) / kChunkK);
}
// Shared memory: two X chunks (128 rows x 128 B, hi + lo) and one or two B
// chunks (two when N <= 256).
__host__ __device__ inline int wide_nb(int p) { return 2 * wide_kp(p) <= 256 ? 2 : 1; }
__host__ __device__ inline size_t wide_smem_bytes(int p) {
    return (size_t)2 * 2 * kTcM * 128 + (size_t)wide_nb(p) * wide_chunk_bytes(p) + 1024;
}
__host__ __device__ inline uint32_t wide_tmem_cols(int p) {
    const int n = 2 * wide_kp(p);
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

// ---------------------------------------------------------------- TMA bulk copy
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Global -> shared bulk copy of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completing on `bar`.
__device__ __forceinline__ void tma_bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------- B image
// One CTA writes the chunked image of B = emb(U) (rows [Re V, -Im V],
// [Im V, Re V] with V = U^H, the same quadratic form) scaled by a power of
// two to unit range; *scale receives that factor.
template <bool BF16>
__device__ void emb_B_cta(const float2 *U, int p, unsigned char *img, float *scale) {
    const int Kp = wide_kp(p), nc8 = Kp / 8;
    __shared__ float sred[kThreads / 32];
    float mx = 0.f;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x)
        mx = fmaxf(mx, fmaxf(fabsf(U[e].x), fabsf(U[e].y)));
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) mx = fmaxf(mx, sred[w]);
    const float sc = mx > 0.f ? exp2f(-ceilf(log2f(mx))) : 1.f;
    if (threadIdx.x == 0) *scale = sc;
    const size_t cb = wide_chunk_bytes(p), half = cb / 2;
    for (int it = threadIdx.x; it < Kp * nc8; it += blockDim.x) {
        const int n = it / nc8, c8 = it - n * nc8;
        const int k0 = c8 * 8;
        float re[8], im[8], nim[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float2 u = make_float2(0.f, 0.f);
            if (n < p && k0 + e < p) u = U[(size_t)n * p + k0 + e];   // U(k, n) = conj(V(n, k))
            re[e] = u.x * sc;
            im[e] = -u.y * sc;
            nim[e] = u.y * sc;
        }
        // column chunk c (8 columns): K-chunk kc = c / 8, chunk cc = c % 8 in it
        auto put = [&](int row, int c, const float *v) {
            uint4 hi, lo;
            split8<BF16>(v, hi, lo);
            const int kc = c >> 3, cc = c & 7;
            const size_t off = (size_t)kc * cb + (size_t)(row >> 3) * 1024 + (row & 7) * 128 +
                               ((cc ^ (row & 7)) << 4);
            *reinterpret_cast<uint4 *>(img + off) = hi;
            *reinterpret_cast<uint4 *>(img + off + half) = lo;
        };
        put(n, c8, re);              // (re row, re col): Re V
        put(Kp + n, nc8 + c8, re);   // (im row, im col): Re V
        put(n, nc8 + c8, nim);       // (re row, im col): -Im V
        put(Kp + n, c8, im);         // (im row, re col): Im V
    }
}

// ---------------------------------------------------------------- operator
struct WideWork {
    unsigned char *X[2];      // X chunk buffers (hi at +0, lo at +16 KB)
    unsigned char *B[2];      // B chunk buffers (one or two)
    uint64_t *barB;           // 2 barriers: a B chunk landed
    uint64_t *barM;           // 2 barriers: the MMAs of a chunk completed
    uint32_t phB[2], phM[2];
    int issued[2], waited[2]; // MMA commits per barrier (all threads agree)
    uint32_t tmem;
    int Kp, nb, timeouts;
};

__device__ inline void wide_setup(WideWork &W, unsigned char *base, uint64_t *bars, uint32_t *slot, int p) {
    W.Kp = wide_kp(p);
    W.nb = wide_nb(p);
    W.X[0] = base;
    W.X[1] = base + 2 * kTcM * 128;
    W.B[0] = base + 4 * kTcM * 128;
    W.B[1] = W.B[0] + wide_chunk_bytes(p);
    W.barB = bars;
    W.barM = bars + 2;
    W.phB[0] = W.phB[1] = W.phM[0] = W.phM[1] = 0;
    W.issued[0] = W.issued[1] = W.waited[0] = W.waited[1] = 0;
    W.timeouts = 0;
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) mbar_init(&bars[k], 1);
    if (threadIdx.x < 32) tmem_alloc(slot, wide_tmem_cols(p));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    W.tmem = *slot;
}

// Wait for the oldest outstanding MMA commit on barrier b, if any.
__device__ __forceinline__ void wide_wait_mma(WideWork &W, int b) {
    if (W.waited[b] < W.issued[b]) {
        if (!mbar_wait(&W.barM[b], W.phM[b])) W.timeouts++;
        W.phM[b] ^= 1u;
        W.waited[b]++;
    }
}

__device__ inline void wide_teardown(WideWork &W, int p) {
    wide_wait_mma(W, 0);
    wide_wait_mma(W, 1);
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(W.tmem, wide_tmem_cols(p));
}

// Chunk kc (columns kc*64 .. kc*64+63 of the 2Kp) of the steering tile t
// into X buffer b.  Column col < Kp holds Re a_col, col >= Kp holds
// Im a_(col-Kp); an 8-column group never straddles the boundary (Kp is a
// multiple of 32), but a 64-column chunk may.
template <bool BF16>
__device__ inline void wide_gen_X(const JobDev &J, const WideWork &W, int b, int t, int kc, float sX) {
    const int p = J.p, Kp = W.Kp, nl = J.n_l;
    unsigned char *xh = W.X[b], *xl = W.X[b] + kTcM * 128;
    const float2 *__restrict__ El = J.El;
    const float2 *__restrict__ Em = J.Em;
    for (int it = threadIdx.x; it < kTcM * 8; it += blockDim.x) {
        const int r = it >> 3, c8 = it & 7;
        const int i = tc_tile_pixel(t, r, nl, J.n_m);
        const int col = kc * kChunkK + c8 * 8;
        const bool re_part = col < Kp;
        const int k0 = re_part ? col : col - Kp;
        float v[8];
        if (i >= 0) {
            const int mm = i / nl, ll = i - mm * nl;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = k0 + q;
                float2 a = make_float2(0.f, 0.f);
                if (k < p) a = cmul(__ldg(El + (size_t)ll * p + k), __ldg(Em + (size_t)mm * p + k));
                v[q] = (re_part ? a.x : a.y) * sX;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) v[q] = 0.f;
        }
        uint4 hi, lo;
        split8<BF16>(v, hi, lo);
        const uint32_t off = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c8 ^ (r & 7)) << 4));
        *reinterpret_cast<uint4 *>(xh + off) = hi;
        *reinterpret_cast<uint4 *>(xl + off) = lo;
    }
}

// MMAs of one K-chunk: X buffer bx (128 rows) against B buffer bb (N rows),
// 4 K-steps x 3 split products; N above 256 takes a second MMA per step.
__device__ inline void wide_issue(const WideWork &W, int bx, int bb, bool first, int BF) {
    const int N = 2 * W.Kp;
    const int n_lo = N <= 256 ? N : 256, n_hi = N - n_lo;
    const uint32_t id_lo = idesc_f16(n_lo, BF), id_hi = idesc_f16(n_hi > 0 ? n_hi : 16, BF);
    tc_fence_after();
    const uint32_t xh = smem_u32(W.X[bx]), xl = xh + kTcM * 128;
    const uint32_t bh = smem_u32(W.B[bb]), bl = bh + N * 128;
    for (int s = 0; s < kChunkK / 16; ++s) {
        const uint32_t o = s * 32;
        const uint32_t acc = (first && s == 0) ? 0u : 1u;
        mma_f16(W.tmem, sw128_desc(xh + o), sw128_desc(bh + o), id_lo, acc);
        mma_f16(W.tmem, sw128_desc(xh + o), sw128_desc(bl + o), id_lo, 1u);
        mma_f16(W.tmem, sw128_desc(xl + o), sw128_desc(bh + o), id_lo, 1u);
        if (n_hi > 0) {
            const uint32_t bo = (uint32_t)n_lo * 128, d = W.tmem + (uint32_t)n_lo;
            mma_f16(d, sw128_desc(xh + o), sw128_desc(bh + bo + o), id_hi, acc);
            mma_f16(d, sw128_desc(xh + o), sw128_desc(bl + bo + o), id_hi, 1u);
            mma_f16(d, sw128_desc(xl + o), sw128_desc(bh + bo + o), id_hi, 1u);
        }
    }
}

// out_i = Re(a_i^H U a_i) over the 2-D tiles t0, t0 + dt, ... (ntiles), with
// the chunked B image Bimg (scale sB) streamed by bulk copies.  epi(i, v).
template <bool BF16, class Epi>
__device__ void wide_adjoint(const JobDev &J, WideWork &W, const unsigned char *Bimg, float sB, int t0, int dt,
                             int ntiles, float *red, Epi epi) {
    const int p = J.p, Kp = W.Kp, N = 2 * Kp, nk = N / kChunkK;
    const float sX = steer_scale(p);
    const float inv = 1.f / (sX * sB);
    const uint32_t cbytes = (uint32_t)wide_chunk_bytes(p);
    const int total = ntiles * nk;
    if (total == 0) return;
    if (threadIdx.x == 0) {
        mbar_expect_tx(&W.barB[0], cbytes);
        tma_bulk_g2s(W.B[0], Bimg, cbytes, &W.barB[0]);
    }
    for (int c = 0; c < total; ++c) {
        const int tt = c / nk, kc = c - tt * nk;
        const int t = t0 + tt * dt;
        const int bx = c & 1, bb = W.nb == 2 ? (c & 1) : 0;
        wide_wait_mma(W, bx);                       // X[bx] free: MMAs of chunk c-2 done
        wide_gen_X<BF16>(J, W, bx, t, kc, sX);
        fence_async_smem();
        if (!mbar_wait(&W.barB[bb], W.phB[bb])) W.timeouts++;   // B chunk c landed
        W.phB[bb] ^= 1u;
        __syncthreads();
        if (threadIdx.x == 0) {
            wide_issue(W, bx, bb, kc == 0, BF16 ? 1 : 0);
            mma_commit(&W.barM[bx]);
        }
        W.issued[bx]++;
        if (c + 1 < total) {
            // the next B chunk goes to a buffer no pending MMA reads
            const int nbb = W.nb == 2 ? ((c + 1) & 1) : 0;
            wide_wait_mma(W, W.nb == 2 ? ((c + 1) & 1) : bx);
            if (threadIdx.x == 0) {
                const int nkc = (c + 1) % nk;
                mbar_expect_tx(&W.barB[nbb], cbytes);
                tma_bulk_g2s(W.B[nbb], Bimg + (size_t)nkc * cbytes, cbytes, &W.barB[nbb]);
            }
        }
        if (kc == nk - 1) {
            // tile complete: its last MMAs, then the epilogue from tensor memory
            wide_wait_mma(W, bx);
            tc_fence_after();
            __syncthreads();
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            const int half = warp >> 2, r = 32 * (warp & 3) + lane;
            const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
            const int i = tc_tile_pixel(t, r, J.n_l, J.n_m);
            int mm = 0, ll = 0;
            if (i >= 0) {
                mm = i / J.n_l;
                ll = i - mm * J.n_l;
            }
            float acc = 0.f;
            for (int c0 = 0; c0 < Kp; c0 += 16) {
                float d[16];
                tmem_ld16(W.tmem + lane_base + (uint32_t)(half * Kp + c0), d);
                if (i >= 0) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int k = c0 + q;
                        if (k < p) {
                            const float2 a = cmul(__ldg(J.El + (size_t)ll * p + k), __ldg(J.Em + (size_t)mm * p + k));
                            acc = fmaf(half ? a.y : a.x, d[q], acc);
                        }
                    }
                }
            }
            red[half * kTcM + r] = acc;
            tc_fence_before();
            __syncthreads();
            if (threadIdx.x < kTcM) {
                const int ii = tc_tile_pixel(t, threadIdx.x, J.n_l, J.n_m);
                if (ii >= 0) epi(ii, (red[threadIdx.x] + red[kTcM + threadIdx.x]) * inv);
            }
            __syncthreads();
        }
    }
    wide_wait_mma(W, 0);
    wide_wait_mma(W, 1);
}

}  // namespace img
