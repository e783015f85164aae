// Tensor-core (tcgen05) form of the adjoint operator Psi^H (Sec. V-B):
//
//   out_i = Re(a_i^H U a_i) = x_i^T B x_i,   x_i = [Re a_i ; Im a_i],
//   B = [[Re U, -Im U], [Im U, Re U]]  (real embedding, 2p x 2p)
//
// For a tile of 128 pixels the product D = X B^T (M = 128 pixels, N = K = 2Kp,
// Kp = p rounded up to 32) runs as tcgen05.mma kind::f16 with FP32
// accumulation in tensor memory.  Each operand is split into two 16-bit
// parts, v = hi + lo, and D = Xhi Bhi + Xhi Blo + Xlo Bhi.  With FP16 parts
// and power-of-two scaling of X and B to unit range, the split keeps about
// 22 bits of every product, which holds the FP32 path's accuracy; BF16 parts
// keep about 16 bits.  The epilogue reads D from tensor memory
// (tcgen05.ld 32x32b: one pixel per lane) and forms the dot with x_i in FP32.
//
// Shared-memory operand layout: K-major with the 128-byte swizzle.  Rows of
// 64 16-bit elements (128 bytes) are grouped in 8-row, 1024-byte atoms; the
// 16-byte chunk c of row r sits at chunk position c ^ (r % 8).  A K extent of
// 2Kp is stored as 2Kp/64 column blocks of R rows x 128 bytes each.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cta_ops.cuh"

namespace img {

constexpr int kTcM = 128;               // pixels per tile (MMA M)
constexpr unsigned kSpinLimit = 1u << 26;   // bounded mbarrier waits

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Wait until the barrier's phase with the given parity completes.  Returns
// false after kSpinLimit polls (the caller records a timeout and goes on).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// ---------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst_smem)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Make generic-proxy shared-memory writes visible to the tensor cores.
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms
// 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: F32 accumulate, A/B format (0 F16,
// 1 BF16), both K-major, M = 128, N.
__host__ __device__ constexpr uint32_t idesc_f16(int n, int ab_fmt) {
    return (1u << 4) | ((uint32_t)ab_fmt << 7) | ((uint32_t)ab_fmt << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accum) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 16 consecutive FP32 columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- splitting
// v = hi + lo in 16-bit parts; the 8 values of a 16-byte chunk at once.
template <bool BF16>
__device__ __forceinline__ void split8(const float *v, uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (BF16) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * q]);
            const __nv_bfloat16 h1 = __float2bfloat16_rn(v[2 * q + 1]);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * q] - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * q + 1] - __bfloat162float(h1));
            h[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            l[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
        } else {
            const __half h0 = __float2half_rn(v[2 * q]);
            const __half h1 = __float2half_rn(v[2 * q + 1]);
            const __half l0 = __float2half_rn(v[2 * q] - __half2float(h0));
            const __half l1 = __float2half_rn(v[2 * q + 1] - __half2float(h1));
            h[q] = (uint32_t)__half_as_ushort(h0) | ((uint32_t)__half_as_ushort(h1) << 16);
            l[q] = (uint32_t)__half_as_ushort(l0) | ((uint32_t)__half_as_ushort(l1) << 16);
        }
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// Byte offset of 16-byte chunk c (8 elements, covering K = 8c .. 8c+7) of
// row r in a swizzled K-major tile with R rows.
__device__ __forceinline__ uint32_t sw128_off(int r, int c, int R) {
    const int kb = c >> 3, cc = c & 7;
    return (uint32_t)(kb * R * 128 + (r >> 3) * 1024 + (r & 7) * 128 + ((cc ^ (r & 7)) << 4));
}

// Tensor-core workspace of one CTA.
struct TcWork {
    unsigned char *Xhi, *Xlo, *Bhi, *Blo;  // 1024-aligned operand tiles
    uint64_t *bar;                          // MMA completion barrier
    uint32_t tmem;                          // accumulator base (lane 0, column 0)
    uint32_t phase;                         // parity of the next completion
    int Kp;                                 // p rounded up to 32
    int timeouts;                           // bounded waits that ran out
};

// Bytes of shared memory the operand tiles need for p (plus 1024 alignment).
__host__ __device__ inline size_t tc_smem_bytes(int p) {
    const int Kp = (p + 31) / 32 * 32;
    const size_t x = (size_t)kTcM * 2 * Kp * 2;      // one 16-bit tile of X
    const size_t b = (size_t)2 * Kp * 2 * Kp * 2;    // one 16-bit tile of B
    return 2 * x + 2 * b + 1024;
}
__host__ __device__ inline uint32_t tc_tmem_cols(int p) {
    const int n = 2 * ((p + 31) / 32 * 32);
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

// Carve the operand tiles from a 1024-aligned shared-memory region.
__device__ inline void tc_carve(TcWork &T, unsigned char *base, int p) {
    T.Kp = (p + 31) / 32 * 32;
    const size_t x = (size_t)kTcM * 2 * T.Kp * 2;
    const size_t b = (size_t)2 * T.Kp * 2 * T.Kp * 2;
    T.Xhi = base;
    T.Xlo = base + x;
    T.Bhi = base + 2 * x;
    T.Blo = base + 2 * x + b;
}

// B = real embedding of U, scaled by a power of two to max |entry| <= 1,
// split into hi/lo 16-bit tiles.  Row n of B^T (N index) holds, for
// n < p: [Re U(n,:), -Im U(n,:)], for Kp <= n < Kp+p: [Im U(n,:), Re U(n,:)].
// Re(a^H U a) = Re(a^H U^H a), so rows are read from columns of U (contiguous)
// as conj(U(:, n)).  Returns the scale.
template <bool BF16>
__device__ float tc_build_B(const float2 *U, int p, TcWork &T, double *sbuf) {
    const int Kp = T.Kp, N = 2 * Kp;
    float mx = 0.f;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const float2 u = U[e];
        mx = fmaxf(mx, fmaxf(fabsf(u.x), fabsf(u.y)));
    }
    // max over the CTA
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) mx = fmaxf(mx, (float)sbuf[w]);
    __syncthreads();
    const float sc = mx > 0.f ? exp2f(-ceilf(log2f(mx))) : 1.f;
    const int cpr = N / 8;                   // 16-byte chunks per row
    for (int it = threadIdx.x; it < N * cpr; it += blockDim.x) {
        const int n = it / cpr, c = it - n * cpr;
        const int k0 = c * 8;                // K index of the chunk
        float v[8];
        const bool nre = n < Kp;
        const int row = nre ? n : n - Kp;    // row of U
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = k0 + q;
            const bool kre = k < Kp;
            const int col = kre ? k : k - Kp;
            float val = 0.f;
            if (row < p && col < p) {
                const float2 u = U[(size_t)row * p + col];   // U(col,row) = conj(U(row,col))
                // B^T[n][k]: (re,re) Re U, (re,im) -Im U, (im,re) Im U, (im,im) Re U
                // with U(row,col) = conj(u): Re U = u.x, Im U = -u.y
                if (nre && kre) val = u.x;
                else if (nre && !kre) val = u.y;
                else if (!nre && kre) val = -u.y;
                else val = u.x;
            }
            v[q] = val * sc;
        }
        uint4 hi, lo;
        split8<BF16>(v, hi, lo);
        const uint32_t off = sw128_off(n, c, N);
        *reinterpret_cast<uint4 *>(T.Bhi + off) = hi;
        *reinterpret_cast<uint4 *>(T.Blo + off) = lo;
    }
    return sc;
}

// Issue the 3-product MMA chain for the current X/B tiles and wait for it.
// Call with all threads after the operand writes (this function fences,
// synchronises and waits).  Returns false if the wait ran out.
__device__ inline bool tc_mma_tile(TcWork &T, uint32_t idesc) {
    fence_async_smem();
    __syncthreads();
    const int Kp = T.Kp, N = 2 * Kp, nks = (2 * Kp) / 16;
    if (threadIdx.x == 0) {
        tc_fence_after();
        const uint32_t xh = smem_u32(T.Xhi), xl = smem_u32(T.Xlo);
        const uint32_t bh = smem_u32(T.Bhi), bl = smem_u32(T.Blo);
        for (int s = 0; s < nks; ++s) {
            const uint32_t kb = s >> 2, off = (s & 3) * 32;
            const uint32_t xo = kb * kTcM * 128 + off, bo = kb * N * 128 + off;
            mma_f16(T.tmem, sw128_desc(xh + xo), sw128_desc(bh + bo), idesc, s > 0 ? 1u : 0u);
            mma_f16(T.tmem, sw128_desc(xh + xo), sw128_desc(bl + bo), idesc, 1u);
            mma_f16(T.tmem, sw128_desc(xl + xo), sw128_desc(bh + bo), idesc, 1u);
        }
        mma_commit(T.bar);
    }
    const bool ok = mbar_wait(T.bar, T.phase);
    T.phase ^= 1u;
    tc_fence_after();
    if (!ok) T.timeouts++;
    return ok;
}

// Epilogue of one tile: this thread's lane (pixel row r) and half (real or
// imaginary columns) dotted with xh[0..Kp) (the thread's own x half, FP32,
// zero beyond p).  Returns the partial sum; the caller adds both halves.
__device__ inline float tc_dot_half(const TcWork &T, const float *xhalf) {
    const int warp = threadIdx.x >> 5;
    const int half = warp >> 2;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    float acc = 0.f;
    for (int c0 = 0; c0 < T.Kp; c0 += 16) {
        float d[16];
        tmem_ld16(T.tmem + lane_base + (uint32_t)(half * T.Kp + c0), d);
#pragma unroll
        for (int q = 0; q < 16; ++q) acc = fmaf(xhalf[c0 + q], d[q], acc);
    }
    return acc;
}

}  // namespace img

namespace img {

// X tile (128 rows) from steering vectors of pixels pix0 .. pix0+np-1; rows
// beyond np are zero.  Values scaled by sX (a power of two).
template <bool BF16>
__device__ inline void tc_gen_X_steer(const JobDev &J, TcWork &T, int pix0, int np, float sX) {
    const int p = J.p, Kp = T.Kp, nc8 = Kp / 8;
    for (int it = threadIdx.x; it < kTcM * nc8; it += blockDim.x) {
        const int r = it / nc8, c8 = it - r * nc8;
        float re[8], im[8];
        if (r < np) {
            const int i = pix0 + r;
            const int mm = i / J.n_l, ll = i - mm * J.n_l;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int k = c8 * 8 + q;
                float2 a = make_float2(0.f, 0.f);
                if (k < p) a = steer(J, ll, mm, k);
                re[q] = a.x * sX;
                im[q] = a.y * sX;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) re[q] = im[q] = 0.f;
        }
        uint4 hi, lo;
        split8<BF16>(re, hi, lo);
        uint32_t off = sw128_off(r, c8, kTcM);
        *reinterpret_cast<uint4 *>(T.Xhi + off) = hi;
        *reinterpret_cast<uint4 *>(T.Xlo + off) = lo;
        split8<BF16>(im, hi, lo);
        off = sw128_off(r, nc8 + c8, kTcM);
        *reinterpret_cast<uint4 *>(T.Xhi + off) = hi;
        *reinterpret_cast<uint4 *>(T.Xlo + off) = lo;
    }
}

// X tile from cached vectors cvec[pos[j0 + r]] (pos == nullptr: j0 + r),
// scaled by a power of two to max |entry| <= 1.  Returns the scale.
template <bool BF16>
__device__ inline float tc_gen_X_cache(const JobDev &J, TcWork &T, const int *pos, int j0, int np,
                                       double *sbuf) {
    const int p = J.p, Kp = T.Kp, nc8 = Kp / 8;
    float mx = 0.f;
    for (int e = threadIdx.x; e < np * p; e += blockDim.x) {
        const int r = e / p, k = e - r * p;
        const int sl = pos ? pos[j0 + r] : j0 + r;
        const float2 c = J.cvec[(size_t)sl * p + k];
        mx = fmaxf(mx, fmaxf(fabsf(c.x), fabsf(c.y)));
    }
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) mx = fmaxf(mx, (float)sbuf[w]);
    __syncthreads();
    const float sX = mx > 0.f ? exp2f(-ceilf(log2f(mx))) : 1.f;
    for (int it = threadIdx.x; it < kTcM * nc8; it += blockDim.x) {
        const int r = it / nc8, c8 = it - r * nc8;
        float re[8], im[8];
        const int sl = r < np ? (pos ? pos[j0 + r] : j0 + r) : -1;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = c8 * 8 + q;
            float2 c = make_float2(0.f, 0.f);
            if (sl >= 0 && k < p) c = J.cvec[(size_t)sl * p + k];
            re[q] = c.x * sX;
            im[q] = c.y * sX;
        }
        uint4 hi, lo;
        split8<BF16>(re, hi, lo);
        uint32_t off = sw128_off(r, c8, kTcM);
        *reinterpret_cast<uint4 *>(T.Xhi + off) = hi;
        *reinterpret_cast<uint4 *>(T.Xlo + off) = lo;
        split8<BF16>(im, hi, lo);
        off = sw128_off(r, nc8 + c8, kTcM);
        *reinterpret_cast<uint4 *>(T.Xhi + off) = hi;
        *reinterpret_cast<uint4 *>(T.Xlo + off) = lo;
    }
    return sX;
}

// Epilogue dot for a steering tile: thread's pixel row and half; red[256]
// receives partial sums, red[r] (r < 128) the tile's outputs after the call
// (unscaled by 1/(sX sB): the caller applies it).
__device__ inline void tc_epilogue_steer(const JobDev &J, const TcWork &T, int pix0, int np,
                                         float *red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = warp >> 2, r = 32 * (warp & 3) + lane;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const int p = J.p;
    int ll = 0, mm = 0;
    if (r < np) {
        const int i = pix0 + r;
        mm = i / J.n_l;
        ll = i - mm * J.n_l;
    }
    float acc = 0.f;
    for (int c0 = 0; c0 < T.Kp; c0 += 16) {
        float d[16];
        tmem_ld16(T.tmem + lane_base + (uint32_t)(half * T.Kp + c0), d);
        if (r < np) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int k = c0 + q;
                if (k < p) {
                    const float2 a = steer(J, ll, mm, k);
                    acc = fmaf(half ? a.y : a.x, d[q], acc);
                }
            }
        }
    }
    red[half * kTcM + r] = acc;
    __syncthreads();
    if (threadIdx.x < kTcM) red[threadIdx.x] = red[threadIdx.x] + red[kTcM + threadIdx.x];
    tc_fence_before();
    __syncthreads();
}

// Epilogue dot for a cached-vector tile.
__device__ inline void tc_epilogue_cache(const JobDev &J, const TcWork &T, const int *pos, int j0,
                                         int np, float *red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = warp >> 2, r = 32 * (warp & 3) + lane;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const int p = J.p;
    const int sl = r < np ? (pos ? pos[j0 + r] : j0 + r) : -1;
    float acc = 0.f;
    for (int c0 = 0; c0 < T.Kp; c0 += 16) {
        float d[16];
        tmem_ld16(T.tmem + lane_base + (uint32_t)(half * T.Kp + c0), d);
        if (sl >= 0) {
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int k = c0 + q;
                if (k < p) {
                    const float2 c = J.cvec[(size_t)sl * p + k];
                    acc = fmaf(half ? c.y : c.x, d[q], acc);
                }
            }
        }
    }
    red[half * kTcM + r] = acc;
    __syncthreads();
    if (threadIdx.x < kTcM) red[threadIdx.x] = red[threadIdx.x] + red[kTcM + threadIdx.x];
    tc_fence_before();
    __syncthreads();
}

__device__ __forceinline__ float steer_scale(int p) { return exp2f(floorf(0.5f * log2f((float)p))); }

}  // namespace img
