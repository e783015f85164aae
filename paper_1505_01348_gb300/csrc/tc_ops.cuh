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
// false after `limit` polls (kSpinLimit by default; the caller records a
// timeout and goes on).
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned limit = kSpinLimit) {
    const uint32_t a = smem_u32(bar);
    for (unsigned it = 0; it < limit; ++it) {
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

// Two 16-column tensor-memory loads, one wait.
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float *a, float *b) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%32];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, "
        "[%33];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
          "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
          "=r"(r[30]), "=r"(r[31])
        : "r"(ta), "r"(tb)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        a[i] = __uint_as_float(r[i]);
        b[i] = __uint_as_float(r[16 + i]);
    }
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

// Two values -> hi and lo 16-bit pairs (packed conversions, round to nearest).
template <bool BF16>
__device__ __forceinline__ void split2(float v0, float v1, uint32_t &hi, uint32_t &lo) {
    if (BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    } else {
        const __half2 h = __floats2half2_rn(v0, v1);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(v0 - hf.x, v1 - hf.y);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
}

// Byte offset of 16-byte chunk c (8 elements, covering K = 8c .. 8c+7) of
// row r in a swizzled K-major tile with R rows.
__device__ __forceinline__ uint32_t sw128_off(int r, int c, int R) {
    const int kb = c >> 3, cc = c & 7;
    return (uint32_t)(kb * R * 128 + (r >> 3) * 1024 + (r & 7) * 128 + ((cc ^ (r & 7)) << 4));
}

// Tensor-core workspace of one CTA: two X tiles and two accumulators so that
// generating tile t+1 and the epilogue of tile t overlap the MMAs.
struct TcWork {
    unsigned char *Xhi[2], *Xlo[2];  // 1024-aligned operand tiles (pixels x 2Kp)
    unsigned char *Bhi, *Blo;        // (2Kp x 2Kp)
    uint64_t *bar;                   // two MMA completion barriers
    uint32_t tmem;                   // accumulator base (lane 0, column 0)
    uint32_t phase[2];               // parity of each barrier's next completion
    float sX[2];                     // scale of the X tile in each buffer
    int Kp;                          // p rounded up to 32
    int timeouts;                    // bounded waits that ran out
};

// Bytes of shared memory the operand tiles need for p (plus 1024 alignment).
__host__ __device__ inline size_t tc_smem_bytes(int p) {
    const int Kp = (p + 31) / 32 * 32;
    const size_t x = (size_t)kTcM * 2 * Kp * 2;      // one 16-bit tile of X
    const size_t b = (size_t)2 * Kp * 2 * Kp * 2;    // one 16-bit tile of B
    return 4 * x + 2 * b + 1024;
}
// Tensor-memory columns: three FP32 accumulators of 2Kp columns each (two
// for the adjoint pipeline, one for the forward product).
__host__ __device__ inline uint32_t tc_tmem_cols(int p) {
    const int n = 6 * ((p + 31) / 32 * 32);
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

// Carve the operand tiles from a 1024-aligned shared-memory region.
__device__ inline void tc_carve(TcWork &T, unsigned char *base, int p) {
    T.Kp = (p + 31) / 32 * 32;
    const size_t x = (size_t)kTcM * 2 * T.Kp * 2;
    const size_t b = (size_t)2 * T.Kp * 2 * T.Kp * 2;
    T.Xhi[0] = base;
    T.Xlo[0] = base + x;
    T.Xhi[1] = base + 2 * x;
    T.Xlo[1] = base + 3 * x;
    T.Bhi = base + 4 * x;
    T.Blo = base + 4 * x + b;
    T.phase[0] = T.phase[1] = 0;
    T.timeouts = 0;
}

// Set up barriers and tensor memory (all threads; warp 0 allocates).
__device__ inline void tc_setup(TcWork &T, uint64_t *bars, uint32_t *slot, int p) {
    T.bar = bars;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
    }
    if (threadIdx.x < 32) tmem_alloc(slot, tc_tmem_cols(p));
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    T.tmem = *slot;
}

__device__ inline void tc_teardown(TcWork &T, int p) {
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(T.tmem, tc_tmem_cols(p));
}

// Operand scale lift.  FP16 holds full precision only in its normal range
// [2^-14, 2^15]; the lo part of a split value is about 2^-11 of the value, so
// with operands scaled to a maximum near 1 the lo part of every value below
// 1/8 of the maximum would be subnormal and lose bits.  Operands are scaled
// to a maximum near 2^13 instead: lo parts stay normal for values down to
// about 2^-16 of the maximum.  Products stay below 2^28 and accumulated
// sums far below the FP32 range.  (BF16 parts have the FP32 exponent range;
// the lift is harmless there.)
constexpr float kLift = 8192.f;

// B = real embedding of U, scaled by a power of two to max |entry| <= 1,
// lifted by kLift and split into hi/lo 16-bit tiles.  Row n of B^T (N index) holds, for
// n < p: [Re V(n,:), -Im V(n,:)], for Kp <= n < Kp+p: [Im V(n,:), Re V(n,:)]
// with V = U^H; Re(a^H U a) = Re(a^H U^H a), and row n of V is the conjugate
// of column n of U, which is contiguous.  One pass: each thread keeps its
// column chunks of U in registers while the CTA finds the scale.
template <bool BF16>
__device__ float tc_build_B(const float2 *U, int p, TcWork &T, double *sbuf) {
    const int Kp = T.Kp, N = 2 * Kp, nc8 = Kp / 8;
    constexpr int kMaxItems = 4;          // (Kp/8) * Kp / kThreads <= 4 for Kp <= 128
    const int items = Kp * nc8;           // (row n < Kp, chunk of 8 columns)
    float2 v[kMaxItems][8];
    float mx = 0.f;
#pragma unroll
    for (int q = 0; q < kMaxItems; ++q) {
        const int it = threadIdx.x + q * kThreads;
        const int n = it / nc8, c8 = it - n * nc8;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[q][e] = make_float2(0.f, 0.f);
        if (it < items && n < p) {
            const int k0 = c8 * 8;
            const float2 *src = U + (size_t)n * p + k0;      // U(k0.., n) = conj(V(n, k0..))
            if ((p & 1) == 0 && k0 + 8 <= p) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float4 x = reinterpret_cast<const float4 *>(src)[e];
                    v[q][2 * e] = make_float2(x.x, x.y);
                    v[q][2 * e + 1] = make_float2(x.z, x.w);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (k0 + e < p) v[q][e] = src[e];
            }
#pragma unroll
            for (int e = 0; e < 8; ++e) mx = fmaxf(mx, fmaxf(fabsf(v[q][e].x), fabsf(v[q][e].y)));
        }
    }
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) mx = fmaxf(mx, (float)sbuf[w]);
    __syncthreads();
    const float sc = (mx > 0.f ? exp2f(-ceilf(log2f(mx))) : 1.f) * kLift;
#pragma unroll
    for (int q = 0; q < kMaxItems; ++q) {
        const int it = threadIdx.x + q * kThreads;
        if (it >= items) break;
        const int n = it / nc8, c8 = it - n * nc8;
        // u = U(k, n) = conj(V(n, k)):  Re V = u.x, Im V = -u.y
        float re[8], nim[8], im[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            re[e] = v[q][e].x * sc;
            im[e] = -v[q][e].y * sc;
            nim[e] = v[q][e].y * sc;
        }
        uint4 hi, lo;
        split8<BF16>(re, hi, lo);                       // (re row, re col): Re V
        uint32_t off = sw128_off(n, c8, N);
        *reinterpret_cast<uint4 *>(T.Bhi + off) = hi;
        *reinterpret_cast<uint4 *>(T.Blo + off) = lo;
        off = sw128_off(Kp + n, nc8 + c8, N);           // (im row, im col): Re V
        *reinterpret_cast<uint4 *>(T.Bhi + off) = hi;
        *reinterpret_cast<uint4 *>(T.Blo + off) = lo;
        split8<BF16>(nim, hi, lo);                      // (re row, im col): -Im V
        off = sw128_off(n, nc8 + c8, N);
        *reinterpret_cast<uint4 *>(T.Bhi + off) = hi;
        *reinterpret_cast<uint4 *>(T.Blo + off) = lo;
        split8<BF16>(im, hi, lo);                       // (im row, re col): Im V
        off = sw128_off(Kp + n, c8, N);
        *reinterpret_cast<uint4 *>(T.Bhi + off) = hi;
        *reinterpret_cast<uint4 *>(T.Blo + off) = lo;
    }
    return sc;
}

// Issue the 3-product MMA chain for X[b] against B into accumulator b and
// commit it to barrier b (one thread).
__device__ inline void tc_issue(const TcWork &T, int b, uint32_t idesc) {
    const int Kp = T.Kp, N = 2 * Kp, nks = (2 * Kp) / 16;
    tc_fence_after();
    const uint32_t xh = smem_u32(T.Xhi[b]), xl = smem_u32(T.Xlo[b]);
    const uint32_t bh = smem_u32(T.Bhi), bl = smem_u32(T.Blo);
    const uint32_t d = T.tmem + (uint32_t)(b * N);
    for (int s = 0; s < nks; ++s) {
        const uint32_t kb = s >> 2, off = (s & 3) * 32;
        const uint32_t xo = kb * kTcM * 128 + off, bo = kb * N * 128 + off;
        mma_f16(d, sw128_desc(xh + xo), sw128_desc(bh + bo), idesc, s > 0 ? 1u : 0u);
        mma_f16(d, sw128_desc(xh + xo), sw128_desc(bl + bo), idesc, 1u);
        mma_f16(d, sw128_desc(xl + xo), sw128_desc(bh + bo), idesc, 1u);
    }
    mma_commit(&T.bar[b]);
}

// Software pipeline over tiles: gen(t, b) fills X[b] (and T.sX[b]) for tile
// t, epi(t, b) consumes accumulator b.  Generating tile t+1 and the epilogue
// of tile t run while the tensor cores work on the other buffer.  The B tile
// must be in place before the call.  All threads call this.
// pre(t) runs before tile t + 1 is generated, so loads that the epilogue of
// tile t needs are in flight during the generation and the MMA.
template <class Gen, class Epi, class Pre>
__device__ inline void tc_run_tiles(TcWork &T, int ntiles, uint32_t idesc, Gen gen, Epi epi, Pre pre) {
    if (ntiles <= 0) return;
    gen(0, 0);
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) tc_issue(T, 0, idesc);
    for (int t = 0; t < ntiles; ++t) {
        const int b = t & 1;
        pre(t);
        if (t + 1 < ntiles) gen(t + 1, b ^ 1);
        fence_async_smem();
        if (!mbar_wait(&T.bar[b], T.phase[b])) T.timeouts++;
        T.phase[b] ^= 1u;
        tc_fence_after();
        __syncthreads();
        if (t + 1 < ntiles && threadIdx.x == 0) tc_issue(T, b ^ 1, idesc);
        epi(t, b);
    }
}

template <class Gen, class Epi>
__device__ inline void tc_run_tiles(TcWork &T, int ntiles, uint32_t idesc, Gen gen, Epi epi) {
    tc_run_tiles(T, ntiles, idesc, gen, epi, [](int) {});
}


}  // namespace img

namespace img {

// X tile (128 rows) from steering vectors of pixels pix0 .. pix0+np-1; rows
// beyond np are zero.  Values scaled by sX (a power of two).
// Pixel tiles are 8 (l) x 16 (m) blocks of the grid, so one tile reads only
// 8 + 16 rows of the separable steering tables (L1-resident) instead of 128.
constexpr int kTileL = 8, kTileM = 16;

__host__ __device__ inline int tc_num_tiles(int n_l, int n_m) {
    return ((n_l + kTileL - 1) / kTileL) * ((n_m + kTileM - 1) / kTileM);
}

// Pixel index of row r of 2-D tile t, or -1 outside the grid.
__device__ __forceinline__ int tc_tile_pixel(int t, int r, int n_l, int n_m) {
    const int tl = (n_l + kTileL - 1) / kTileL;
    const int bm = t / tl, bl = t - bm * tl;
    const int il = bl * kTileL + (r % kTileL), im = bm * kTileM + r / kTileL;
    return (il < n_l && im < n_m) ? il + n_l * im : -1;
}

// X tile (128 rows) of steering vectors for the pixels of 2-D tile t
// (rows outside the grid are zero), scaled by sX (a power of two).
template <bool BF16>
__device__ inline void tc_gen_X_steer(const JobDev &J, TcWork &T, int b, int t, float sX) {
    const int p = J.p, Kp = T.Kp, nc8 = Kp / 8, nl = J.n_l;
    const float2 *__restrict__ El = J.El;
    const float2 *__restrict__ Em = J.Em;
    unsigned char *xh = T.Xhi[b], *xl = T.Xlo[b];
    const bool vec = (p & 7) == 0;       // 64-byte aligned antenna chunks
    for (int it = threadIdx.x; it < kTcM * nc8; it += blockDim.x) {
        const int r = it / nc8, c8 = it - r * nc8;
        float re[8], im[8];
        const int k0 = c8 * 8;
        const int i = tc_tile_pixel(t, r, nl, J.n_m);
        if (i >= 0 && k0 < p) {
            const int mm = i / nl, ll = i - mm * nl;
            if (vec) {
                const float4 *e = reinterpret_cast<const float4 *>(El + (size_t)ll * p + k0);
                const float4 *f = reinterpret_cast<const float4 *>(Em + (size_t)mm * p + k0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 x = __ldg(e + q), y = __ldg(f + q);
                    const float2 a0 = cmul(make_float2(x.x, x.y), make_float2(y.x, y.y));
                    const float2 a1 = cmul(make_float2(x.z, x.w), make_float2(y.z, y.w));
                    re[2 * q] = a0.x * sX;
                    im[2 * q] = a0.y * sX;
                    re[2 * q + 1] = a1.x * sX;
                    im[2 * q + 1] = a1.y * sX;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = k0 + q;
                    float2 a = make_float2(0.f, 0.f);
                    if (k < p) a = cmul(__ldg(El + (size_t)ll * p + k), __ldg(Em + (size_t)mm * p + k));
                    re[q] = a.x * sX;
                    im[q] = a.y * sX;
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) re[q] = im[q] = 0.f;
        }
        uint4 hi, lo;
        split8<BF16>(re, hi, lo);
        uint32_t off = sw128_off(r, c8, kTcM);
        *reinterpret_cast<uint4 *>(xh + off) = hi;
        *reinterpret_cast<uint4 *>(xl + off) = lo;
        split8<BF16>(im, hi, lo);
        off = sw128_off(r, nc8 + c8, kTcM);
        *reinterpret_cast<uint4 *>(xh + off) = hi;
        *reinterpret_cast<uint4 *>(xl + off) = lo;
    }
}

// X tile of the consecutive pixels pix0 .. pix0+np-1 (forward over all
// pixels, where every pixel's weight comes from a linear array).
template <bool BF16>
__device__ inline void tc_gen_X_range(const JobDev &J, TcWork &T, int b, int pix0, int np, float sX) {
    const int p = J.p, Kp = T.Kp, nc8 = Kp / 8, nl = J.n_l;
    unsigned char *xh = T.Xhi[b], *xl = T.Xlo[b];
    for (int it = threadIdx.x; it < kTcM * nc8; it += blockDim.x) {
        const int r = it / nc8, c8 = it - r * nc8;
        float re[8], im[8];
        const int i = pix0 + r;
        const int mm = i / nl, ll = i - mm * nl;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = c8 * 8 + q;
            float2 a = make_float2(0.f, 0.f);
            if (r < np && k < p) a = steer(J, ll, mm, k);
            re[q] = a.x * sX;
            im[q] = a.y * sX;
        }
        uint4 hi, lo;
        split8<BF16>(re, hi, lo);
        uint32_t off = sw128_off(r, c8, kTcM);
        *reinterpret_cast<uint4 *>(xh + off) = hi;
        *reinterpret_cast<uint4 *>(xl + off) = lo;
        split8<BF16>(im, hi, lo);
        off = sw128_off(r, nc8 + c8, kTcM);
        *reinterpret_cast<uint4 *>(xh + off) = hi;
        *reinterpret_cast<uint4 *>(xl + off) = lo;
    }
}

// X tile from cached vectors cvec[pos[j0 + r]] (pos == nullptr: j0 + r),
// scaled by sX (a power of two keeping every entry within unit range).
template <bool BF16>
__device__ inline void tc_gen_X_cache(const JobDev &J, TcWork &T, int b, const int *pos, int j0, int np,
                                      float sX) {
    const int p = J.p, Kp = T.Kp, nc8 = Kp / 8;
    unsigned char *xh = T.Xhi[b], *xl = T.Xlo[b];
    const bool vec = (p & 7) == 0;
    for (int it = threadIdx.x; it < kTcM * nc8; it += blockDim.x) {
        const int r = it / nc8, c8 = it - r * nc8;
        float re[8], im[8];
        const int k0 = c8 * 8;
        const int sl = r < np ? (pos ? pos[j0 + r] : j0 + r) : -1;
        if (sl >= 0 && k0 < p) {
            const float2 *c = J.cvec + (size_t)sl * p + k0;
            if (vec) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 x = reinterpret_cast<const float4 *>(c)[q];
                    re[2 * q] = x.x * sX;
                    im[2 * q] = x.y * sX;
                    re[2 * q + 1] = x.z * sX;
                    im[2 * q + 1] = x.w * sX;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float2 x = (k0 + q < p) ? c[q] : make_float2(0.f, 0.f);
                    re[q] = x.x * sX;
                    im[q] = x.y * sX;
                }
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) re[q] = im[q] = 0.f;
        }
        uint4 hi, lo;
        split8<BF16>(re, hi, lo);
        uint32_t off = sw128_off(r, c8, kTcM);
        *reinterpret_cast<uint4 *>(xh + off) = hi;
        *reinterpret_cast<uint4 *>(xl + off) = lo;
        split8<BF16>(im, hi, lo);
        off = sw128_off(r, nc8 + c8, kTcM);
        *reinterpret_cast<uint4 *>(xh + off) = hi;
        *reinterpret_cast<uint4 *>(xl + off) = lo;
    }
}

// Epilogue of one tile: thread (row r = pixel, half h = real / imaginary
// columns) forms sum_k xs_k D[r][h Kp + k], with xs = hi + lo rebuilt from the
// operand tile in shared memory (the scaled x the MMA consumed; conflict-free
// 16-byte reads).  red[r] (r < 128) holds the tile's sums after the call; the
// caller multiplies by 1/(sX^2 sB).  SQ: the sum of squares of the row's
// accumulator, ||D[r]||^2 (B built from V = L^-1: the whitened MVDR
// denominator); the caller multiplies by 1/(sX sB)^2.
template <bool BF16, bool SQ = false>
__device__ inline void tc_epilogue(const TcWork &T, int b, float *red) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = warp >> 2, r = 32 * (warp & 3) + lane;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    const int nc8 = T.Kp / 8;
    float acc = 0.f;
    for (int c00 = 0; c00 < T.Kp; c00 += 32) {
        float dd[2][16];
        const uint32_t ta = T.tmem + lane_base + (uint32_t)(b * 2 * T.Kp + half * T.Kp + c00);
        tmem_ld16x2(ta, ta + 16, dd[0], dd[1]);
        if (SQ) {
#pragma unroll
            for (int g = 0; g < 2; ++g)
#pragma unroll
                for (int q = 0; q < 16; ++q) acc = fmaf(dd[g][q], dd[g][q], acc);
        } else {
#pragma unroll
            for (int g = 0; g < 2; ++g) {
            const int c0 = c00 + 16 * g;
            const float *d = dd[g];
#pragma unroll
            for (int s8 = 0; s8 < 2; ++s8) {
                const uint32_t off = sw128_off(r, half * nc8 + c0 / 8 + s8, kTcM);
                const uint4 h4 = *reinterpret_cast<const uint4 *>(T.Xhi[b] + off);
                const uint4 l4 = *reinterpret_cast<const uint4 *>(T.Xlo[b] + off);
                const uint32_t hw[4] = {h4.x, h4.y, h4.z, h4.w}, lw[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float h0, h1, l0, l1;
                    if (BF16) {
                        h0 = __uint_as_float(hw[q] << 16);
                        h1 = __uint_as_float(hw[q] & 0xffff0000u);
                        l0 = __uint_as_float(lw[q] << 16);
                        l1 = __uint_as_float(lw[q] & 0xffff0000u);
                    } else {
                        h0 = __half2float(__ushort_as_half((unsigned short)(hw[q] & 0xffffu)));
                        h1 = __half2float(__ushort_as_half((unsigned short)(hw[q] >> 16)));
                        l0 = __half2float(__ushort_as_half((unsigned short)(lw[q] & 0xffffu)));
                        l1 = __half2float(__ushort_as_half((unsigned short)(lw[q] >> 16)));
                    }
                    acc = fmaf(h0 + l0, d[s8 * 8 + 2 * q], acc);
                    acc = fmaf(h1 + l1, d[s8 * 8 + 2 * q + 1], acc);
                }
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
// Scale of the steering tiles of the one-CTA tensor-core paths (p <= 64):
// unit range, lifted as above.
__device__ __forceinline__ float tc_steer_scale(int p) { return steer_scale(p) * kLift; }

}  // namespace img

namespace img {

// ---------------------------------------------------------------- forward
// Forward operator on tensor cores: G = sum_j w_j x_j x_j^T (2Kp x 2Kp real),
// from which K = sum_j w_j c_j c_j^H follows as
//   Re K(a,b) = G(a,b) + G(Kp+a, Kp+b),  Im K(a,b) = G(Kp+a, b) - G(a, Kp+b).
// The contraction runs over pixels, so the pixel-major X tiles of the adjoint
// serve directly as MN-major operands: A = X_w^T (rows scaled by w_j), B = X^T.
// In the MN-major 128-byte-swizzled reading of those tiles, 64 consecutive
// MN elements form one 128-byte row, 8 rows (8 pixels, the K direction) form
// a 1024-byte atom (SBO = 1024), and the next 64 MN elements sit one column
// block further (LBO = 128 rows x 128 bytes).

__device__ __forceinline__ uint64_t sw128_desc_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// kind::f16 instruction descriptor with both operands MN-major, M = N = n.
__host__ __device__ constexpr uint32_t idesc_f16_mn(int n, int ab_fmt) {
    return (1u << 4) | ((uint32_t)ab_fmt << 7) | ((uint32_t)ab_fmt << 10) | (1u << 15) | (1u << 16) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(n >> 4) << 24);
}

// Weighted copy of the pixel-major tile in buffer 0 into buffer 1:
// Xw[j][.] = sW * w_j * X[j][.], re-split into hi/lo (rows j >= np are zero).
template <bool BF16>
__device__ inline void tc_weight_rows(TcWork &T, const float *w, int np, float sW) {
    const int nch = 2 * T.Kp / 8;
    for (int it = threadIdx.x; it < kTcM * nch; it += blockDim.x) {
        const int r = it / nch, c = it - r * nch;
        const uint32_t off = sw128_off(r, c, kTcM);
        const uint4 h4 = *reinterpret_cast<const uint4 *>(T.Xhi[0] + off);
        const uint4 l4 = *reinterpret_cast<const uint4 *>(T.Xlo[0] + off);
        const uint32_t hw[4] = {h4.x, h4.y, h4.z, h4.w}, lw[4] = {l4.x, l4.y, l4.z, l4.w};
        const float wr = r < np ? sW * w[r] : 0.f;
        float v[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float h0, h1, l0, l1;
            if (BF16) {
                h0 = __uint_as_float(hw[q] << 16);
                h1 = __uint_as_float(hw[q] & 0xffff0000u);
                l0 = __uint_as_float(lw[q] << 16);
                l1 = __uint_as_float(lw[q] & 0xffff0000u);
            } else {
                h0 = __half2float(__ushort_as_half((unsigned short)(hw[q] & 0xffffu)));
                h1 = __half2float(__ushort_as_half((unsigned short)(hw[q] >> 16)));
                l0 = __half2float(__ushort_as_half((unsigned short)(lw[q] & 0xffffu)));
                l1 = __half2float(__ushort_as_half((unsigned short)(lw[q] >> 16)));
            }
            v[2 * q] = wr * (h0 + l0);
            v[2 * q + 1] = wr * (h1 + l1);
        }
        uint4 hi, lo;
        split8<BF16>(v, hi, lo);
        *reinterpret_cast<uint4 *>(T.Xhi[1] + off) = hi;
        *reinterpret_cast<uint4 *>(T.Xlo[1] + off) = lo;
    }
}

// Accumulate X_w^T X of the current tile pair (buffers 1 and 0) into the
// forward accumulator (tensor-memory columns 4Kp .. 6Kp).  One thread.
__device__ inline void tc_issue_fwd(const TcWork &T, uint32_t idesc, bool first) {
    const int N = 2 * T.Kp;
    tc_fence_after();
    const uint32_t ah = smem_u32(T.Xhi[1]), al = smem_u32(T.Xlo[1]);
    const uint32_t bh = smem_u32(T.Xhi[0]), bl = smem_u32(T.Xlo[0]);
    const uint32_t d = T.tmem + (uint32_t)(2 * N);
    const uint32_t lbo = kTcM * 128, sbo = 1024;
    for (int s = 0; s < kTcM / 16; ++s) {
        const uint32_t o = s * 2048;
        mma_f16(d, sw128_desc_mn(ah + o, lbo, sbo), sw128_desc_mn(bh + o, lbo, sbo), idesc,
                (first && s == 0) ? 0u : 1u);
        mma_f16(d, sw128_desc_mn(ah + o, lbo, sbo), sw128_desc_mn(bl + o, lbo, sbo), idesc, 1u);
        mma_f16(d, sw128_desc_mn(al + o, lbo, sbo), sw128_desc_mn(bh + o, lbo, sbo), idesc, 1u);
    }
    mma_commit(&T.bar[0]);
}

// Read the forward accumulator into shared memory G (2Kp x 2Kp FP32, row m
// at stride 2Kp + 1 against bank conflicts), reusing the operand buffers.
// All threads.
__device__ inline float *tc_read_fwd(const TcWork &T, float *G) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = warp >> 2, m = 32 * (warp & 3) + lane;
    const int N = 2 * T.Kp;
    const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
    for (int c0 = 0; c0 < T.Kp; c0 += 16) {
        float d[16];
        tmem_ld16(T.tmem + lane_base + (uint32_t)(2 * N + half * T.Kp + c0), d);
#pragma unroll
        for (int q = 0; q < 16; ++q) G[m * (N + 1) + half * T.Kp + c0 + q] = d[q];
    }
    tc_fence_before();
    __syncthreads();
    return G;
}

// Power-of-two scale taking max |w_j| (j < n) to at most 1 (all threads).
__device__ inline float pow2_scale_of(const float *w, int n, double *sbuf) {
    float mx = 0.f;
    for (int j = threadIdx.x; j < n; j += blockDim.x) mx = fmaxf(mx, fabsf(w[j]));
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sbuf[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = 0.f;
    for (int w2 = 0; w2 < kThreads / 32; ++w2) mx = fmaxf(mx, (float)sbuf[w2]);
    __syncthreads();
    return mx > 0.f ? exp2f(-ceilf(log2f(mx))) : 1.f;
}

}  // namespace img

namespace img {

__device__ inline void tc_combine_fwd(const TcWork &T, int p, const float *G, float inv,
                                      const float2 *base, bool base_identity, float2 *K);

// K(a, b) from the forward Gram matrix G (row stride 2Kp + 1), unscaled.
__device__ __forceinline__ float2 tc_k_entry(const float *G, int Kp, int a, int b) {
    const int ld = 2 * Kp + 1;
    return make_float2(G[a * ld + b] + G[(Kp + a) * ld + Kp + b], G[(Kp + a) * ld + b] - G[a * ld + Kp + b]);
}

// Forward driver: K = base + sum_j wt[j] c_j c_j^H over n list entries whose
// unweighted pixel-major tiles gen0(t, np) writes into buffer 0 (scaled by
// sX).  Needs Kp = 64 (M = N = 128).  K: p x p complex, global memory.
template <bool BF16, class Gen0>
__device__ void tc_forward(TcWork &T, int p, int n, const float *wt, float sX, Gen0 gen0,
                           const float2 *base, bool base_identity, float2 *K, double *dbuf) {
    const float sW = pow2_scale_of(wt, n, dbuf);
    const int N = 2 * T.Kp;
    const uint32_t idesc = idesc_f16_mn(N, BF16 ? 1 : 0);
    const int ntiles = (n + kTcM - 1) / kTcM;
    for (int t = 0; t < ntiles; ++t) {
        const int np = min(kTcM, n - t * kTcM);
        gen0(t, np);
        __syncthreads();
        tc_weight_rows<BF16>(T, wt + t * kTcM, np, sW);
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) tc_issue_fwd(T, idesc, t == 0);
        if (!mbar_wait(&T.bar[0], T.phase[0])) T.timeouts++;
        T.phase[0] ^= 1u;
        tc_fence_after();
        __syncthreads();
    }
    const float *G = ntiles ? tc_read_fwd(T, reinterpret_cast<float *>(T.Xhi[0])) : nullptr;
    tc_combine_fwd(T, p, G, 1.f / (sX * sX * sW), base, base_identity, K);
}

// K = base + (G -> complex p x p), scaled by inv; G may be null (empty sum).
__device__ inline void tc_combine_fwd(const TcWork &T, int p, const float *G, float inv,
                                      const float2 *base, bool base_identity, float2 *K) {
    const int N = 2 * T.Kp;
    const int ld = N + 1, Kp = T.Kp;
    for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
        const int bcol = e / p, a = e - bcol * p;
        float kr = 0.f, ki = 0.f;
        if (G) {
            kr = (G[a * ld + bcol] + G[(Kp + a) * ld + Kp + bcol]) * inv;
            ki = (G[(Kp + a) * ld + bcol] - G[a * ld + Kp + bcol]) * inv;
        }
        float2 bb = make_float2(0.f, 0.f);
        if (base) bb = base[e];
        else if (base_identity && a == bcol) bb = make_float2(1.f, 0.f);
        K[e] = make_float2(bb.x + kr, bb.y + ki);
    }
    __syncthreads();
}

}  // namespace img

namespace img {

// ---------------------------------------------------------------- resident LSQR
// During one LSQR solve the free set is fixed, so (for f <= 256 and Kp = 64)
// its X tiles stay in shared memory for every iteration: tile 0 in buffer 0,
// tile 1 in buffer 1.  The forward product stages only the weighted K-chunks
// (32 pixels, both MN blocks) in a 16 KB region after the B tiles.
constexpr int kChunk = 16;              // pixels per forward K-chunk (one MMA K-step)

// Two staging buffers (hi + lo, MN blocks x 16 rows x 128 bytes each).
__host__ __device__ inline size_t tc_stage_bytes(int p) {
    const int Kp = (p + 31) / 32 * 32;
    return (size_t)2 * 2 * (2 * Kp / 64) * kChunk * 128;
}

// Weighted chunk rows r0 .. r0+31 of resident tile `tile` into the staging
// region (MN blocks of 32 rows x 128 bytes), rows j >= nrow zero.
template <bool BF16>
__device__ inline void tc_weight_chunk(TcWork &T, unsigned char *stage, int tile, int r0, int nrow,
                                       const float *w, float sW) {
    const int nch = 2 * T.Kp / 8;
    const size_t half_bytes = (size_t)(2 * T.Kp / 64) * kChunk * 128;
    for (int it = threadIdx.x; it < kChunk * nch; it += blockDim.x) {
        const int rr = it / nch, c = it - rr * nch;
        const uint32_t src = sw128_off(r0 + rr, c, kTcM);
        const uint32_t dst = sw128_off(rr, c, kChunk);
        const float wr = rr < nrow ? sW * w[rr] : 0.f;
        const uint4 h4 = *reinterpret_cast<const uint4 *>(T.Xhi[tile] + src);
        const uint4 l4 = *reinterpret_cast<const uint4 *>(T.Xlo[tile] + src);
        const uint32_t hw[4] = {h4.x, h4.y, h4.z, h4.w}, lw[4] = {l4.x, l4.y, l4.z, l4.w};
        float v[8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float h0, h1, l0, l1;
            if (BF16) {
                h0 = __uint_as_float(hw[q] << 16);
                h1 = __uint_as_float(hw[q] & 0xffff0000u);
                l0 = __uint_as_float(lw[q] << 16);
                l1 = __uint_as_float(lw[q] & 0xffff0000u);
            } else {
                h0 = __half2float(__ushort_as_half((unsigned short)(hw[q] & 0xffffu)));
                h1 = __half2float(__ushort_as_half((unsigned short)(hw[q] >> 16)));
                l0 = __half2float(__ushort_as_half((unsigned short)(lw[q] & 0xffffu)));
                l1 = __half2float(__ushort_as_half((unsigned short)(lw[q] >> 16)));
            }
            v[2 * q] = wr * (h0 + l0);
            v[2 * q + 1] = wr * (h1 + l1);
        }
        uint4 hi, lo;
        split8<BF16>(v, hi, lo);
        *reinterpret_cast<uint4 *>(stage + dst) = hi;
        *reinterpret_cast<uint4 *>(stage + half_bytes + dst) = lo;
    }
}

// MMAs of one staged chunk against resident rows r0 .. r0+31 of `tile`,
// accumulating into the forward accumulator; commits to barrier 0.
__device__ inline void tc_issue_fwd_chunk(const TcWork &T, const unsigned char *stage, int tile, int r0,
                                          uint32_t idesc, bool first, int bar) {
    const int N = 2 * T.Kp;
    tc_fence_after();
    const size_t half_bytes = (size_t)(N / 64) * kChunk * 128;
    const uint32_t ah = smem_u32(stage), al = smem_u32(stage + half_bytes);
    const uint32_t bh = smem_u32(T.Xhi[tile]), bl = smem_u32(T.Xlo[tile]);
    const uint32_t d = T.tmem + (uint32_t)(2 * N);
    for (int s = 0; s < kChunk / 16; ++s) {
        const uint32_t ao = s * 2048, bo = (uint32_t)((r0 + 16 * s) / 8) * 1024;
        const uint32_t alb = kChunk * 128, blb = kTcM * 128;
        mma_f16(d, sw128_desc_mn(ah + ao, alb, 1024), sw128_desc_mn(bh + bo, blb, 1024), idesc,
                (first && s == 0) ? 0u : 1u);
        mma_f16(d, sw128_desc_mn(ah + ao, alb, 1024), sw128_desc_mn(bl + bo, blb, 1024), idesc, 1u);
        mma_f16(d, sw128_desc_mn(al + ao, alb, 1024), sw128_desc_mn(bh + bo, blb, 1024), idesc, 1u);
    }
    mma_commit(&T.bar[bar]);
}

// Forward over the resident free-set tiles: G = sum_j w_j x_j x_j^T read out
// into the B + staging region (the B tile is rebuilt later).  Weighted
// 16-pixel chunks alternate between two staging buffers, so weighting chunk
// c+1 overlaps the MMAs of chunk c; a buffer is reused only after the MMAs
// that read it completed.  Returns G (scaled by sX^2 sW; *scale = 1/that).
template <bool BF16>
__device__ const float *tc_forward_resident(TcWork &T, unsigned char *stage, int f, const float *w,
                                            float sX, float *scale, double *dbuf, double *cyc = nullptr) {
    long long c0 = clock64();
    const float sW = pow2_scale_of(w, f, dbuf);
    const uint32_t idesc = idesc_f16_mn(2 * T.Kp, BF16 ? 1 : 0);
    const int nchunks = (f + kChunk - 1) / kChunk;
    const size_t buf = (size_t)2 * (2 * T.Kp / 64) * kChunk * 128;   // one staging buffer (hi + lo)
    for (int c = 0; c < nchunks; ++c) {
        const int b = c & 1;
        if (c >= 2) {
            if (!mbar_wait(&T.bar[b], T.phase[b])) T.timeouts++;
            T.phase[b] ^= 1u;
            tc_fence_after();
        }
        const int j0 = c * kChunk, tile = j0 / kTcM, r0 = j0 % kTcM;
        tc_weight_chunk<BF16>(T, stage + b * buf, tile, r0, min(kChunk, f - j0), w + j0, sW);
        fence_async_smem();
        __syncthreads();
        if (threadIdx.x == 0) tc_issue_fwd_chunk(T, stage + b * buf, tile, r0, idesc, c == 0, b);
    }
    for (int c = max(0, nchunks - 2); c < nchunks; ++c) {
        const int b = c & 1;
        if (!mbar_wait(&T.bar[b], T.phase[b])) T.timeouts++;
        T.phase[b] ^= 1u;
    }
    tc_fence_after();
    __syncthreads();
    long long c1 = clock64();
    *scale = 1.f / (sX * sX * sW);
    const float *G = nchunks ? tc_read_fwd(T, reinterpret_cast<float *>(T.Bhi)) : nullptr;
    if (cyc) {
        cyc[0] += (double)(c1 - c0);
        cyc[1] += (double)(clock64() - c1);
    }
    return G;
}

// Adjoint over the resident tiles: epi(j, Re(c_j^H U c_j)) for j < f.
template <bool BF16, class Epi>
__device__ void tc_adjoint_resident(TcWork &T, const float2 *U, int p, int f, float sX, float *red,
                                    double *dbuf, Epi epi, double *cyc = nullptr) {
    long long c0 = clock64();
    const float sB = tc_build_B<BF16>(U, p, T, dbuf);
    const uint32_t idesc = idesc_f16(2 * T.Kp, BF16 ? 1 : 0);
    const int ntiles = (f + kTcM - 1) / kTcM;
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0)
        for (int t = 0; t < ntiles; ++t) tc_issue(T, t, idesc);
    const float inv = 1.f / (sX * sX * sB);
    long long c1 = clock64(), cw = 0, ce = 0;
    for (int t = 0; t < ntiles; ++t) {
        long long a0 = clock64();
        if (!mbar_wait(&T.bar[t], T.phase[t])) T.timeouts++;
        T.phase[t] ^= 1u;
        tc_fence_after();
        __syncthreads();
        long long a1 = clock64();
        tc_epilogue<BF16>(T, t, red);
        const int j = t * kTcM + threadIdx.x;
        if (threadIdx.x < kTcM && j < f) epi(j, red[threadIdx.x] * inv);
        __syncthreads();
        cw += a1 - a0;
        ce += clock64() - a1;
    }
    if (cyc) {
        cyc[3] += (double)(c1 - c0);
        cyc[4] += (double)cw;
        cyc[5] += (double)ce;
    }
}

}  // namespace img
