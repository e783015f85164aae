// Tensor-core adjoint Psi^H for wide arrays, 64 < p <= 256: out_i =
// x_i^T B x_i with x_i = [Re a_i; Im a_i] and B the real embedding of U
// (Sec. V-B), as in tc_ops.cuh, but the 2Kp x 2Kp operand (Kp = p rounded up
// to 32, N = 2Kp) no longer fits in shared memory.
//
// * emb_B_chunk writes B once per operator to global memory (L2-resident, at
//   most 2 MB) as K-chunks of 64 columns; each chunk is one or two "units",
//   each the exact shared-memory image (hi part, then lo part) of a swizzled
//   K-major tile of at most 256 rows, so a unit moves with one bulk copy
//   (cp.async.bulk, completion counted in bytes on an mbarrier).
// * The operator is warp-specialised, with mbarrier hand-offs only:
//     warps 0-3  epilogue: tensor memory -> x_i^T (B x_i), one pixel per
//                thread, table rows staged per warp by asynchronous copies;
//     warps 4-7  steering producers: 64-column chunks of the 128-pixel tile
//                (FP32 products of the separable tables, split hi + lo);
//     warp 8     copies of B units and the MMAs (lane 0 issues).
//   Two X stages, two B stages (64 KB each) and two accumulator regions of
//   256 tensor-memory columns: for Kp <= 128 consecutive tiles alternate
//   regions, so the epilogue of one tile overlaps the MMAs of the next; for
//   Kp > 128 each tile spans both regions (B rows split in two units) and a
//   region is handed back as soon as the epilogue has read it.
#pragma once
#include <type_traits>

#include "tc_ops.cuh"

namespace img {

constexpr int kWideMaxP = 256;
constexpr int kChunkK = 64;                 // K columns per chunk (one 128-byte swizzle atom)
constexpr int kWideThreads = 288;           // 9 warps
constexpr size_t kWideXStage = 2 * kTcM * 128;       // hi + lo, 32 KB
constexpr size_t kWideBStage = 64 * 1024;

__host__ __device__ inline int wide_kp(int p) { return (p + 31) / 32 * 32; }
// B units per chunk: two when N = 2Kp > 256 (one MMA takes N <= 256).
__host__ __device__ inline int wide_units(int p) { return 2 * wide_kp(p) > 256 ? 2 : 1; }
__host__ __device__ inline int wide_unit_rows(int p) { return wide_units(p) == 2 ? wide_kp(p) : 2 * wide_kp(p); }
__host__ __device__ inline size_t wide_unit_bytes(int p) { return (size_t)2 * wide_unit_rows(p) * 128; }
__host__ __device__ inline size_t wide_chunk_bytes(int p) { return (size_t)2 * 2 * wide_kp(p) * 128; }
__host__ __device__ inline int wide_nk(int p) { return 2 * wide_kp(p) / kChunkK; }
__host__ __device__ inline size_t wide_B_bytes(int p) { return wide_chunk_bytes(p) * wide_nk(p); }
// Epilogue staging per warp: 3 buffers x 12 table rows x 16 k (row stride
// 18 float2, so 16-byte reads of the 8 E_l rows hit distinct banks).
constexpr int kEpiRow = 18;
constexpr size_t kEpiStage = (size_t)3 * 12 * kEpiRow * 8;
__host__ __device__ inline size_t wide_smem_bytes(int) {
    return 2 * kWideXStage + 2 * kWideBStage + 4 * kEpiStage + 1024;
}

// Row n of B (the N index, i.e. column n of the accumulator) holds the
// (part, k) of x it multiplies in the epilogue.  One unit: [Re 0..Kp-1,
// Im 0..Kp-1].  Two units: unit g holds k in [g*h, (g+1)*h), h = Kp/2, as
// [Re ..., Im ...], so each accumulator region covers both parts of its k.
__device__ __forceinline__ void wide_row(int n, int Kp, int nu, int &part, int &k) {
    if (nu == 1) {
        part = n >= Kp;
        k = n - part * Kp;
    } else {
        const int h = Kp >> 1, g = n / Kp, r = n - g * Kp;
        part = r >= h;
        k = g * h + r - part * h;
    }
}

// ---------------------------------------------------------------- barriers, bulk copy
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
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
// 8-byte asynchronous global -> shared copy (zero-filled when !valid; src
// must still be a readable address).
__device__ __forceinline__ void cp_async8(void *dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(valid ? 8 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }

// ---------------------------------------------------------------- B image
__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
__device__ __forceinline__ float2 to_f2(double2 v) { return make_float2((float)v.x, (float)v.y); }

// max |Re|, |Im| over the p^2 entries of U (rounded to FP32), one block's
// share (grid-stride over blocks `b` of `nb`), folded into *mx as the bit
// pattern of a non-negative float (atomicMax on the bits is monotonic).
// *mx must be zero before the first block adds to it.
template <class TC>
__device__ inline void emb_absmax(const TC *U, int p, int b, int nb, unsigned *mx_bits) {
    __shared__ float sred[32];
    const int n2 = p * p, stride = nb * blockDim.x;
    float mx = 0.f;
    int e = b * blockDim.x + threadIdx.x;
    for (; e + 3 * stride < n2; e += 4 * stride) {
        float2 v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = to_f2(U[e + q * stride]);
#pragma unroll
        for (int q = 0; q < 4; ++q) mx = fmaxf(mx, fmaxf(fabsf(v[q].x), fabsf(v[q].y)));
    }
    for (; e < n2; e += stride) {
        const float2 v = to_f2(U[e]);
        mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.y)));
    }
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x + 31) / 32; ++w) mx = fmaxf(mx, sred[w]);
        mx = fmaxf(mx, sred[0]);
        atomicMax(mx_bits, __float_as_uint(mx));
    }
}

// Power-of-two scale that brings max |U| to (1/2, 1].
__device__ __forceinline__ float emb_scale_of(unsigned mx_bits) {
    const float mx = __uint_as_float(mx_bits);
    return mx > 0.f ? exp2f(-ceilf(log2f(mx))) : 1.f;
}

// Rows per CTA of the B image kernels (grid: chunks x N / kEmbRows).
constexpr int kEmbRows = 64;

// Rows [rb * kEmbRows, +kEmbRows) of chunk kc of the B image of U
// (column-major p x p, FP32 or FP64 complex, used as FP32): B = emb(V), V = U^H, whose quadratic form equals
// that of emb(U).  With u = U[k_row * p + k_col] (= conj V(k_row, k_col)):
// blocks (Re, Re) and (Im, Im) hold u.x, (Re, Im) holds u.y, (Im, Re) holds
// -u.y; scaled by the power of two of emb_scale_of(mx_bits) (max |U| from
// emb_absmax).  The CTA of chunk 0, row block 0 stores the scale.
template <bool BF16, class TC>
__device__ void emb_B_chunk(const TC *U, int p, unsigned char *img, unsigned mx_bits, float *scale, int kc,
                            int rb) {
    const int Kp = wide_kp(p), nc8 = Kp / 8, nu = wide_units(p), rows_u = wide_unit_rows(p);
    const float sc = emb_scale_of(mx_bits);
    if (kc == 0 && rb == 0 && threadIdx.x == 0) *scale = sc;
    unsigned char *chunk = img + (size_t)kc * wide_chunk_bytes(p);
    const size_t ub = wide_unit_bytes(p);
    for (int it = threadIdx.x; it < kEmbRows * 8; it += blockDim.x) {
        const int n = rb * kEmbRows + (it >> 3), cc = it & 7;
        const int g = kc * 8 + cc;                    // global 8-column group
        const int cpart = g >= nc8, k0 = (g - cpart * nc8) * 8;
        int rpart, kr;
        wide_row(n, Kp, nu, rpart, kr);
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            float2 u = make_float2(0.f, 0.f);
            if (kr < p && k0 + e < p) u = to_f2(U[(size_t)kr * p + k0 + e]);
            const float val = (rpart == cpart) ? u.x : (rpart == 0 ? u.y : -u.y);
            v[e] = val * sc;
        }
        uint4 hi, lo;
        split8<BF16>(v, hi, lo);
        const int un = n / rows_u, rr = n - un * rows_u;
        const size_t off = (size_t)un * ub + (size_t)(rr >> 3) * 1024 + (rr & 7) * 128 + ((cc ^ (rr & 7)) << 4);
        *reinterpret_cast<uint4 *>(chunk + off) = hi;
        *reinterpret_cast<uint4 *>(chunk + off + (size_t)rows_u * 128) = lo;
    }
}

// ---------------------------------------------------------------- operator
// Barrier slots in the caller's kWideBars-entry shared array.
enum : int { kBFull = 0, kBEmpty = 2, kXFull = 4, kXEmpty = 6, kAFull = 8, kAEmpty = 10, kWideBars = 12 };

// Wait for the next phase of barrier `slot`; its parity is bit `slot` of ph.
// After one wait of this thread has timed out the pipeline is broken: later
// waits poll once, so the kernel still ends in bounded time (and reports).
__device__ __forceinline__ void wide_wait(uint64_t *bars, int slot, uint32_t &ph, int &timeouts) {
    const uint32_t par = (ph >> slot) & 1u;
    ph ^= 1u << slot;
    if (timeouts) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(&bars[slot])), "r"(par)
            : "memory");
        if (!done) timeouts++;
        return;
    }
    if (!mbar_wait(&bars[slot], par)) timeouts++;
}

// out = Re(a_i^H U_s a_i) for npass <= 2 operators s (B images B0, B1,
// scales sB[s]) over the 2-D tiles t0, t0 + dt, ... (ntiles of them);
// epi(s, i, v) receives each pixel's value.  Bit s of sq_mask makes pass s
// a sum of squares instead, out = ||V_s a_i||^2 with V_s = U_s^H (the B
// image of U_s = L^-H gives the whitened MVDR denominator ||L^-1 a_i||^2).  Needs kWideThreads threads,
// 1024-aligned dynamic shared memory `dyn` of wide_smem_bytes(p) - 1024
// bytes and kWideBars mbarriers.  Returns the number of waits that timed out.
template <bool BF16, class Epi>
__device__ int wide_adjoint(const JobDev &J, unsigned char *dyn, uint64_t *bars, uint32_t *slot,
                            const unsigned char *B0, const unsigned char *B1, const float *sB, int npass,
                            int t0, int dt, int ntiles, int sq_mask, Epi epi) {
    const int p = J.p, Kp = wide_kp(p), nk = wide_nk(p), nu = wide_units(p), rows_u = wide_unit_rows(p);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *Xs = dyn, *Bs = dyn + 2 * kWideXStage;
    __shared__ int s_timeouts;
    if (threadIdx.x == 0) {
        s_timeouts = 0;
        for (int q = 0; q < 2; ++q) {
            mbar_init(&bars[kBFull + q], 1);
            mbar_init(&bars[kBEmpty + q], 1);
            mbar_init(&bars[kXFull + q], 4);
            mbar_init(&bars[kXEmpty + q], 1);
            mbar_init(&bars[kAFull + q], 1);
            mbar_init(&bars[kAEmpty + q], 4);
        }
    }
    if (warp == 0) tmem_alloc(slot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const float sX = steer_scale(p);
    const int tiles = npass * ntiles;             // tile uses, pass-major
    const int total = tiles * nk;                 // X chunks
    const int nl = J.n_l, nm = J.n_m, tl = (nl + kTileL - 1) / kTileL;
    int timeouts = 0;

    if (warp == 8) {
        // ---------------- copies and MMAs.  The whole warp walks the unit
        // sequence and waits (warp-uniform control flow); lane 0 issues.
        // Unit u = (chunk c, part pp) uses B stage u & 1; the copy of unit
        // u + 1 is issued once the MMAs of unit u - 1 released its stage.
        if (total > 0) {
            const bool leader = lane == 0;
            const uint32_t ub = (uint32_t)wide_unit_bytes(p);
            const size_t cb = wide_chunk_bytes(p);
            const uint32_t idesc = idesc_f16(rows_u, BF16 ? 1 : 0);
            const int units = total * nu;
            uint32_t ph = 0;
            const int first_reuse = nu == 2 ? 1 : 2;   // first use of a region needs no hand-back
            auto src = [&](int u) {
                const int c = u / nu, pp = u - c * nu, T = c / nk, kc = c - T * nk;
                return (T < ntiles ? B0 : B1) + (size_t)kc * cb + (size_t)pp * ub;
            };
            if (leader) {
                mbar_expect_tx(&bars[kBFull], ub);
                tma_bulk_g2s(Bs, src(0), ub, &bars[kBFull]);
            }
            for (int u = 0; u < units; ++u) {
                const int c = u / nu, pp = u - c * nu, T = c / nk, kc = c - T * nk, s = u & 1;
                if (pp == 0) wide_wait(bars, kXFull + (c & 1), ph, timeouts);
                const int g = nu == 2 ? pp : (T & 1);
                if (kc == 0 && T >= first_reuse) wide_wait(bars, kAEmpty + g, ph, timeouts);
                wide_wait(bars, kBFull + s, ph, timeouts);
                tc_fence_after();
                if (leader) {
                    const uint32_t xh = smem_u32(Xs + (c & 1) * kWideXStage), xl = xh + kTcM * 128;
                    const uint32_t bh = smem_u32(Bs + s * kWideBStage), bl = bh + (uint32_t)rows_u * 128;
                    const uint32_t d = tmem + (uint32_t)(g * 256);
#pragma unroll
                    for (int st = 0; st < kChunkK / 16; ++st) {
                        const uint32_t o = st * 32;
                        mma_f16(d, sw128_desc(xh + o), sw128_desc(bh + o), idesc, (kc > 0 || st > 0) ? 1u : 0u);
                        mma_f16(d, sw128_desc(xh + o), sw128_desc(bl + o), idesc, 1u);
                        mma_f16(d, sw128_desc(xl + o), sw128_desc(bh + o), idesc, 1u);
                    }
                    mma_commit(&bars[kBEmpty + s]);
                    if (pp == nu - 1) mma_commit(&bars[kXEmpty + (c & 1)]);
                    if (kc == nk - 1) mma_commit(&bars[kAFull + g]);
                }
                __syncwarp();
                if (u + 1 < units) {
                    // stage s^1 was last read by the MMAs of unit u - 1
                    const int s1 = s ^ 1;
                    if (u >= 1) wide_wait(bars, kBEmpty + s1, ph, timeouts);
                    if (leader) {
                        mbar_expect_tx(&bars[kBFull + s1], ub);
                        tma_bulk_g2s(Bs + s1 * kWideBStage, src(u + 1), ub, &bars[kBFull + s1]);
                    }
                }
            }
        }
    } else if (warp >= 4) {
        // ---------------- steering producers: chunk c of tile use T into X stage c & 1.
        // Warp w fills rows 32w + 8b + a (l offset a = 0..7, m offset 4w + b),
        // lane j columns 2j, 2j+1 of the chunk; all 12 table loads of a chunk
        // are issued before the wait for the stage.
        const int w = warp - 4;
        const bool vec = (p & 1) == 0;
        const float2 *__restrict__ El = J.El;
        const float2 *__restrict__ Em = J.Em;
        // byte offset of (row 32w + a, this lane's column pair); row 32w + 8b + a adds b * 1024
        uint32_t xo[8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
            xo[a] = (uint32_t)(4 * w * 1024 + a * 128 + (((lane >> 2) ^ a) << 4) + (lane & 3) * 4);
        uint32_t ph = 0;
        // the 12 table loads of chunk c + 1 are in flight while chunk c is written
        float2 e[8][2], f[4][2];
        auto load = [&](int c) {
            const int T = c / nk, kc = c - T * nk;
            const int t = t0 + (T % ntiles) * dt;
            const int bm = t / tl, bl = t - bm * tl;
            const int il0 = bl * kTileL, im0 = bm * kTileM + 4 * w;
            const int col = kc * kChunkK + 2 * lane;
            const int k = col >= Kp ? col - Kp : col;
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const int il = il0 + a;
                e[a][0] = e[a][1] = make_float2(0.f, 0.f);
                if (il < nl && k < p) {
                    const float2 *src = El + (size_t)il * p + k;
                    if (vec) {
                        const float4 v = __ldg(reinterpret_cast<const float4 *>(src));
                        e[a][0] = make_float2(v.x, v.y);
                        e[a][1] = make_float2(v.z, v.w);
                    } else {
                        e[a][0] = __ldg(src);
                        if (k + 1 < p) e[a][1] = __ldg(src + 1);
                    }
                }
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int im = im0 + b;
                f[b][0] = f[b][1] = make_float2(0.f, 0.f);
                if (im < nm && k < p) {
                    const float2 *src = Em + (size_t)im * p + k;
                    if (vec) {
                        const float4 v = __ldg(reinterpret_cast<const float4 *>(src));
                        f[b][0] = make_float2(v.x, v.y);
                        f[b][1] = make_float2(v.z, v.w);
                    } else {
                        f[b][0] = __ldg(src);
                        if (k + 1 < p) f[b][1] = __ldg(src + 1);
                    }
                }
            }
        };
        if (total > 0) load(0);
        for (int c = 0; c < total; ++c) {
            const int kc = c % nk, s = c & 1;
            const int part = kc * kChunkK + 2 * lane >= Kp;
            float2 ec[8][2], fc[4][2];
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                ec[a][0] = e[a][0];
                ec[a][1] = e[a][1];
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                fc[b][0] = f[b][0];
                fc[b][1] = f[b][1];
            }
            if (c + 1 < total) load(c + 1);
            // v = Re(e f) = e.x (f.x) + e.y (-f.y), or Im(e f) = e.x (f.y) + e.y (f.x):
            // fold the part and the scale into f once per chunk
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const float2 v = fc[b][q];
                    fc[b][q] = part ? make_float2(v.y * sX, v.x * sX) : make_float2(v.x * sX, -v.y * sX);
                }
            if (c >= 2) wide_wait(bars, kXEmpty + s, ph, timeouts);
            unsigned char *xh = Xs + s * kWideXStage, *xl = xh + kTcM * 128;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const float v0 = fmaf(ec[a][0].x, fc[b][0].x, ec[a][0].y * fc[b][0].y);
                    const float v1 = fmaf(ec[a][1].x, fc[b][1].x, ec[a][1].y * fc[b][1].y);
                    uint32_t hi, lo;
                    split2<BF16>(v0, v1, hi, lo);
                    const uint32_t off = xo[a] + b * 1024;
                    *reinterpret_cast<uint32_t *>(xh + off) = hi;
                    *reinterpret_cast<uint32_t *>(xl + off) = lo;
                }
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[kXFull + s]);
        }
    } else {
        // ---------------- epilogue: one pixel row per thread.  Each warp
        // stages, 16 k at a time, the 8 E_l rows and its 4 E_m rows of the
        // tile in shared memory (asynchronous copies, three buffers, two
        // groups ahead), then reads the accumulator 2 x 16 columns at a time.
        const int r = 32 * warp + lane;
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        const int wcols = nu == 2 ? Kp / 2 : Kp, ng = Kp / 16;
        const float2 *__restrict__ El = J.El;
        const float2 *__restrict__ Em = J.Em;
        float2 *S = reinterpret_cast<float2 *>(Bs + 2 * kWideBStage + warp * kEpiStage);
        uint32_t ph = 0;
        for (int T = 0; T < tiles; ++T) {
            const int pass = T / ntiles, t = t0 + (T - pass * ntiles) * dt;
            const int bm = t / tl, bl = t - bm * tl;
            const int il0 = bl * kTileL, im0 = bm * kTileM + 4 * warp;
            // group gi: rows 0-7 E_l(il0 + row), rows 8-11 E_m(im0 + row - 8), k = 16 gi ..
            auto issue = [&](int gi) {
                if (gi < ng) {
                    float2 *dst = S + (gi % 3) * 12 * kEpiRow;
#pragma unroll
                    for (int q0 = 0; q0 < 12 * 16; q0 += 32) {
                        const int q = q0 + lane, row = q >> 4, kk = q & 15, k = gi * 16 + kk;
                        const bool isl = row < kTileL;
                        const int gr = isl ? il0 + row : im0 + row - kTileL;
                        const bool ok = (isl ? gr < nl : gr < nm) && k < p;
                        const float2 *src = ok ? (isl ? El : Em) + (size_t)gr * p + k : El;
                        cp_async8(dst + row * kEpiRow + kk, src, ok);
                    }
                }
                cp_async_commit();
            };
            issue(0);
            issue(1);
            const int i = tc_tile_pixel(t, r, nl, nm);
            const bool sq = (sq_mask >> pass) & 1;
            float acc = 0.f;
            int grp = 0;
            for (int pp = 0; pp < nu; ++pp) {
                const int g = nu == 2 ? pp : (T & 1);
                wide_wait(bars, kAFull + g, ph, timeouts);
                tc_fence_after();
                const uint32_t base = tmem + lane_base + (uint32_t)(g * 256);
                for (int kk = 0; kk < wcols; kk += 16, ++grp) {
                    issue(grp + 2);
                    cp_async_wait2();
                    __syncwarp();
                    const float2 *sb = S + (grp % 3) * 12 * kEpiRow;
                    const float4 *se = reinterpret_cast<const float4 *>(sb + (lane & 7) * kEpiRow);
                    const float4 *sf = reinterpret_cast<const float4 *>(sb + (kTileL + (lane >> 3)) * kEpiRow);
                    float ar[16], ai[16];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float4 ev = se[j], fv = sf[j];
                        const float2 a0 = cmul(make_float2(ev.x, ev.y), make_float2(fv.x, fv.y));
                        const float2 a1 = cmul(make_float2(ev.z, ev.w), make_float2(fv.z, fv.w));
                        ar[2 * j] = a0.x;
                        ai[2 * j] = a0.y;
                        ar[2 * j + 1] = a1.x;
                        ai[2 * j + 1] = a1.y;
                    }
                    float dr[16], di[16];
                    tmem_ld16x2(base + kk, base + wcols + kk, dr, di);
                    if (sq) {
#pragma unroll
                        for (int q = 0; q < 16; ++q) acc = fmaf(dr[q], dr[q], fmaf(di[q], di[q], acc));
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q) acc = fmaf(ar[q], dr[q], fmaf(ai[q], di[q], acc));
                    }
                    __syncwarp();
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars[kAEmpty + g]);
            }
            if (i >= 0) {
                // the steering side entered the MMA scaled by sX, the dot above
                // unscaled; a sum of squares carries both scales twice
                const float sc = sq ? (sX * sB[pass]) * (sX * sB[pass]) : sX * sB[pass];
                epi(pass, i, acc / sc);
            }
        }
    }
    if (timeouts) atomicAdd(&s_timeouts, timeouts);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
    return s_timeouts;
}


// ================================================================ forward
// Psi x for 64 < p <= 256 on tensor cores: K = sum_i w_i a_i a_i^H from the
// real Gram matrix G = sum_i w_i x_i x_i^T (2Kp x 2Kp), K = (G_rr + G_ii) +
// j (G_ir - G_ri).  G is tiled in blocks of 128 rows (features 128m ..) by up
// to 256 columns (features 256nb ..); only blocks that reach the upper
// triangle are formed.  One CTA accumulates one block over a strided share
// of 64-pixel stages (8 x 8 grid blocks) with the pixel index as the MMA's K
// dimension: both operands are pixel-major tiles read as MN-major operands
// (the same swizzled layout the adjoint's steering tiles use), A unweighted
// and B weighted by w_i, split hi + lo as in the adjoint.  Each CTA writes its
// FP32 block to a partial buffer; fwd_assemble sums the partials in a fixed
// order (deterministic) and forms K.
//   warps 0-7  steering producers (then warps 0-3 read the accumulator);
//   warp 8     MMA issue (lane 0).
constexpr int kFwdPix = 64;                                  // pixels per stage
constexpr size_t kFwdChunk = (size_t)kFwdPix * 128;          // one 64-feature chunk, 8 KB
constexpr size_t kFwdStage = (2 + 4) * 2 * kFwdChunk;        // A: 2 chunks, B: 4 chunks, hi + lo
constexpr int kFwdThreads = 288;
__host__ __device__ inline size_t fwd_smem_bytes() { return 2 * kFwdStage + 1024; }
__host__ __device__ inline int fwd_n_of(int p, int nb) {
    const int n = 2 * wide_kp(p) - 256 * nb;
    return n < 256 ? n : 256;
}
// Blocks (m, nb) of G that reach the upper triangle, in a fixed order.
__host__ __device__ inline int fwd_pairs(int p, int *pm, int *pnb) {
    const int N = 2 * wide_kp(p), nm = (N + 127) / 128, nnb = (N + 255) / 256;
    int k = 0;
    for (int m = 0; m < nm; ++m)
        for (int nb = 0; nb < nnb; ++nb)
            if (256 * nb + fwd_n_of(p, nb) - 1 >= 128 * m) {
                if (pm) pm[k] = m;
                if (pnb) pnb[k] = nb;
                ++k;
            }
    return k;
}
__host__ __device__ inline int fwd_nblocks(int n_l, int n_m) { return ((n_l + 7) / 8) * ((n_m + 7) / 8); }

// Instruction descriptor, kind::f16, F32 accumulate, both operands MN-major,
// M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_f16_mn128(int n, int ab_fmt) {
    return (1u << 4) | ((uint32_t)ab_fmt << 7) | ((uint32_t)ab_fmt << 10) | (1u << 15) | (1u << 16) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

// max |w| over Q weights (block share of a grid-stride pass), into *mx_bits.
__device__ inline void fwd_wmax(const float *w, int Q, unsigned *mx_bits) {
    __shared__ float sred[32];
    float mx = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Q; i += gridDim.x * blockDim.x) mx = fmaxf(mx, fabsf(w[i]));
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x + 31) / 32; ++q) mx = fmaxf(mx, sred[q]);
        mx = fmaxf(mx, sred[0]);
        atomicMax(mx_bits, __float_as_uint(mx));
    }
}

// One CTA: block `pair` of G over the pixel blocks s, s + S, ... of the grid;
// writes the FP32 block (128 x 256, row-major) to out.  w: pixel weights;
// wbits: max |w| bits.  Returns the number of waits that timed out.
template <bool BF16>
__device__ int wide_forward(const JobDev &J, unsigned char *dyn, uint64_t *bars, uint32_t *slot, const float *w,
                            unsigned wbits, int m, int nb, int s0, int S, float *out) {
    const int p = J.p, Kp = wide_kp(p), Nf = 2 * Kp, N = fwd_n_of(p, nb);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nl = J.n_l, nm = J.n_m, tlb = (nl + 7) / 8, nblk = fwd_nblocks(nl, nm);
    const int mine = nblk > s0 ? (nblk - 1 - s0) / S + 1 : 0;
    const float sX = steer_scale(p);
    const float sW = emb_scale_of(wbits);
    enum { kFull = 0, kEmpty = 2, kAcc = 4 };
    __shared__ int s_timeouts;
    if (threadIdx.x == 0) {
        s_timeouts = 0;
        for (int q = 0; q < 2; ++q) {
            mbar_init(&bars[kFull + q], 8);
            mbar_init(&bars[kEmpty + q], 1);
        }
        mbar_init(&bars[kAcc], 1);
    }
    if (warp == 0) tmem_alloc(slot, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    int timeouts = 0;
    uint32_t ph = 0;
    // chunks of features: A = {2m, 2m+1}, B = {4nb .. 4nb+3}; chunk list without repeats
    int chunk[6], nchunk = 0;
    for (int q = 0; q < 2; ++q) chunk[nchunk++] = 2 * m + q;
    for (int q = 0; q < 4; ++q) {
        const int c = 4 * nb + q;
        if (64 * c < 256 * nb + N && c != 2 * m && c != 2 * m + 1) chunk[nchunk++] = c;
    }

    if (warp == 8) {
        if (lane == 0 && mine > 0) {
            const uint32_t idesc = idesc_f16_mn128(N, BF16 ? 1 : 0);
            for (int t = 0; t < mine; ++t) {
                const int sg = t & 1;
                wide_wait(bars, kFull + sg, ph, timeouts);
                tc_fence_after();
                const uint32_t base = smem_u32(dyn + sg * kFwdStage);
                const uint32_t ah = base, al = base + 2 * kFwdChunk;
                const uint32_t bh = base + 4 * kFwdChunk, bl = base + 8 * kFwdChunk;
#pragma unroll
                for (int st = 0; st < kFwdPix / 16; ++st) {
                    const uint32_t o = st * 2048;
                    const uint32_t acc = (t > 0 || st > 0) ? 1u : 0u;
                    mma_f16(tmem, sw128_desc_mn(ah + o, kFwdChunk, 1024), sw128_desc_mn(bh + o, kFwdChunk, 1024),
                            idesc, acc);
                    mma_f16(tmem, sw128_desc_mn(ah + o, kFwdChunk, 1024), sw128_desc_mn(bl + o, kFwdChunk, 1024),
                            idesc, 1u);
                    mma_f16(tmem, sw128_desc_mn(al + o, kFwdChunk, 1024), sw128_desc_mn(bh + o, kFwdChunk, 1024),
                            idesc, 1u);
                }
                mma_commit(&bars[kEmpty + sg]);
                if (t == mine - 1) mma_commit(&bars[kAcc]);
            }
        }
    } else {
        // ---------------- producers: warp w takes tasks (chunk, half h) w, w + 8, ...
        // of each stage: the 32 pixel rows of m offsets b = 4h .. 4h+3 (l offsets
        // a = 0..7), lane j the features 2j, 2j+1 of the chunk.  The 8 E_l and
        // 4 E_m entries and the 32 weights of the warp's next task (in this
        // stage or the next) load while the current task is written.
        const bool vec = (p & 1) == 0, wvec = (nl & 3) == 0;
        const float2 *__restrict__ El = J.El;
        const float2 *__restrict__ Em = J.Em;
        const int ntask = nchunk * 2;
        const int my = warp < ntask ? (ntask - 1 - warp) / 8 + 1 : 0;    // tasks per stage
        // swizzled byte offset of (row a, this lane's column pair) in an 8-row group
        uint32_t xo[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) xo[a] = (uint32_t)(a * 128 + (((lane >> 2) ^ a) << 4) + (lane & 3) * 4);
        float2 e[8][2], fm[4][2];
        float wr[4][8];
        auto load = [&](int t, int task) {
            const int blk = s0 + t * S, bm = blk / tlb, bl = blk - bm * tlb;
            const int ci = task >> 1, h = task & 1, c = chunk[ci];
            const int f = c * 64 + 2 * lane, part = f >= Kp, k = f - part * Kp;
            const bool kok = f < Nf && k < p;
#pragma unroll
            for (int a = 0; a < 8; ++a) {
                const int il = bl * 8 + a;
                e[a][0] = e[a][1] = make_float2(0.f, 0.f);
                if (kok && il < nl) {
                    const float2 *src = El + (size_t)il * p + k;
                    if (vec) {
                        const float4 v = __ldg(reinterpret_cast<const float4 *>(src));
                        e[a][0] = make_float2(v.x, v.y);
                        e[a][1] = make_float2(v.z, v.w);
                    } else {
                        e[a][0] = __ldg(src);
                        if (k + 1 < p) e[a][1] = __ldg(src + 1);
                    }
                }
            }
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) {
                const int im = bm * 8 + 4 * h + bb;
                fm[bb][0] = fm[bb][1] = make_float2(0.f, 0.f);
                if (kok && im < nm) {
                    const float2 *src = Em + (size_t)im * p + k;
                    if (vec) {
                        const float4 v = __ldg(reinterpret_cast<const float4 *>(src));
                        fm[bb][0] = make_float2(v.x, v.y);
                        fm[bb][1] = make_float2(v.z, v.w);
                    } else {
                        fm[bb][0] = __ldg(src);
                        if (k + 1 < p) fm[bb][1] = __ldg(src + 1);
                    }
                }
                // the 8 weights of this m row (same address in every lane)
                const int il0 = bl * 8;
                const float *wrow = w + (size_t)im * nl + il0;
                if (im < nm && wvec && il0 + 8 <= nl) {
                    const float4 w0 = __ldg(reinterpret_cast<const float4 *>(wrow));
                    const float4 w1 = __ldg(reinterpret_cast<const float4 *>(wrow) + 1);
                    wr[bb][0] = w0.x; wr[bb][1] = w0.y; wr[bb][2] = w0.z; wr[bb][3] = w0.w;
                    wr[bb][4] = w1.x; wr[bb][5] = w1.y; wr[bb][6] = w1.z; wr[bb][7] = w1.w;
                } else {
#pragma unroll
                    for (int a = 0; a < 8; ++a) wr[bb][a] = (im < nm && il0 + a < nl) ? __ldg(wrow + a) : 0.f;
                }
            }
        };
        // write one task: rows of m offsets 4h + bb; A (unweighted) and/or B (weighted) copies
        auto emit = [&](unsigned char *st, int c, int h, int part, auto inA_t, auto inB_t) {
            constexpr bool inA = decltype(inA_t)::value, inB = decltype(inB_t)::value;
            unsigned char *ah = st + (size_t)(c - 2 * m) * kFwdChunk + h * 4096;
            unsigned char *bh = st + 4 * kFwdChunk + (size_t)(c - 4 * nb) * kFwdChunk + h * 4096;
            float2 fc[4][2];
#pragma unroll
            for (int bb = 0; bb < 4; ++bb)
#pragma unroll
                for (int qq = 0; qq < 2; ++qq) {
                    const float2 v = fm[bb][qq];
                    fc[bb][qq] = part ? make_float2(v.y * sX, v.x * sX) : make_float2(v.x * sX, -v.y * sX);
                }
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) {
#pragma unroll
                for (int a = 0; a < 8; ++a) {
                    const float v0 = fmaf(e[a][0].x, fc[bb][0].x, e[a][0].y * fc[bb][0].y);
                    const float v1 = fmaf(e[a][1].x, fc[bb][1].x, e[a][1].y * fc[bb][1].y);
                    const uint32_t off = xo[a] + bb * 1024;
                    uint32_t hi, lo;
                    if (inA) {
                        split2<BF16>(v0, v1, hi, lo);
                        *reinterpret_cast<uint32_t *>(ah + off) = hi;
                        *reinterpret_cast<uint32_t *>(ah + 2 * kFwdChunk + off) = lo;
                    }
                    if (inB) {
                        const float wi = wr[bb][a] * sW;
                        split2<BF16>(v0 * wi, v1 * wi, hi, lo);
                        *reinterpret_cast<uint32_t *>(bh + off) = hi;
                        *reinterpret_cast<uint32_t *>(bh + 4 * kFwdChunk + off) = lo;
                    }
                }
            }
        };
        if (mine > 0 && my > 0) load(0, warp);
        for (int t = 0; t < mine; ++t) {
            const int sg = t & 1;
            if (t >= 2) wide_wait(bars, kEmpty + sg, ph, timeouts);
            unsigned char *st = dyn + sg * kFwdStage;
            for (int q = 0; q < my; ++q) {
                const int task = warp + 8 * q;
                const int ci = task >> 1, h = task & 1, c = chunk[ci];
                const int part = c * 64 + 2 * lane >= Kp;
                const bool inA = c == 2 * m || c == 2 * m + 1;
                const bool inB = c >= 4 * nb && 64 * c < 256 * nb + N;
                if (inA && inB) emit(st, c, h, part, std::true_type{}, std::true_type{});
                else if (inA) emit(st, c, h, part, std::true_type{}, std::false_type{});
                else emit(st, c, h, part, std::false_type{}, std::true_type{});
                // next task of this warp (after the registers of this one are consumed)
                if (q + 1 < my) load(t, task + 8);
                else if (t + 1 < mine) load(t + 1, warp);
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[kFull + sg]);
        }
        // ---------------- accumulator -> out (warps 0-3: one row of the block per thread)
        if (warp < 4) {
            const int r = 32 * warp + lane;
            float *row = out + (size_t)r * 256;
            if (mine > 0) {
                wide_wait(bars, kAcc, ph, timeouts);
                tc_fence_after();
                const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16);
                for (int c0 = 0; c0 < N; c0 += 32) {
                    float d0[16], d1[16];
                    tmem_ld16x2(base + c0, base + c0 + 16, d0, d1);
#pragma unroll
                    for (int q = 0; q < 16; q += 4) {
                        *reinterpret_cast<float4 *>(row + c0 + q) = make_float4(d0[q], d0[q + 1], d0[q + 2], d0[q + 3]);
                        *reinterpret_cast<float4 *>(row + c0 + 16 + q) =
                            make_float4(d1[q], d1[q + 1], d1[q + 2], d1[q + 3]);
                    }
                }
            } else {
                for (int c0 = 0; c0 < N; ++c0) row[c0] = 0.f;
            }
        }
    }
    if (timeouts) atomicAdd(&s_timeouts, timeouts);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 256);
    return s_timeouts;
}

}  // namespace img
