// Work-item tensor-core operators for the wide solver, 64 < p <= 384.
//
// The adjoint out_i = x_i^T B x_i (x_i = [Re a_i; Im a_i], B the real
// embedding of a Hermitian U, Sec. V-B) is split by the ROWS of B into nu
// "units": unit u holds the rows (Re, k) and (Im, k) for k in
// [u ku, (u+1) ku), 2 ku <= 256 rows.  A work item is one (128-pixel tile,
// unit) pair: its accumulator D = X B_u^T (M = 128, N = 2 ku, K = 2 Kp) fits in
// one 256-column region of tensor memory whatever p is, and its epilogue dot
// sum_n x_i[n] D[i][n] runs over the unit's rows only, so the full value is
// the sum of the units' partial dots (taken in unit order by the caller).
// Items of one CTA alternate two accumulator regions, so the epilogue of an
// item overlaps the MMAs of the next.
//
// The X tile of an item comes either from the separable steering tables
// (producer warps, as in tc_wide.cuh) or from a "list image": the cached
// vectors of a pixel list, already scaled, split hi + lo and laid out as
// swizzled K-major tiles in global memory, moved by bulk copies.
//
// The forward K = sum_j w_j c_j c_j^H over a pixel list forms the real Gram
// matrix G = sum_j w_j x_j x_j^T in blocks of 128 x <= 256 features with the
// list index as the MMA's K dimension (both operands MN-major, as in
// tc_wide.cuh): the unweighted side is bulk-copied from the list image, the
// weighted side is produced from the FP32 vectors.
//
// Images in global memory (all blocks 1024-byte aligned):
//   B unit image   block (u, kc) at ((u nk + kc) * 2 rows_u * 128) bytes:
//                  rows_u x 64 columns hi, then lo (rows_u = 2 ku).
//   list image     block (tile, kc) at ((tile nkA + kc) * 32768) bytes:
//                  128 rows x 64 columns hi, then lo; chunks nk .. nkA-1 are
//                  zero (nkA = nk rounded up to even, for the forward's pairs).
#pragma once
#include "tc_wide.cuh"

namespace img {

constexpr int kItemsMaxP = 384;
constexpr size_t kListBlock = (size_t)2 * kTcM * 128;    // one (tile, chunk) block, hi + lo: 32 KB


struct UnitGeom {
    int Kp;     // padded antenna count (multiple of 32)
    int nu;     // units
    int ku;     // antennas per unit (multiple of 16); unit rows = 2 ku <= 256
    int nk;     // 64-column K chunks: 2 Kp / 64
    int nkA;    // chunks per list-image tile (nk rounded up to even)
};

// Smallest unit count with ku = Kp / nu a multiple of 16 and 2 ku <= 256;
// Kp grows by 32 when no split exists (p in (320, 352] uses Kp = 384).
__host__ __device__ inline UnitGeom unit_geom(int p) {
    int Kp = (p + 31) / 32 * 32;
    for (;;) {
        for (int nu = (Kp + 127) / 128; nu <= 8; ++nu) {
            if (Kp % nu == 0 && (Kp / nu) % 16 == 0) {
                const int nk = 2 * Kp / kChunkK;
                return UnitGeom{Kp, nu, Kp / nu, nk, (nk + 1) / 2 * 2};
            }
        }
        Kp += 32;
    }
}
__host__ __device__ inline int unit_rows(const UnitGeom &g) { return 2 * g.ku; }
__host__ __device__ inline size_t unit_block_bytes(const UnitGeom &g) { return (size_t)2 * unit_rows(g) * 128; }
__host__ __device__ inline size_t unit_image_bytes(const UnitGeom &g) {
    return unit_block_bytes(g) * g.nu * g.nk;
}
__host__ __device__ inline size_t list_image_bytes(const UnitGeom &g, int rows) {
    return (size_t)((rows + kTcM - 1) / kTcM) * g.nkA * kListBlock;
}

// Byte offset of 16-byte chunk c16 (0..7) of row r in a swizzled block.
__host__ __device__ inline uint32_t sw_row_off(int r, int c16) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((c16 ^ (r & 7)) << 4));
}

// ---------------------------------------------------------------- B unit image
// One 16-byte chunk (8 K columns) of row n of unit block (u, kc) of the
// embedding of U (p x p column-major FP32 complex, Hermitian):
//   B[(Re, kr), (Re, kc)] = B[(Im, kr), (Im, kc)] = Re U(kc, kr)
//   B[(Re, kr), (Im, kc)] = Im U(kc, kr),  B[(Im, kr), (Re, kc)] = -Im U(kc, kr)
// so that x^T B x = Re(a^H U a) for x = [Re a; Im a].  sc: power-of-two scale.
template <bool BF16>
__device__ inline void unit_image_chunk(const float2 *__restrict__ U, int p, const UnitGeom &g, float sc,
                                        unsigned char *img, int u, int kc, int n, int c16) {
    const int ku = g.ku, rows = unit_rows(g);
    const int rpart = n >= ku, kr = u * ku + n - rpart * ku;
    const int col0 = kc * kChunkK + c16 * 8;
    const int cpart = col0 >= g.Kp, k0 = col0 - cpart * g.Kp;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        float2 w = make_float2(0.f, 0.f);
        if (kr < p && k0 + e < p) w = U[(size_t)kr * p + k0 + e];
        v[e] = sc * ((rpart == cpart) ? w.x : (rpart == 0 ? w.y : -w.y));
    }
    uint4 hi, lo;
    split8<BF16>(v, hi, lo);
    unsigned char *blk = img + (size_t)(u * g.nk + kc) * unit_block_bytes(g);
    const uint32_t off = sw_row_off(n, c16);
    *reinterpret_cast<uint4 *>(blk + off) = hi;
    *reinterpret_cast<uint4 *>(blk + (size_t)rows * 128 + off) = lo;
}

// ---------------------------------------------------------------- list image
// One 16-byte chunk of row r of tile block (t, kc) of the list image of the
// vectors vec[pos[j] * p + k] (j = 128 t + r < n; zero beyond), scaled by sX
// and, when wgt is given, by the row weight wgt[j].
template <bool BF16>
__device__ inline void list_image_chunk(const float2 *__restrict__ vec, const int *__restrict__ pos,
                                        const float *__restrict__ wgt, int n, int p, const UnitGeom &g, float sX,
                                        unsigned char *img, int t, int kc, int r, int c16) {
    const int j = t * kTcM + r;
    const int col0 = kc * kChunkK + c16 * 8;
    const int part = col0 >= g.Kp, k0 = col0 - part * g.Kp;
    float v[8];
    const bool live = j < n && kc < g.nk;
    const float2 *src = live ? vec + (size_t)pos[j] * p : nullptr;
    const float sw = live ? (wgt ? wgt[j] * sX : sX) : 0.f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        float2 w = make_float2(0.f, 0.f);
        if (src && k0 + e < p) w = src[k0 + e];
        v[e] = sw * (part ? w.y : w.x);
    }
    uint4 hi, lo;
    split8<BF16>(v, hi, lo);
    unsigned char *blk = img + (size_t)(t * g.nkA + kc) * kListBlock;
    const uint32_t off = sw_row_off(r, c16);
    *reinterpret_cast<uint4 *>(blk + off) = hi;
    *reinterpret_cast<uint4 *>(blk + (size_t)kTcM * 128 + off) = lo;
}

// ---------------------------------------------------------------- item adjoint
// Shared memory: two X stages (32 KB each), two B stages (64 KB each), then
// 1024 bytes of alignment slack.
__host__ __device__ inline size_t items_smem_bytes() { return 2 * kWideXStage + 2 * kWideBStage + 1024; }

// Items item = first, first + stride, ... < nitems = ntiles nu nkg, with
// t = item % ntiles, u = (item / ntiles) % nu, kg = item / (ntiles nu)
// (unit-major: CTAs working at the same time share a unit's B blocks in L2).
// kg selects the K group: chunks [kg nk / nkg, (kg + 1) nk / nkg) of the
// contraction (nkg divides nk), so a short list still spreads over many
// CTAs; the partial dots of the K groups add up (the dot is linear in D).
// LIST = false: tile t is 2-D steering tile t of the grid (tc_tile_pixel);
// LIST = true:  tile t is rows 128 t .. of the list image Ximg, whose row j
// holds the vector vec[pos[j] * p ..] (j < nrows).
// epi(q, t, r, v) receives, on the epilogue thread of row r, the partial dot
// of unit u and K group kg, q = u nkg + kg (still scaled by the X and B
// scales; a steering tile's scale is steer_scale(p) kLift).  Needs kWideThreads
// threads, kWideBars mbarriers and the 1024-aligned dynamic shared memory of
// items_smem_bytes() - 1024 bytes.  Returns the number of waits that timed out.
// sq (nkg = 1 only): the partial is the unit's sum of squares ||D[r]||^2
// instead of the dot (B from V = L^-1: the whitened MVDR denominator
// ||L^-1 a_i||^2 as the sum of the units' partials, scaled twice).
template <bool BF16, bool LIST, class Epi>
__device__ int items_adjoint(const JobDev &J, const UnitGeom &g, unsigned char *dyn, uint64_t *bars, uint32_t *slot,
                             const unsigned char *Bimg, const unsigned char *Ximg, const float2 *vec, const int *pos,
                             int nrows, int ntiles, int nkg, int first, int stride, bool sq, Epi epi) {
    const int p = J.p, Kp = g.Kp, nk = g.nk, ku = g.ku, rows_u = unit_rows(g);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char *Xs = dyn, *Bs = dyn + 2 * kWideXStage;
    const int nitems = ntiles * g.nu * nkg, nkc = nk / nkg;
    const int mine = first < nitems ? (nitems - 1 - first) / stride + 1 : 0;
    const int total = mine * nkc;                    // chunks
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
    int timeouts = 0;
    auto item_of = [&](int k, int &u, int &t, int &kg) {
        const int it = first + k * stride;
        t = it % ntiles;
        const int r = it / ntiles;
        u = r % g.nu;
        kg = r / g.nu;
    };
    // chunk c of this CTA: its item's unit, tile and global K chunk
    auto chunk_of = [&](int c, int &u, int &t, int &kc) {
        int kg;
        item_of(c / nkc, u, t, kg);
        kc = kg * nkc + c % nkc;
    };

    if (warp == 8) {
        // ---------------- bulk copies and MMAs (lane 0 issues, the warp waits)
        if (total > 0) {
            const bool leader = lane == 0;
            const uint32_t ub = (uint32_t)unit_block_bytes(g);
            const uint32_t xb = LIST ? (uint32_t)kListBlock : 0u;
            const uint32_t idesc = idesc_f16(rows_u, BF16 ? 1 : 0);
            uint32_t ph = 0;
            auto issue_copy = [&](int c, int s) {
                int u, t, kc;
                chunk_of(c, u, t, kc);
                mbar_expect_tx(&bars[kBFull + s], ub + xb);
                tma_bulk_g2s(Bs + s * kWideBStage, Bimg + (size_t)(u * nk + kc) * ub, ub, &bars[kBFull + s]);
                if (LIST)
                    tma_bulk_g2s(Xs + s * kWideXStage, Ximg + (size_t)(t * g.nkA + kc) * kListBlock,
                                 (uint32_t)kListBlock, &bars[kBFull + s]);
            };
            if (leader) issue_copy(0, 0);
            for (int c = 0; c < total; ++c) {
                const int k = c / nkc, jc = c - k * nkc, s = c & 1, rg = k & 1;
                if (!LIST) wide_wait(bars, kXFull + s, ph, timeouts);
                if (jc == 0 && k >= 2) wide_wait(bars, kAEmpty + rg, ph, timeouts);
                wide_wait(bars, kBFull + s, ph, timeouts);
                tc_fence_after();
                if (leader) {
                    const uint32_t xh = smem_u32(Xs + s * kWideXStage), xl = xh + kTcM * 128;
                    const uint32_t bh = smem_u32(Bs + s * kWideBStage), bl = bh + (uint32_t)rows_u * 128;
                    const uint32_t d = tmem + (uint32_t)(rg * 256);
#pragma unroll
                    for (int st = 0; st < kChunkK / 16; ++st) {
                        const uint32_t o = st * 32;
                        mma_f16(d, sw128_desc(xh + o), sw128_desc(bh + o), idesc, (jc > 0 || st > 0) ? 1u : 0u);
                        mma_f16(d, sw128_desc(xh + o), sw128_desc(bl + o), idesc, 1u);
                        mma_f16(d, sw128_desc(xl + o), sw128_desc(bh + o), idesc, 1u);
                    }
                    mma_commit(&bars[kBEmpty + s]);
                    if (!LIST) mma_commit(&bars[kXEmpty + s]);
                    if (jc == nkc - 1) mma_commit(&bars[kAFull + rg]);
                }
                __syncwarp();
                if (c + 1 < total) {
                    // stage s^1 was last read by the MMAs of chunk c - 1
                    const int s1 = s ^ 1;
                    if (c >= 1) wide_wait(bars, kBEmpty + s1, ph, timeouts);
                    if (leader) issue_copy(c + 1, s1);
                }
            }
        }
    } else if (warp >= 4) {
        // ---------------- steering producers (2-D tiles only): chunk c into X
        // stage c & 1.  Warp w fills rows 32w + 8b + a (l offset a, m offset
        // 4w + b), lane j columns 2j, 2j + 1 of the chunk.
        if (!LIST) {
            const int w = warp - 4;
            const bool vec2 = (p & 1) == 0;
            const float2 *__restrict__ El = J.El;
            const float2 *__restrict__ Em = J.Em;
            const int nl = J.n_l, nm = J.n_m, tl = (nl + kTileL - 1) / kTileL;
            const float sX = steer_scale(p) * kLift;
            uint32_t xo[8];
#pragma unroll
            for (int a = 0; a < 8; ++a)
                xo[a] = (uint32_t)(4 * w * 1024 + a * 128 + (((lane >> 2) ^ a) << 4) + (lane & 3) * 4);
            uint32_t ph = 0;
            float2 e[8][2], f[4][2];
            auto load = [&](int c) {
                int u, t, kc;
                chunk_of(c, u, t, kc);
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
                        if (vec2) {
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
                        if (vec2) {
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
                int cu, ct, kc;
                chunk_of(c, cu, ct, kc);
                const int s = c & 1;
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
        }
    } else {
        // ---------------- epilogue: one row per thread, the unit's 2 ku
        // accumulator columns 16 + 16 at a time against the row's vector.
        const int r = 32 * warp + lane;
        const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
        const bool vec2 = (p & 1) == 0;
        uint32_t ph = 0;
        for (int k = 0; k < mine; ++k) {
            int u, t, kg;
            item_of(k, u, t, kg);
            const int rg = k & 1;
            // this row's vector: steering element (E_l row il) * (E_m row im),
            // or the cached vector of list row j
            const float2 *ra = nullptr, *rb = nullptr;
            if (LIST) {
                const int j = t * kTcM + r;
                if (j < nrows) ra = vec + (size_t)pos[j] * p;
            } else {
                const int i = tc_tile_pixel(t, r, J.n_l, J.n_m);
                if (i >= 0) {
                    const int im = i / J.n_l, il = i - im * J.n_l;
                    ra = J.El + (size_t)il * p;
                    rb = J.Em + (size_t)im * p;
                }
            }
            wide_wait(bars, kAFull + rg, ph, timeouts);
            tc_fence_after();
            const uint32_t base = tmem + lane_base + (uint32_t)(rg * 256);
            float acc = 0.f;
            for (int kk = 0; kk < ku; kk += 16) {
                const int k0 = u * ku + kk;
                float ar[16], ai[16];
#pragma unroll
                for (int q = 0; q < 16; q += 2) {
                    float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
                    if (ra && !sq && k0 + q < p) {
                        if (vec2) {
                            const float4 x = __ldg(reinterpret_cast<const float4 *>(ra + k0 + q));
                            a0 = make_float2(x.x, x.y);
                            a1 = make_float2(x.z, x.w);
                            if (!LIST) {
                                const float4 y = __ldg(reinterpret_cast<const float4 *>(rb + k0 + q));
                                a0 = cmul(a0, make_float2(y.x, y.y));
                                a1 = cmul(a1, make_float2(y.z, y.w));
                            }
                        } else {
                            a0 = __ldg(ra + k0 + q);
                            if (!LIST) a0 = cmul(a0, __ldg(rb + k0 + q));
                            if (k0 + q + 1 < p) {
                                a1 = __ldg(ra + k0 + q + 1);
                                if (!LIST) a1 = cmul(a1, __ldg(rb + k0 + q + 1));
                            }
                        }
                    }
                    ar[q] = a0.x;
                    ai[q] = a0.y;
                    ar[q + 1] = a1.x;
                    ai[q + 1] = a1.y;
                }
                float dr[16], di[16];
                tmem_ld16x2(base + kk, base + ku + kk, dr, di);
                if (sq) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) acc = fmaf(dr[q], dr[q], fmaf(di[q], di[q], acc));
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) acc = fmaf(ar[q], dr[q], fmaf(ai[q], di[q], acc));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[kAEmpty + rg]);
            epi(u * nkg + kg, t, r, acc);
        }
    }
    if (timeouts) atomicAdd(&s_timeouts, timeouts);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, 512);
    return s_timeouts;
}

// ---------------------------------------------------------------- list forward
// Gram blocks (m, nb) of G = sum_j w_j x_j x_j^T over a list of n vectors:
// rows = features 128 m .. (chunks 2m, 2m+1 of the list image, unweighted),
// columns = features 256 nb .. (chunks 4 nb .. 4 nb + 3, weighted by w_j,
// produced from the FP32 vectors).  Blocks of 128 x N, N = fwd_n_of(Kp, nb).
__host__ __device__ inline int items_fwd_n(const UnitGeom &g, int nb) {
    const int n = 2 * g.Kp - 256 * nb;
    return n < 256 ? n : 256;
}
// Blocks that reach the upper triangle of G, in a fixed order; pm/pnb may be null.
__host__ __device__ inline int items_fwd_pairs(const UnitGeom &g, int *pm, int *pnb) {
    const int N = 2 * g.Kp, nm = (N + 127) / 128, nnb = (N + 255) / 256;
    int k = 0;
    for (int m = 0; m < nm; ++m)
        for (int nb = 0; nb < nnb; ++nb)
            if (256 * nb + items_fwd_n(g, nb) - 1 >= 128 * m) {
                if (pm) pm[k] = m;
                if (pnb) pnb[k] = nb;
                ++k;
            }
    return k;
}
constexpr int kItemsFwdMaxPairs = 24;

// One CTA: block (m, nb) over list stages s0, s0 + S, ... (64 entries each);
// writes the FP32 block (128 x 256 column-major: entry (r, c) at c 128 + r,
// still scaled by the images' scales) to out.  XA: unweighted list image
// (rows features 128 m ..), XB: weighted list image (columns features
// 256 nb ..); every operand arrives by bulk copy: per stage, chunks 2m, 2m+1
// of XA and 4nb .. 4nb+3 of XB, the 64-row half of the stage's tile, hi and
// lo.  Warp 4 issues the copies and the MMAs, warps 0-3 read the
// accumulator out.  Needs kItemsFwdThreads threads, items_fwd_smem_bytes() of
// dynamic shared memory (1024 aligned by the caller), 5 mbarriers and 256
// columns of tensor memory at tmem, allocated by the caller once per CTA
// (a CTA that gave up its allocation permit cannot allocate again, so one
// allocation serves every task of the CTA).  Returns the waits that timed out.
constexpr int kItemsFwdThreads = 160;
__host__ __device__ inline size_t items_fwd_smem_bytes() { return 2 * kFwdStage + 1024; }

template <bool BF16>
__device__ int items_forward(const UnitGeom &g, unsigned char *dyn, uint64_t *bars, uint32_t tmem,
                             const unsigned char *XA, const unsigned char *XB, int n, int m, int nb, int s0, int S,
                             float *out) {
    const int N = items_fwd_n(g, nb);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nstages = (n + kFwdPix - 1) / kFwdPix;
    const int mine = nstages > s0 ? (nstages - 1 - s0) / S + 1 : 0;
    // B chunks 4nb + q that exist in the image: the last block may be short,
    // and an MMA of N columns reads only its first N / 64 chunks (N / 64 <= nbq)
    const int nbq = min(4, g.nkA - 4 * nb);
    enum { kFull = 0, kEmpty = 2, kAcc = 4 };
    __shared__ int s_timeouts;
    if (threadIdx.x == 0) {
        s_timeouts = 0;
        for (int q = 0; q < 2; ++q) {
            mbar_init(&bars[kFull + q], 1);
            mbar_init(&bars[kEmpty + q], 1);
        }
        mbar_init(&bars[kAcc], 1);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    int timeouts = 0;
    uint32_t ph = 0;

    if (warp == 4) {
        // ---------------- copies and MMAs.  Stage layout: A hi chunks 0, 1
        // (8 KB each), A lo chunks 0, 1, then B hi chunks 0..3, B lo chunks 0..3.
        if (mine > 0) {
            const bool leader = lane == 0;
            const uint32_t idesc = idesc_f16_mn128(N, BF16 ? 1 : 0);
            auto issue_copy = [&](int t, int sg) {
                const int st = s0 + t * S, tile = st >> 1, half = st & 1;
                unsigned char *dst = dyn + sg * kFwdStage;
                mbar_expect_tx(&bars[kFull + sg], (uint32_t)((4 + 2 * nbq) * kFwdChunk));
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const unsigned char *src =
                        XA + (size_t)(tile * g.nkA + 2 * m + q) * kListBlock + (size_t)half * kFwdChunk;
                    tma_bulk_g2s(dst + q * kFwdChunk, src, (uint32_t)kFwdChunk, &bars[kFull + sg]);
                    tma_bulk_g2s(dst + (2 + q) * kFwdChunk, src + (size_t)kTcM * 128, (uint32_t)kFwdChunk,
                                 &bars[kFull + sg]);
                }
                for (int q = 0; q < nbq; ++q) {
                    const unsigned char *src =
                        XB + (size_t)(tile * g.nkA + 4 * nb + q) * kListBlock + (size_t)half * kFwdChunk;
                    tma_bulk_g2s(dst + (4 + q) * kFwdChunk, src, (uint32_t)kFwdChunk, &bars[kFull + sg]);
                    tma_bulk_g2s(dst + (8 + q) * kFwdChunk, src + (size_t)kTcM * 128, (uint32_t)kFwdChunk,
                                 &bars[kFull + sg]);
                }
            };
            if (leader) issue_copy(0, 0);
            for (int t = 0; t < mine; ++t) {
                const int sg = t & 1;
                wide_wait(bars, kFull + sg, ph, timeouts);
                tc_fence_after();
                if (leader) {
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
                __syncwarp();
                if (t + 1 < mine) {
                    const int s1 = sg ^ 1;
                    if (t >= 1) wide_wait(bars, kEmpty + s1, ph, timeouts);
                    if (leader) issue_copy(t + 1, s1);
                }
            }
        }
    }
    if (warp < 4) {
        // ---------------- accumulator -> out: lanes hold consecutive rows, so
        // each column's 32 rows are one 128-byte store
        const int r = 32 * warp + lane;
        float *col = out + r;
        if (mine > 0) {
            wide_wait(bars, kAcc, ph, timeouts);
            tc_fence_after();
            const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16);
            for (int c0 = 0; c0 < N; c0 += 32) {
                float d0[16], d1[16];
                tmem_ld16x2(base + c0, base + c0 + 16, d0, d1);
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    col[(size_t)(c0 + q) * kTcM] = d0[q];
                    col[(size_t)(c0 + 16 + q) * kTcM] = d1[q];
                }
            }
        } else {
            for (int c0 = 0; c0 < N; ++c0) col[(size_t)c0 * kTcM] = 0.f;
        }
    }
    if (timeouts) atomicAdd(&s_timeouts, timeouts);
    tc_fence_before();
    __syncthreads();
    return s_timeouts;
}

}  // namespace img
