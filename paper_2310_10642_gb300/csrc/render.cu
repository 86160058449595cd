// render.cu -- tile-based front-to-back compositing (Eq. 6) and its adjoint.
//
// One thread block of 256 threads per compositing tile (16x16 or 32x32
// pixels).  It walks the depth-ordered splat list of the binning tile that
// contains it (the same tile, or a 2x2 / 4x4 group of compositing tiles).
// With 16x16 tiles each thread owns one pixel; with 32x32 tiles each thread
// owns four, which amortises a splat's shared-memory reads over them.  Each
// warp owns a compact region of the tile (8x4 pixels, resp. 16x8 in four 8x4
// sub-regions).  The list is walked in batches of up to 256: each thread
// stages one splat record into shared memory together with a mask of the
// tile's 8x4 sub-regions the splat can reach (its support box, narrowed by
// its support ellipse); each warp then ballots over the masks of 32 slots at
// a time and visits, in list order, only the splats that reach one of its
// own sub-regions.  The forward stops a block as soon as all its pixels have
// terminated (__syncthreads_count); the adjoint double-buffers its batches.
//
// Per pixel and splat (readings R4-R6):
//   power = -1/2 (a dx^2 + c dy^2) - b dx dy, dx = x - u, dy = y - v
//   skip if power > 0; alpha = min(alpha_max, alpha_eff * exp(power));
//   skip if alpha < alpha_min; stop (splat excluded) if T (1 - alpha) < T_min;
//   C += c alpha T; T *= 1 - alpha.  Finally C += T bg.
// alpha_eff = sigmoid(logit) p(t) carries the marginal of Eq. 6.  Outside the
// support box |dx| <= hx, |dy| <= hy of a splat alpha < alpha_min holds by
// construction (the box bounds the ellipse alpha_eff G >= alpha_min with half
// a pixel to spare), so skipping a region that lies entirely outside the box
// takes the same decision the per-pixel test would.
//
// The exponent is evaluated as exp2 of a quadratic form pre-scaled by log2(e)
// (the conic, or with 16-bit records its Cholesky factor), with explicitly
// rounded operations, so the forward and the adjoint take bit-identical skip
// decisions.
#include "fgs4d_internal.cuh"

namespace fgs4d {

__device__ __forceinline__ int find_view(const ViewSet& VS, uint32_t tile) {
    int lo = 0, hi = VS.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (VS.v[mid].tile_base <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Thread block b composites one TS x TS tile of the binning tile it walks
// the list of: binning tiles of side O.bin hold (O.bin / TS)^2 compositing
// tiles, whose blocks are consecutive (they share the list's records in
// L2).  Sets the binning tile, the view and the pixel origin (x0, y0) of
// the block's tile; false when that tile lies outside the view.
template <int TS>
__device__ __forceinline__ bool block_tile(const ViewSet& VS, const DevOpts& O, uint32_t& tile, int& v, int& x0,
                                           int& y0) {
    const int fsh = __ffs(O.bin / TS) - 1;  // log2 of compositing tiles per binning tile side
    tile = blockIdx.x >> (2 * fsh);
    const uint32_t q = blockIdx.x & ((1u << (2 * fsh)) - 1u);
    v = find_view(VS, tile);
    const DevView& V = VS.v[v];
    const uint32_t local = tile - V.tile_base;
    const int ty = (int)(local / (uint32_t)V.tiles_x), tx = (int)local - ty * V.tiles_x;
    x0 = tx * O.bin + (int)(q & ((1u << fsh) - 1u)) * TS;
    y0 = ty * O.bin + (int)(q >> fsh) * TS;
    return x0 < V.width && y0 < V.height;
}

// How a staged splat evaluates log2 of its Gaussian factor at (dx, dy) from
// three staged coefficients (X, Y, Z).
template <class Rec>
struct Form;
template <>
struct Form<SplatRecord> {  // conic pre-scaled: X = -log2e/2 a, Y = -log2e b, Z = -log2e/2 c
    // power2 can round to a positive value: pixels with power2 > 0 are skipped
    static constexpr bool kNeverPositive = false;
    __device__ __forceinline__ static void stage(const SplatView& r, float& X, float& Y, float& Z) {
        X = __fmul_rn(-0.5f * kLog2e, r.a);
        Y = __fmul_rn(-kLog2e, r.b);
        Z = __fmul_rn(-0.5f * kLog2e, r.c);
    }
    __device__ __forceinline__ static float power2(float X, float Y, float Z, float dx, float dy) {
        return __fmaf_rn(__fmul_rn(X, dx), dx, __fmaf_rn(__fmul_rn(Z, dy), dy, __fmul_rn(__fmul_rn(Y, dx), dy)));
    }
    // power2 split into a part of dx (one per pixel column of a lane) and a
    // part of dy (one per pixel row), each computed once per visit;
    // combine(col(dx), row(dy)) equals power2(X, Y, Z, dx, dy) bit for bit.
    struct Col {
        float dx, xdx, ydx;
    };
    struct Row {
        float dy, zdy;
    };
    __device__ __forceinline__ static Col col(float X, float Y, float dx) {
        return Col{dx, __fmul_rn(X, dx), __fmul_rn(Y, dx)};
    }
    __device__ __forceinline__ static Row row(float Y, float Z, float dy) { return Row{dy, __fmul_rn(Z, dy)}; }
    __device__ __forceinline__ static float combine(float X, const Col& c, const Row& r) {
        return __fmaf_rn(c.xdx, c.dx, __fmaf_rn(r.zdy, r.dy, __fmul_rn(c.ydx, r.dy)));
    }
};
template <>
struct Form<SplatRecordH> {  // Cholesky factor pre-scaled by kappa, kappa^2 = log2(e) / 2
    static constexpr float kKappa = 0.8493218002880191f;
    // power2 is a negated sum of squares: never positive, NaN only from non-finite inputs
    static constexpr bool kNeverPositive = true;
    __device__ __forceinline__ static void stage(const SplatView& r, float& X, float& Y, float& Z) {
        X = __fmul_rn(kKappa, r.l11);
        Y = __fmul_rn(kKappa, r.l21);
        Z = __fmul_rn(kKappa, r.l22);
    }
    __device__ __forceinline__ static float power2(float X, float Y, float Z, float dx, float dy) {
        const float t1 = __fmaf_rn(X, dx, __fmul_rn(Y, dy));
        const float t2 = __fmul_rn(Z, dy);
        return -__fmaf_rn(t1, t1, __fmul_rn(t2, t2));
    }
    // as for Form<SplatRecord>: combine(col(dx), row(dy)) equals power2 bit for bit
    struct Col {
        float dx;
    };
    struct Row {
        float ydy, t22;  // Y dy and (Z dy)^2
    };
    __device__ __forceinline__ static Col col(float X, float Y, float dx) { return Col{dx}; }
    __device__ __forceinline__ static Row row(float Y, float Z, float dy) {
        const float t2 = __fmul_rn(Z, dy);
        return Row{__fmul_rn(Y, dy), __fmul_rn(t2, t2)};
    }
    __device__ __forceinline__ static float combine(float X, const Col& c, const Row& r) {
        const float t1 = __fmaf_rn(X, c.dx, r.ydy);
        return -__fmaf_rn(t1, t1, r.t22);
    }
};

// min(a, b) that returns NaN when b is NaN (fminf would return a): the alpha
// clamp with it and the test alpha >= alpha_min reject a NaN power2 without
// a test of its own.
__device__ __forceinline__ float min_nan(float a, float b) {
    float r;
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// Shared-memory form of a record: a = (u, v, X, Y), b = (Z, alpha_eff, R, G),
// c = (B, hx, hy, 0), with (X, Y, Z) as Form<Rec> stages them.
template <class Rec>
__device__ __forceinline__ void stage_record(const SplatView& r, float4& sa, float4& sb, float4& sc) {
    float X, Y, Z;
    Form<Rec>::stage(r, X, Y, Z);
    sa = make_float4(r.u, r.v, X, Y);
    sb = make_float4(Z, r.alpha_eff, r.R, r.G);
    sc = make_float4(r.B, r.hx, r.hy, 0.0f);
}

// Pixel layout of a TS x TS tile: warp w owns a region of RW x RH pixels
// (2 regions across, 4 down).  With 32x32 tiles the region is 16x8 and splits
// into four 8x4 sub-regions (k = 0..3: left/right, top/bottom); lane l owns
// pixel (l & 7, l >> 3) of each, so that pixel k of every lane lies in
// sub-region k and a splat whose box misses a sub-region skips that pixel
// for the whole warp at once.  With 16x16 tiles the 8x4 region is the
// lane's only pixel.
template <int TS>
struct TilePixels {
    static constexpr int P = TS * TS / kTilePix;  // pixels per thread: 1 or 4
    static constexpr int RW = TS / 2, RH = TS / 4;
    __device__ __forceinline__ static void region(int tid, int x0, int y0, int& rx, int& ry) {
        const int w = tid >> 5;
        rx = x0 + (w & 1) * RW;
        ry = y0 + (w >> 1) * RH;
    }
    __device__ __forceinline__ static void coords(int tid, int x0, int y0, int k, int& px, int& py) {
        int rx, ry;
        region(tid, x0, y0, rx, ry);
        const int l = tid & 31;
        px = rx + (l & 7) + (P == 4 ? (k & 1) * 8 : 0);
        py = ry + (l >> 3) + (P == 4 ? (k >> 1) * 4 : 0);
    }
    // offset of pixel k from pixel 0 (exact in float)
    __device__ __forceinline__ static constexpr float off_x(int k) { return P == 4 ? (float)((k & 1) * 8) : 0.0f; }
    __device__ __forceinline__ static constexpr float off_y(int k) { return P == 4 ? (float)((k >> 1) * 4) : 0.0f; }
    // Sub-regions of the tile: NC = TS/8 columns of 8 pixels, NR = TS/4 rows
    // of 4.  Sub-region (c, r) is sub-region k of warp w with
    // bit(c, r) = w * P + k; warp w's P bits are its sub-regions 0..P-1.
    static constexpr int NC = TS / 8, NR = TS / 4;
    static constexpr int kSubAll = (1 << P) - 1;
    __device__ __forceinline__ static constexpr int col_bit(int c) { return (c / (NC / 2)) * P + c % (NC / 2); }
    __device__ __forceinline__ static constexpr int row_shift(int r) {
        return (r / (NR / 4)) * 2 * P + (r % (NR / 4)) * (NC / 2);
    }
    // Bit bit(c, r) set when the support box [u - hx, u + hx] x [v - hy, v + hy]
    // reaches the pixel centres of sub-region (c, r) of the tile whose corner
    // pixel is (x0, y0).  Evaluated once per staged splat; every warp then
    // visits only the splats with one of its own bits set.  Outside the box
    // alpha < alpha_min, so a pixel of a sub-region without its bit would not
    // have been blended.
    __device__ __forceinline__ static uint32_t sub_masks(float u, float v, float hx, float hy, float x0, float y0) {
        const float xl = u - hx, xr = u + hx, yt = v - hy, yb = v + hy;
        uint32_t row = 0;
#pragma unroll
        for (int c = 0; c < NC; c++)
            if (xr >= x0 + (float)(8 * c) && xl <= x0 + (float)(8 * c + 7)) row |= 1u << col_bit(c);
        uint32_t m = 0;
#pragma unroll
        for (int r = 0; r < NR; r++)
            if (yb >= y0 + (float)(4 * r) && yt <= y0 + (float)(4 * r + 3)) m |= row << row_shift(r);
        return m;
    }
    // The bits of `box` (sub_masks) whose sub-region the support ellipse
    // reaches: per band of 4 pixel rows, the columns the ellipse spans over
    // those rows (the conservative spans the binning takes per tile row,
    // taken here per band), for the tile with corner pixel (x0, y0).
    __device__ __forceinline__ static uint32_t ellipse_masks(uint32_t box, const EllipseRows& e, const DevView& V,
                                                             int x0, int y0) {
        uint32_t all = 0;
#pragma unroll
        for (int c = 0; c < NC; c++) all |= 1u << col_bit(c);
        uint32_t m = 0;
#pragma unroll
        for (int r = 0; r < NR; r++) {
            if (!((box >> row_shift(r)) & all)) continue;  // the box misses the band (or the band the image)
            const int ry = y0 + 4 * r;
            float px0, px1;
            if (!ellipse_row_span(e, V, (float)ry, (float)min(ry + 3, V.height - 1), &px0, &px1)) continue;
            const int c0 = max(((int)px0 - x0) >> 3, 0), c1 = min(((int)px1 - x0) >> 3, NC - 1);
            uint32_t row = 0;
#pragma unroll
            for (int c = 0; c < NC; c++)
                if (c >= c0 && c <= c1) row |= 1u << col_bit(c);
            m |= row << row_shift(r);
        }
        return box & m;
    }
    // Sub-region mask of a staged splat: box test, narrowed by the ellipse.
    __device__ __forceinline__ static uint32_t splat_mask(const SplatView& r, float ln_alpha_min, const DevView& V,
                                                          int x0, int y0) {
        const uint32_t box = sub_masks(r.u, r.v, r.hx, r.hy, (float)x0, (float)y0);
        if (!box) return 0u;
        const EllipseRows e = ellipse_rows(r, ln_alpha_min);
        return e.exact ? ellipse_masks(box, e, V, x0, y0) : box;
    }
};

__device__ __forceinline__ unsigned long long warp_sum_u64(uint32_t x) {
    unsigned long long v = x;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// kMode 0: the compositing of Eq. 6 (image, final T, n_last).
// kMode 1: the same, and it accumulates into stats[0..3] the work the walk
// did: (pixel, splat) pairs with the pixel inside the splat's support box and
// not yet stopped, the pairs blended into the pixel, the sum of n_last, and
// the pairs this kernel evaluated (pixel not stopped, its sub-region reached).
// kMode 2: the same walk compositing each splat's aux record (depth, flow u,
// flow v) instead of its colour, background 0, into aux_image only.
template <int TS, class Rec, int kMode>
__global__ void __launch_bounds__(kTilePix, 4) render_fwd_kernel(const __grid_constant__ ViewSet VS, const DevOpts O,
                                                              const uint2* __restrict__ ranges,
                                                              const uint32_t* __restrict__ pair_vals,
                                                              const Rec* __restrict__ rec, uint32_t n_splats,
                                                              float* __restrict__ image, float* __restrict__ final_T,
                                                              int32_t* __restrict__ n_last,
                                                              unsigned long long* __restrict__ stats,
                                                              const float4* __restrict__ aux_rec,
                                                              float* __restrict__ aux_image) {
    using TP = TilePixels<TS>;
    constexpr int P = TP::P;
    constexpr bool kStats = kMode == 1, kAux = kMode == 2;
    __shared__ float4 s_a[kTilePix];
    __shared__ float4 s_b[kTilePix];
    __shared__ float4 s_c[kTilePix];
    __shared__ float4 s_x[kAux ? kTilePix : 1];
    __shared__ uint32_t s_m[kTilePix];  // sub-region mask of each staged splat
    const int tid = threadIdx.x, lane = tid & 31, wshift = (tid >> 5) * P;
    const unsigned F = 0xffffffffu;
    uint32_t tile;
    int v, x0, y0;
    if (!block_tile<TS>(VS, O, tile, v, x0, y0)) return;  // the whole block lies outside the view
    const DevView& V = VS.v[v];
    const uint2 range = ranges[tile];
    float T[P], C0[P], C1[P], C2[P];
    int32_t last[P];
    // bit k of `inside`: pixel k lies in the image; of `live`: it has not stopped
    uint32_t inside = 0;
    uint32_t st_box = 0, st_blend = 0, st_eval = 0;
    int bpx, bpy;  // pixel 0 of this thread; pixel k lies at a constant offset
    TP::coords(tid, x0, y0, 0, bpx, bpy);
    const float fbx = (float)bpx, fby = (float)bpy;
#pragma unroll
    for (int k = 0; k < P; k++) {
        int px, py;
        TP::coords(tid, x0, y0, k, px, py);
        if (px < V.width && py < V.height) inside |= 1u << k;
        T[k] = 1.0f;
        C0[k] = C1[k] = C2[k] = 0.0f;
        last[k] = 0;
    }
    uint32_t live = inside;
    const int B = O.batch;  // records per batch, <= kTilePix
    for (uint32_t base = range.x; base < range.y; base += (uint32_t)B) {
        if (__syncthreads_count(live == 0u) == kTilePix) break;
        const uint32_t idx = base + tid;
        if (tid < B && idx < range.y) {
            const uint32_t sid = pair_vals[idx];
            if (sid < n_splats) {
                const SplatView r = decode_record(rec[sid], O.ln_alpha_min);
                stage_record<Rec>(r, s_a[tid], s_b[tid], s_c[tid]);
                s_m[tid] = TP::splat_mask(r, O.ln_alpha_min, V, x0, y0);
                if constexpr (kAux) s_x[tid] = aux_rec[sid];
            } else {  // never produced by bin_sort; an empty splat keeps the access in bounds
                s_m[tid] = 0u;
            }
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)B, range.y - base);
        // The warp walks the batch 32 slots at a time; a ballot picks the
        // slots whose splat reaches one of its sub-regions, visited in order.
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            if (__all_sync(F, live == 0u)) break;
            const int jl = c0 + lane;
            const uint32_t nib = jl < cnt ? (s_m[jl] >> wshift) & (uint32_t)TP::kSubAll : 0u;
            uint32_t hits = __ballot_sync(F, nib != 0u);
            while (hits) {
                const int l = __ffs(hits) - 1;
                hits &= hits - 1u;
                const unsigned sub = __shfl_sync(F, nib, l);
                const int j = c0 + l;
                const float4 a = s_a[j];
                const float4 b = s_b[j];
                const float4 c = s_c[j];
                const int32_t pos1 = (int32_t)(base - range.x) + j + 1;
                const uint32_t act = sub & live;
                // the lane's pixels share two columns and two rows (one each with
                // 16x16 tiles): their parts of the quadratic form, once per visit
                const auto col0 = Form<Rec>::col(a.z, a.w, __fsub_rn(fbx, a.x));
                const auto row0 = Form<Rec>::row(a.w, b.x, __fsub_rn(fby, a.y));
                const auto col1 = Form<Rec>::col(a.z, a.w, __fsub_rn(fbx + TP::off_x(1), a.x));
                const auto row1 = Form<Rec>::row(a.w, b.x, __fsub_rn(fby + TP::off_y(2), a.y));
#pragma unroll
                for (int k = 0; k < P; k++) {
                    if (!(act >> k & 1u)) continue;
                    if (kStats) {
                        const float dx = __fsub_rn(fbx + TP::off_x(k), a.x), dy = __fsub_rn(fby + TP::off_y(k), a.y);
                        st_eval++;
                        st_box += (fabsf(dx) <= c.y && fabsf(dy) <= c.z);
                    }
                    const float p2 = Form<Rec>::combine(a.z, (k & 1) ? col1 : col0, (k >> 1) ? row1 : row0);
                    if (!Form<Rec>::kNeverPositive && !(p2 <= 0.0f)) continue;
                    const float araw = __fmul_rn(b.y, ex2_approx(p2));
                    const float alpha = min_nan(O.alpha_max, araw);
                    if (!(alpha >= O.alpha_min)) continue;  // also a NaN power2
                    const float Tn = T[k] * (1.0f - alpha);
                    if (Tn < O.T_min) {
                        live &= ~(1u << k);
                        continue;
                    }
                    if (kStats) st_blend++;
                    const float w = alpha * T[k];
                    if constexpr (kAux) {
                        const float4 x = s_x[j];
                        C0[k] = fmaf(x.x, w, C0[k]);
                        C1[k] = fmaf(x.y, w, C1[k]);
                        C2[k] = fmaf(x.z, w, C2[k]);
                    } else {
                        C0[k] = fmaf(b.z, w, C0[k]);
                        C1[k] = fmaf(b.w, w, C1[k]);
                        C2[k] = fmaf(c.x, w, C2[k]);
                    }
                    T[k] = Tn;
                    last[k] = pos1;
                }
                // a pixel stopped: the warp is done once all of its pixels have
                if (__any_sync(F, act & ~live) && __all_sync(F, live == 0u)) hits = 0u;
            }
        }
    }
    const size_t npix = (size_t)V.width * V.height;
#pragma unroll
    for (int k = 0; k < P; k++) {
        if (!(inside >> k & 1u)) continue;
        const size_t p = (size_t)(bpy + (int)TP::off_y(k)) * V.width + (size_t)(bpx + (int)TP::off_x(k));
        if constexpr (kAux) {
            float* ax = aux_image + 3 * (size_t)V.pix_base;
            ax[p] = C0[k];
            ax[npix + p] = C1[k];
            ax[2 * npix + p] = C2[k];
            continue;
        }
        float* img = image + 3 * (size_t)V.pix_base;
        img[p] = fmaf(T[k], V.bg[0], C0[k]);
        img[npix + p] = fmaf(T[k], V.bg[1], C1[k]);
        img[2 * npix + p] = fmaf(T[k], V.bg[2], C2[k]);
        final_T[V.pix_base + p] = T[k];
        n_last[V.pix_base + p] = last[k];
    }
    if (kStats) {
        uint32_t walked = 0;
#pragma unroll
        for (int k = 0; k < P; k++) walked += (uint32_t)last[k];
        const unsigned long long w_box = warp_sum_u64(st_box), w_blend = warp_sum_u64(st_blend),
                                 w_walk = warp_sum_u64(walked), w_eval = warp_sum_u64(st_eval);
        if ((tid & 31) == 0) {
            atomicAdd(stats + 0, w_box);
            atomicAdd(stats + 1, w_blend);
            atomicAdd(stats + 2, w_walk);
            atomicAdd(stats + 3, w_eval);
        }
    }
}

// (rcp_approx, 1/x to within about one ulp: recovering T back to front
// through ~10^2..10^3 of these stays within ~1e-4 relative.)

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Reduce-scatter of eight per-lane values over the warp with 4+2+1+1+1
// shuffles: afterwards lane l holds the warp total of value (l >> 2) & 7.
__device__ __forceinline__ float warp_reduce8(const float (&v)[8], int lane) {
    const unsigned F = 0xffffffffu;
    const bool h4 = lane & 16, h3 = lane & 8, h2 = lane & 4;
    float a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; i++) a[i] = (h4 ? v[i + 4] : v[i]) + __shfl_xor_sync(F, h4 ? v[i] : v[i + 4], 16);
#pragma unroll
    for (int i = 0; i < 2; i++) b[i] = (h3 ? a[i + 2] : a[i]) + __shfl_xor_sync(F, h3 ? a[i] : a[i + 2], 8);
    float c = (h2 ? b[1] : b[0]) + __shfl_xor_sync(F, h2 ? b[0] : b[1], 4);
    c += __shfl_xor_sync(F, c, 2);
    c += __shfl_xor_sync(F, c, 1);
    return c;
}

constexpr int kGradStride = 12;  // floats per staged splat in the shared gradient accumulator

// One staged batch of the adjoint: records, sub-region masks, splat ids and
// the per-splat gradient sums of the block.
struct BwdStage {
    float4 a[kTilePix];
    float4 b[kTilePix];
    float4 n[kTilePix];  // natural conic (a, b, c) for the flush, and the colour's B
    uint32_t m[kTilePix];
    uint32_t sid[kTilePix];
    float g[kTilePix * kGradStride];
};
constexpr size_t kBwdSmem = 2 * sizeof(BwdStage);  // double-buffered: 53,248 bytes (dynamic)

template <int TS, class Rec>
__global__ void __launch_bounds__(kTilePix, 4) render_bwd_kernel(
    const __grid_constant__ ViewSet VS, const DevOpts O, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ pair_vals, const Rec* __restrict__ rec, uint32_t n_splats,
    const float* __restrict__ final_T, const int32_t* __restrict__ n_last, const float* __restrict__ dL_dimage,
    float4* __restrict__ grad2d) {
    using TP = TilePixels<TS>;
    constexpr int P = TP::P;
    // Two staging buffers: while the warps walk batch k in one, each thread
    // flushes its slot of batch k - 1 and stages its slot of batch k + 1 in
    // the other, so one barrier per batch separates the batches.
    extern __shared__ __align__(16) unsigned char s_dyn[];
    BwdStage* S = reinterpret_cast<BwdStage*>(s_dyn);
    __shared__ int s_max;
    const int tid = threadIdx.x, lane = tid & 31, wshift = (tid >> 5) * P;
    const unsigned F = 0xffffffffu;
    uint32_t tile;
    int v, x0, y0;
    if (!block_tile<TS>(VS, O, tile, v, x0, y0)) return;  // the whole block lies outside the view
    const DevView& V = VS.v[v];
    const uint2 range = ranges[tile];
    const size_t npix = (size_t)V.width * V.height;
    const float* gimg = dL_dimage + 3 * (size_t)V.pix_base;
    // Per pixel: T (recovered back to front), dL/dC, and S = dL/dC . acc where
    // acc = sum_{j > i} c_j alpha_j T_j + T_final bg is built back to front, so
    // that dL/dalpha_i = T_i (dL/dC . c_i) - S / (1 - alpha_i).
    float T[P], dC0[P], dC1[P], dC2[P], Sacc[P];
    int32_t last[P];
    int my_max = 0;
    int bpx, bpy;  // pixel 0 of this thread; pixel k lies at a constant offset
    TP::coords(tid, x0, y0, 0, bpx, bpy);
    const float fbx = (float)bpx, fby = (float)bpy;
#pragma unroll
    for (int k = 0; k < P; k++) {
        int px, py;
        TP::coords(tid, x0, y0, k, px, py);
        T[k] = 1.0f;
        dC0[k] = dC1[k] = dC2[k] = 0.0f;
        last[k] = 0;
        if (px < V.width && py < V.height) {
            const size_t p = (size_t)py * V.width + px;
            T[k] = final_T[V.pix_base + p];
            last[k] = n_last[V.pix_base + p];
            dC0[k] = gimg[p];
            dC1[k] = gimg[npix + p];
            dC2[k] = gimg[2 * npix + p];
        }
        Sacc[k] = T[k] * (dC0[k] * V.bg[0] + dC1[k] * V.bg[1] + dC2[k] * V.bg[2]);
        my_max = max(my_max, last[k]);
    }
    const int warp_last = __reduce_max_sync(0xffffffffu, my_max);  // positions >= this: nothing in this warp
    if (tid == 0) s_max = 0;
#pragma unroll
    for (int k = 0; k < kGradStride; k++) {
        S[0].g[tid * kGradStride + k] = 0.0f;
        S[1].g[tid * kGradStride + k] = 0.0f;
    }
    __syncthreads();
    if (lane == 0) atomicMax(&s_max, warp_last);
    __syncthreads();
    const int max_last = min(s_max, (int)(range.y - range.x));
    const int B = O.batch;  // records per batch, <= kTilePix
    const int nb = (max_last + B - 1) / B;
    // batch bi covers list positions [end - cnt, end), end = max_last - bi B, in slot order back to front
    auto stage = [&](int bi, BwdStage& st) {
        const int end = max_last - bi * B, cnt = min(end, B);
        if (tid < cnt) {
            const uint32_t idx = range.x + (uint32_t)(end - 1 - tid);
            uint32_t sid = pair_vals[idx];
            if (sid >= n_splats) sid = 0;  // never produced by bin_sort; keeps the access in bounds
            const SplatView r = decode_record(rec[sid], O.ln_alpha_min);
            float4 sc;
            stage_record<Rec>(r, st.a[tid], st.b[tid], sc);
            st.n[tid] = make_float4(r.a, r.b, r.c, sc.x);
            st.m[tid] = TP::splat_mask(r, O.ln_alpha_min, V, x0, y0);
            st.sid[tid] = sid;
        }
    };
    auto flush = [&](int bi, BwdStage& st) {
        const int end = max_last - bi * B, cnt = min(end, B);
        if (tid < cnt) {
            float4* sg = reinterpret_cast<float4*>(&st.g[tid * kGradStride]);
            const float4 m0 = sg[0];
            float4 q1 = sg[1];
            const float q2 = st.g[tid * kGradStride + 8];
            // power = -1/2 (a dx^2 + 2 b dx dy + c dy^2), dx = x - u, dy = y - v
            const float4 nc = st.n[tid];
            const float4 q0 = make_float4(fmaf(nc.x, m0.x, nc.y * m0.y), fmaf(nc.y, m0.x, nc.z * m0.y), -0.5f * m0.z,
                                          -m0.w);
            q1.x = -0.5f * q1.x;
            if (q0.x != 0.f || q0.y != 0.f || q0.z != 0.f || q0.w != 0.f || q1.x != 0.f || q1.y != 0.f ||
                q1.z != 0.f || q1.w != 0.f || q2 != 0.f) {
                float4* dst = grad2d + 3 * (size_t)st.sid[tid];
                atomicAdd(dst + 0, q0);
                atomicAdd(dst + 1, q1);
                atomicAdd(reinterpret_cast<float*>(dst + 2), q2);
            }
            sg[0] = make_float4(0.f, 0.f, 0.f, 0.f);
            sg[1] = make_float4(0.f, 0.f, 0.f, 0.f);
            st.g[tid * kGradStride + 8] = 0.0f;
        }
    };
    if (nb > 0) stage(0, S[0]);
    __syncthreads();
    for (int bi = 0; bi < nb; bi++) {
        BwdStage& cur = S[bi & 1];
        BwdStage& nxt = S[(bi & 1) ^ 1];
        // the other buffer holds batch bi - 1, which every warp finished before the last barrier
        if (bi > 0) flush(bi - 1, nxt);
        if (bi + 1 < nb) stage(bi + 1, nxt);
        const int end = max_last - bi * B, cnt = min(end, B);
        // a reduced visit waiting for a second one to share its last reduction and atomic
        int pend_j = -1;
        float pend_tot = 0.0f, pend_9 = 0.0f;
        // The warp walks the batch 32 slots at a time (back to front); a
        // ballot picks the slots whose splat reaches one of its sub-regions
        // and lies in front of the warp's last blended position.
        for (int c0 = 0; c0 < cnt; c0 += 32) {
            const int jl = c0 + lane;
            const uint32_t nib =
                (jl < cnt && end - 1 - jl < warp_last) ? (cur.m[jl] >> wshift) & (uint32_t)TP::kSubAll : 0u;
            uint32_t hits = __ballot_sync(F, nib != 0u);
            while (hits) {
                const int l = __ffs(hits) - 1;
                hits &= hits - 1u;
                const unsigned sub = __shfl_sync(F, nib, l);
                const int j = c0 + l;
                const int pos = end - 1 - j;  // 0-based position in the tile list
                const float4 a = cur.a[j];
                const float4 b = cur.b[j];
                const float cB = cur.n[j].w;
                // sums over the warp's pixels, with g = dL/dpower:
                //   g dx, g dy, g dx^2, g dx dy, g dy^2, dL/dalpha_eff, dL/dR, dL/dG (and dL/dB);
                // the flush turns the first five into dL/d(u, v, a, b, c) with the splat's conic
                float gv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                float g_bl = 0.0f;
                bool contrib = false;
                // the Gaussian factor of every pixel first (independent chains), -1 where
                // the pixel takes no part; then the adjoint updates in order
                float Gv[P];
                const auto col0 = Form<Rec>::col(a.z, a.w, __fsub_rn(fbx, a.x));
                const auto row0 = Form<Rec>::row(a.w, b.x, __fsub_rn(fby, a.y));
                const auto col1 = Form<Rec>::col(a.z, a.w, __fsub_rn(fbx + TP::off_x(1), a.x));
                const auto row1 = Form<Rec>::row(a.w, b.x, __fsub_rn(fby + TP::off_y(2), a.y));
#pragma unroll
                for (int k = 0; k < P; k++) {
                    const float p2 = Form<Rec>::combine(a.z, (k & 1) ? col1 : col0, (k >> 1) ? row1 : row0);
                    const float G = ex2_approx(p2);
                    const bool on = (sub >> k & 1u) && pos < last[k] && (Form<Rec>::kNeverPositive || p2 <= 0.0f) &&
                                    min_nan(O.alpha_max, __fmul_rn(b.y, G)) >= O.alpha_min;
                    Gv[k] = on ? G : -1.0f;
                }
#pragma unroll
                for (int k = 0; k < P; k++) {
                    const float G = Gv[k];
                    if (G < 0.0f) continue;
                    const float dx = __fsub_rn(fbx + TP::off_x(k), a.x), dy = __fsub_rn(fby + TP::off_y(k), a.y);
                    const float araw = __fmul_rn(b.y, G);
                    const float alpha = fminf(O.alpha_max, araw);
                    contrib = true;
                    const float inv_om = rcp_approx(1.0f - alpha);
                    const float Ti = T[k] * inv_om;  // transmittance before this splat
                    const float dCc = fmaf(dC0[k], b.z, fmaf(dC1[k], b.w, dC2[k] * cB));
                    const float dalpha = fmaf(Ti, dCc, -Sacc[k] * inv_om);
                    const float w = alpha * Ti;
                    gv[6] = fmaf(dC0[k], w, gv[6]);
                    gv[7] = fmaf(dC1[k], w, gv[7]);
                    g_bl = fmaf(dC2[k], w, g_bl);
                    Sacc[k] = fmaf(w, dCc, Sacc[k]);
                    T[k] = Ti;
                    if (!(araw > O.alpha_max)) {
                        gv[5] = fmaf(dalpha, G, gv[5]);
                        const float dpow = dalpha * araw;
                        const float hx = dpow * dx, hy = dpow * dy;
                        gv[0] += hx;
                        gv[1] += hy;
                        gv[2] = fmaf(hx, dx, gv[2]);
                        gv[3] = fmaf(hx, dy, gv[3]);
                        gv[4] = fmaf(hy, dy, gv[4]);
                    }
                }
                if (__any_sync(F, contrib)) {
                    // lanes 4i..4i+3 hold the warp total of value i
                    const float tot = warp_reduce8(gv, lane);
                    if (pend_j < 0) {
                        pend_j = j;
                        pend_tot = tot;
                        pend_9 = g_bl;
                    } else {
                        // Two visits share the ninth values' reduction (lanes with bit 1 end
                        // with this visit's, the others with the pending one's) and one shared
                        // atomic instruction: lane 4i adds the pending visit's value i, lane
                        // 4i + 2 this visit's, lanes 1 and 3 the two ninth values.
                        const bool h1 = lane & 2;
                        float n9 = (h1 ? g_bl : pend_9) + __shfl_xor_sync(F, h1 ? pend_9 : g_bl, 2);
                        n9 += __shfl_xor_sync(F, n9, 16);
                        n9 += __shfl_xor_sync(F, n9, 8);
                        n9 += __shfl_xor_sync(F, n9, 4);
                        n9 += __shfl_xor_sync(F, n9, 1);
                        const bool odd = lane & 1;
                        if (!odd || lane < 4)
                            atomicAdd(&cur.g[(h1 ? j : pend_j) * kGradStride + (odd ? 8 : lane >> 2)],
                                      odd ? n9 : (h1 ? tot : pend_tot));
                        pend_j = -1;
                    }
                }
            }
        }
        if (pend_j >= 0) {  // a visit left without a partner: its ninth value alone (lane 1 adds it)
            const float tb = warp_sum(pend_9);
            if ((lane & 3) == 0 || lane == 1)
                atomicAdd(&cur.g[pend_j * kGradStride + (lane == 1 ? 8 : lane >> 2)], lane == 1 ? tb : pend_tot);
            pend_j = -1;
        }
        __syncthreads();
    }
    if (nb > 0) flush(nb - 1, S[(nb - 1) & 1]);
}

// One thread block per compositing tile: (O.bin / O.tile)^2 per binning tile.
static uint32_t blocks_for(const ViewSet& VS, const DevOpts& O) {
    const int f = O.bin / O.tile;
    return VS.total_tiles * (uint32_t)(f * f);
}

template <int kMode>
static cudaError_t launch_fwd_tiles(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state,
                                    int pair_buf, float* image, float* final_T, int32_t* n_last,
                                    unsigned long long* stats, float* aux_image, cudaStream_t st) {
    const auto* aux = kMode == 2 ? reinterpret_cast<const float4*>(state + lay.aux) : nullptr;
    if (VS.total_tiles == 0) return cudaSuccess;
    const auto* ranges = reinterpret_cast<const uint2*>(state + lay.ranges);
    const auto* pv = reinterpret_cast<const uint32_t*>(state + lay.pair_vals[pair_buf]);
    const auto* rec = reinterpret_cast<const SplatRecord*>(state + lay.records);
    const auto* rech = reinterpret_cast<const SplatRecordH*>(state + lay.records);
    const uint32_t S = (uint32_t)lay.n_splats;
    const dim3 grid(blocks_for(VS, O));
    if (O.tile == 32 && O.record_fp16)
        render_fwd_kernel<32, SplatRecordH, kMode>
            <<<grid, kTilePix, 0, st>>>(VS, O, ranges, pv, rech, S, image, final_T, n_last, stats, aux, aux_image);
    else if (O.tile == 32)
        render_fwd_kernel<32, SplatRecord, kMode>
            <<<grid, kTilePix, 0, st>>>(VS, O, ranges, pv, rec, S, image, final_T, n_last, stats, aux, aux_image);
    else if (O.record_fp16)
        render_fwd_kernel<16, SplatRecordH, kMode>
            <<<grid, kTilePix, 0, st>>>(VS, O, ranges, pv, rech, S, image, final_T, n_last, stats, aux, aux_image);
    else
        render_fwd_kernel<16, SplatRecord, kMode>
            <<<grid, kTilePix, 0, st>>>(VS, O, ranges, pv, rec, S, image, final_T, n_last, stats, aux, aux_image);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_render(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state, int pair_buf,
                          float* image, float* final_T, int32_t* n_last, cudaStream_t st) {
    return launch_fwd_tiles<0>(VS, O, lay, state, pair_buf, image, final_T, n_last, nullptr, nullptr, st);
}

cudaError_t launch_render_stats(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state,
                                int pair_buf, float* image, float* final_T, int32_t* n_last,
                                unsigned long long* stats, cudaStream_t st) {
    return launch_fwd_tiles<1>(VS, O, lay, state, pair_buf, image, final_T, n_last, stats, nullptr, st);
}

cudaError_t launch_render_aux(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state, int pair_buf,
                              float* aux_image, cudaStream_t st) {
    return launch_fwd_tiles<2>(VS, O, lay, state, pair_buf, nullptr, nullptr, nullptr, nullptr, aux_image, st);
}

static cudaError_t launch_bwd_tiles(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state,
                                    int pair_buf, const float* final_T, const int32_t* n_last, const float* dL_dimage,
                                    float4* g2, cudaStream_t st) {
    const auto* ranges = reinterpret_cast<const uint2*>(state + lay.ranges);
    const auto* pv = reinterpret_cast<const uint32_t*>(state + lay.pair_vals[pair_buf]);
    const auto* rec = reinterpret_cast<const SplatRecord*>(state + lay.records);
    const auto* rech = reinterpret_cast<const SplatRecordH*>(state + lay.records);
    const uint32_t S = (uint32_t)lay.n_splats;
    const dim3 grid(blocks_for(VS, O));
    // the staging buffers exceed the 48 KB of static shared memory a block gets by default
    auto smem = [](const void* k) {
        cudaError_t r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
        if (r == cudaSuccess)  // four blocks per SM need the largest shared-memory carve-out
            r = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        return r;
    };
    cudaError_t e;
    if (O.tile == 32 && O.record_fp16) {
        if ((e = smem((const void*)render_bwd_kernel<32, SplatRecordH>)) != cudaSuccess) return e;
        render_bwd_kernel<32, SplatRecordH><<<grid, kTilePix, kBwdSmem, st>>>(VS, O, ranges, pv, rech, S, final_T,
                                                                              n_last, dL_dimage, g2);
    } else if (O.tile == 32) {
        if ((e = smem((const void*)render_bwd_kernel<32, SplatRecord>)) != cudaSuccess) return e;
        render_bwd_kernel<32, SplatRecord><<<grid, kTilePix, kBwdSmem, st>>>(VS, O, ranges, pv, rec, S, final_T,
                                                                             n_last, dL_dimage, g2);
    } else if (O.record_fp16) {
        if ((e = smem((const void*)render_bwd_kernel<16, SplatRecordH>)) != cudaSuccess) return e;
        render_bwd_kernel<16, SplatRecordH><<<grid, kTilePix, kBwdSmem, st>>>(VS, O, ranges, pv, rech, S, final_T,
                                                                              n_last, dL_dimage, g2);
    } else {
        if ((e = smem((const void*)render_bwd_kernel<16, SplatRecord>)) != cudaSuccess) return e;
        render_bwd_kernel<16, SplatRecord><<<grid, kTilePix, kBwdSmem, st>>>(VS, O, ranges, pv, rec, S, final_T,
                                                                             n_last, dL_dimage, g2);
    }
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_render_backward(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state,
                                   int pair_buf, const float* final_T, const int32_t* n_last, const float* dL_dimage,
                                   cudaStream_t st) {
    float4* g2 = reinterpret_cast<float4*>(state + lay.grad2d);
    cudaError_t e = cudaMemsetAsync(g2, 0, sizeof(float4) * 3 * (size_t)lay.n_splats, st);
    if (e != cudaSuccess) return e;
    if (VS.total_tiles == 0) return cudaSuccess;
    return launch_bwd_tiles(VS, O, lay, state, pair_buf, final_T, n_last, dL_dimage, g2, st);
}

// Same as launch_render_backward, accumulating the per-splat 2D gradient into
// g2 (zeroed here) instead of the state (used by the allocation-free
// backward entry point).
cudaError_t launch_render_backward_into(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state,
                                        int pair_buf, const float* final_T, const int32_t* n_last,
                                        const float* dL_dimage, float4* g2, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(g2, 0, sizeof(float4) * 3 * (size_t)lay.n_splats, st);
    if (e != cudaSuccess) return e;
    if (VS.total_tiles == 0) return cudaSuccess;
    return launch_bwd_tiles(VS, O, lay, state, pair_buf, final_T, n_last, dL_dimage, g2, st);
}

}  // namespace fgs4d
