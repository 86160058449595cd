// render.cu -- tile-based front-to-back compositing (Eq. 6) and its adjoint.
//
// One CTA of 256 threads per 16x16 tile, one pixel per thread.  The tile's
// depth-ordered splat list is walked in batches of 256: each thread gathers
// one splat record into shared memory, then every pixel evaluates the batch.
// A CTA stops as soon as all its pixels have terminated (__syncthreads_count).
//
// Per pixel and splat (readings R4-R6):
//   power = -1/2 (a dx^2 + c dy^2) - b dx dy, dx = x - u, dy = y - v
//   skip if power > 0; alpha = min(alpha_max, alpha_eff * exp(power));
//   skip if alpha < alpha_min; stop (splat excluded) if T (1 - alpha) < T_min;
//   C += c alpha T; T *= 1 - alpha.  Finally C += T bg.
// alpha_eff = sigmoid(logit) p(t) carries the marginal of Eq. 6.
//
// The exponent is evaluated as exp2 of a conic pre-scaled by -log2(e)/2
// (resp. -log2(e)) with explicitly rounded operations, so the forward and the
// adjoint take bit-identical skip decisions.
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

struct Staged {
    float4 a;  // (u, v, A', B')  A' = -log2e/2 a, B' = -log2e b
    float4 b;  // (C', alpha_eff, R, G)
    float c;   // B
};

__device__ __forceinline__ void stage_record(const SplatRecord& r, float4& sa, float4& sb, float& sc) {
    sa = make_float4(r.r0.x, r.r0.y, __fmul_rn(-0.5f * kLog2e, r.r0.z), __fmul_rn(-kLog2e, r.r0.w));
    sb = make_float4(__fmul_rn(-0.5f * kLog2e, r.r1.x), r.r1.y, r.r1.z, r.r1.w);
    sc = r.r2.x;
}

// log2 of the Gaussian factor at (dx, dy): A' dx^2 + C' dy^2 + B' dx dy
__device__ __forceinline__ float power2(float A, float B, float C, float dx, float dy) {
    return __fmaf_rn(__fmul_rn(A, dx), dx, __fmaf_rn(__fmul_rn(C, dy), dy, __fmul_rn(__fmul_rn(B, dx), dy)));
}

__global__ void __launch_bounds__(kTilePix) render_fwd_kernel(const __grid_constant__ ViewSet VS, const DevOpts O,
                                                              const uint2* __restrict__ ranges,
                                                              const uint32_t* __restrict__ pair_vals,
                                                              const SplatRecord* __restrict__ rec, uint32_t n_splats,
                                                              float* __restrict__ image, float* __restrict__ final_T,
                                                              int32_t* __restrict__ n_last) {
    __shared__ float4 s_a[kTilePix];
    __shared__ float4 s_b[kTilePix];
    __shared__ float s_c[kTilePix];
    const uint32_t tile = blockIdx.x;
    const int v = find_view(VS, tile);
    const DevView& V = VS.v[v];
    const uint32_t local = tile - V.tile_base;
    const int ty = (int)(local / (uint32_t)V.tiles_x), tx = (int)local - ty * V.tiles_x;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1));
    const int py = ty * kTile + (threadIdx.x / kTile);
    const bool inside = px < V.width && py < V.height;
    const uint2 range = ranges[tile];
    const float fpx = (float)px, fpy = (float)py;
    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    int32_t last = 0;
    bool done = !inside;
    for (uint32_t base = range.x; base < range.y; base += kTilePix) {
        if (__syncthreads_count(done) == kTilePix) break;
        const uint32_t idx = base + threadIdx.x;
        if (idx < range.y) {
            const uint32_t sid = pair_vals[idx];
            if (sid < n_splats) {
                stage_record(rec[sid], s_a[threadIdx.x], s_b[threadIdx.x], s_c[threadIdx.x]);
            } else {  // never produced by bin_sort; an invisible splat keeps the access in bounds
                s_a[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                s_b[threadIdx.x] = make_float4(0.f, 0.f, 0.f, 0.f);
                s_c[threadIdx.x] = 0.f;
            }
        }
        __syncthreads();
        const int cnt = (int)min((uint32_t)kTilePix, range.y - base);
        if (!done) {
            for (int j = 0; j < cnt; j++) {
                const float4 a = s_a[j];
                const float4 b = s_b[j];
                const float dx = __fsub_rn(fpx, a.x), dy = __fsub_rn(fpy, a.y);
                const float p2 = power2(a.z, a.w, b.x, dx, dy);
                if (!(p2 <= 0.0f)) continue;
                const float araw = __fmul_rn(b.y, ex2_approx(p2));
                const float alpha = fminf(O.alpha_max, araw);
                if (alpha < O.alpha_min) continue;
                const float Tn = T * (1.0f - alpha);
                if (Tn < O.T_min) {
                    done = true;
                    break;
                }
                const float w = alpha * T;
                C0 = fmaf(b.z, w, C0);
                C1 = fmaf(b.w, w, C1);
                C2 = fmaf(s_c[j], w, C2);
                T = Tn;
                last = (int32_t)(base - range.x) + j + 1;
            }
        }
    }
    if (inside) {
        const size_t npix = (size_t)V.width * V.height;
        const size_t p = (size_t)py * V.width + px;
        float* img = image + 3 * (size_t)V.pix_base;
        img[p] = fmaf(T, V.bg[0], C0);
        img[npix + p] = fmaf(T, V.bg[1], C1);
        img[2 * npix + p] = fmaf(T, V.bg[2], C2);
        final_T[V.pix_base + p] = T;
        n_last[V.pix_base + p] = last;
    }
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

__global__ void __launch_bounds__(kTilePix) render_bwd_kernel(
    const __grid_constant__ ViewSet VS, const DevOpts O, const uint2* __restrict__ ranges,
    const uint32_t* __restrict__ pair_vals, const SplatRecord* __restrict__ rec, uint32_t n_splats,
    const float* __restrict__ final_T,
    const int32_t* __restrict__ n_last, const float* __restrict__ dL_dimage, float4* __restrict__ grad2d) {
    __shared__ float4 s_a[kTilePix];
    __shared__ float4 s_b[kTilePix];
    __shared__ float s_c[kTilePix];
    __shared__ uint32_t s_sid[kTilePix];
    __shared__ int s_max;
    const uint32_t tile = blockIdx.x;
    const int v = find_view(VS, tile);
    const DevView& V = VS.v[v];
    const uint32_t local = tile - V.tile_base;
    const int ty = (int)(local / (uint32_t)V.tiles_x), tx = (int)local - ty * V.tiles_x;
    const int px = tx * kTile + (threadIdx.x & (kTile - 1));
    const int py = ty * kTile + (threadIdx.x / kTile);
    const bool inside = px < V.width && py < V.height;
    const uint2 range = ranges[tile];
    const float fpx = (float)px, fpy = (float)py;
    const size_t npix = (size_t)V.width * V.height;
    const size_t p = (size_t)py * V.width + px;
    float T = 1.0f, dC0 = 0.0f, dC1 = 0.0f, dC2 = 0.0f;
    int32_t last = 0;
    if (inside) {
        T = final_T[V.pix_base + p];
        last = n_last[V.pix_base + p];
        const float* g = dL_dimage + 3 * (size_t)V.pix_base;
        dC0 = g[p];
        dC1 = g[npix + p];
        dC2 = g[2 * npix + p];
    }
    // acc = sum_{j > i} c_j alpha_j T_j + T_final bg, built back to front
    float acc0 = T * V.bg[0], acc1 = T * V.bg[1], acc2 = T * V.bg[2];
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    atomicMax(&s_max, last);
    __syncthreads();
    const int max_last = min(s_max, (int)(range.y - range.x));
    for (int end = max_last; end > 0; end -= kTilePix) {
        const int start = max(0, end - kTilePix);
        const int cnt = end - start;
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            const uint32_t idx = range.x + (uint32_t)(end - 1 - (int)threadIdx.x);
            uint32_t sid = pair_vals[idx];
            if (sid >= n_splats) sid = 0;  // never produced by bin_sort; keeps the access in bounds
            stage_record(rec[sid], s_a[threadIdx.x], s_b[threadIdx.x], s_c[threadIdx.x]);
            s_sid[threadIdx.x] = sid;
        }
        __syncthreads();
        for (int j = 0; j < cnt; j++) {
            const int pos = end - 1 - j;  // 0-based position in the tile list
            float g_u = 0.f, g_v = 0.f, g_a = 0.f, g_b = 0.f, g_c = 0.f, g_ae = 0.f, g_r = 0.f, g_g = 0.f, g_bl = 0.f;
            bool contrib = false;
            if (pos < last) {
                const float4 a = s_a[j];
                const float4 b = s_b[j];
                const float dx = __fsub_rn(fpx, a.x), dy = __fsub_rn(fpy, a.y);
                const float p2 = power2(a.z, a.w, b.x, dx, dy);
                if (p2 <= 0.0f) {
                    const float G = ex2_approx(p2);
                    const float araw = __fmul_rn(b.y, G);
                    const float alpha = fminf(O.alpha_max, araw);
                    if (alpha >= O.alpha_min) {
                        contrib = true;
                        const float om = 1.0f - alpha;
                        const float Ti = T / om;
                        const float cr = b.z, cg = b.w, cb = s_c[j];
                        const float dalpha =
                            dC0 * (cr * Ti - acc0 / om) + dC1 * (cg * Ti - acc1 / om) + dC2 * (cb * Ti - acc2 / om);
                        const float w = alpha * Ti;
                        g_r = dC0 * w;
                        g_g = dC1 * w;
                        g_bl = dC2 * w;
                        acc0 = fmaf(cr, w, acc0);
                        acc1 = fmaf(cg, w, acc1);
                        acc2 = fmaf(cb, w, acc2);
                        T = Ti;
                        if (!(araw > O.alpha_max)) {
                            g_ae = dalpha * G;
                            const float dpow = dalpha * araw;
                            // natural conic from the pre-scaled one
                            const float ca = a.z * (-2.0f * kLn2), cb2 = a.w * (-kLn2), cc = b.x * (-2.0f * kLn2);
                            g_a = -0.5f * dpow * dx * dx;
                            g_c = -0.5f * dpow * dy * dy;
                            g_b = -dpow * dx * dy;
                            g_u = dpow * (ca * dx + cb2 * dy);
                            g_v = dpow * (cc * dy + cb2 * dx);
                        }
                    }
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                g_u = warp_sum(g_u);
                g_v = warp_sum(g_v);
                g_a = warp_sum(g_a);
                g_b = warp_sum(g_b);
                g_c = warp_sum(g_c);
                g_ae = warp_sum(g_ae);
                g_r = warp_sum(g_r);
                g_g = warp_sum(g_g);
                g_bl = warp_sum(g_bl);
                if ((threadIdx.x & 31) == 0) {
                    float4* dst = grad2d + 3 * (size_t)s_sid[j];
                    atomicAdd(dst + 0, make_float4(g_u, g_v, g_a, g_b));
                    atomicAdd(dst + 1, make_float4(g_c, g_ae, g_r, g_g));
                    atomicAdd(reinterpret_cast<float*>(dst + 2), g_bl);
                }
            }
        }
    }
}

cudaError_t launch_render(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state, int pair_buf,
                          float* image, float* final_T, int32_t* n_last, cudaStream_t st) {
    if (VS.total_tiles == 0) return cudaSuccess;
    const auto* ranges = reinterpret_cast<const uint2*>(state + lay.ranges);
    const auto* pv = reinterpret_cast<const uint32_t*>(state + lay.pair_vals[pair_buf]);
    const auto* rec = reinterpret_cast<const SplatRecord*>(state + lay.records);
    render_fwd_kernel<<<VS.total_tiles, kTilePix, 0, st>>>(VS, O, ranges, pv, rec, (uint32_t)lay.n_splats, image,
                                                          final_T, n_last);
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
    const auto* ranges = reinterpret_cast<const uint2*>(state + lay.ranges);
    const auto* pv = reinterpret_cast<const uint32_t*>(state + lay.pair_vals[pair_buf]);
    const auto* rec = reinterpret_cast<const SplatRecord*>(state + lay.records);
    render_bwd_kernel<<<VS.total_tiles, kTilePix, 0, st>>>(VS, O, ranges, pv, rec, (uint32_t)lay.n_splats, final_T,
                                                          n_last, dL_dimage, g2);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace fgs4d
