// train.cu -- the training step around the rendering routine (Sec. 3.3, 4.1):
// the photometric loss L = (1 - lambda) L1 + lambda (1 - SSIM) with its
// gradient w.r.t. the rendered images, and a fused Adam update of all
// Gaussian parameters (FP32 master weights, optional BF16 copy of the 4DSH
// coefficients for the mixed-precision renderer).
//
// SSIM per channel (structural similarity with an 11x11 Gaussian window,
// sigma 1.5, normalised to sum 1, zero padding at the image border):
//   mu_x = w * x, e_xx = w * x^2, e_xy = w * (x y)  (likewise mu_y, e_yy)
//   s = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2))
//   with s_xx = e_xx - mu_x^2, s_xy = e_xy - mu_x mu_y, C1 = 0.01^2, C2 = 0.03^2.
// L is the mean over all pixels and channels of the batch of
// (1 - lambda) |x - y| + lambda (1 - s).  With the window symmetric,
//   d sum(s) / dx(p) = (w * S_mu)(p) + 2 x(p) (w * S_xx)(p) + y(p) (w * S_xy)(p),
// where S_mu = ds/dmu_x, S_xx = ds/de_xx, S_xy = ds/de_xy at every pixel q
// (moments held fixed), so the gradient is three more window sums.
//
// Kernels: ssim_moments_kernel (one CTA per 32x32 output tile and channel:
// window sums of x, y, x^2, y^2, xy from a shared-memory tile with a 5-pixel
// halo, then s and its three partials, stored per pixel, and the tile's loss
// sum); ssim_grad_kernel (window sums of the three partials, combined with x,
// y and the L1 sign); loss_reduce_kernel (the per-tile sums, in FP64, in a
// fixed order; a tile's sum is FP32 within each warp, FP64 across warps).
#include <math.h>

#include "fgs4d_internal.cuh"

namespace fgs4d {

namespace {

constexpr int kT = 32;              // output tile side (256 threads, four output pixels each)
constexpr int kPPT = kT * kT / 256; // output pixels per thread
constexpr int kR = 5;               // window radius (11 taps)
constexpr int kE = kT + 2 * kR;     // tile side with halo
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

// Views of the batch, by value (no device state to initialise, so capture-safe),
// with the Gaussian window taps exp(-(i - 5)^2 / (2 * 1.5^2)) normalised to sum 1.
struct LossViews {
    float win[2 * kR + 1];
    uint32_t n;
    uint32_t total_tiles;
    struct V {
        uint32_t tile_base, tiles_x;
        int width, height;
        int64_t pix_base;
    } v[FGS4D_MAX_VIEWS];
};

__device__ __forceinline__ int loss_view(const LossViews& LV, uint32_t tile) {
    int lo = 0, hi = (int)LV.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (LV.v[mid].tile_base <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Loads a kE x kE window of plane `p` (row-major, w x h) around tile origin
// (x0, y0) into sh, zero outside the image.
__device__ __forceinline__ void load_halo(float (*sh)[kE + 1], const float* __restrict__ p, int w, int h, int x0,
                                          int y0) {
    for (int i = threadIdx.x; i < kE * kE; i += blockDim.x) {
        const int ly = i / kE, lx = i - ly * kE;
        const int gx = x0 - kR + lx, gy = y0 - kR + ly;
        sh[ly][lx] = (gx >= 0 && gx < w && gy >= 0 && gy < h) ? p[(size_t)gy * w + gx] : 0.0f;
    }
}

}  // namespace

// One CTA (256 threads) per 32x32 tile of one channel of one view.
__global__ void __launch_bounds__(256) ssim_moments_kernel(const __grid_constant__ LossViews LV,
                                                           const float* __restrict__ image,
                                                           const float* __restrict__ target, float lambda,
                                                           float* __restrict__ partials,
                                                           double* __restrict__ tile_loss) {
    __shared__ float sx[kE][kE + 1], sy[kE][kE + 1];
    __shared__ float hx[kE][kT + 1], hy[kE][kT + 1], hxx[kE][kT + 1], hyy[kE][kT + 1], hxy[kE][kT + 1];
    __shared__ double red[8];
    const uint32_t tile = blockIdx.x;
    const int ch = blockIdx.y;
    const int vi = loss_view(LV, tile);
    const auto& V = LV.v[vi];
    const uint32_t local = tile - V.tile_base;
    const int ty = (int)(local / V.tiles_x), tx = (int)(local - (uint32_t)ty * V.tiles_x);
    const int x0 = tx * kT, y0 = ty * kT;
    const size_t npix = (size_t)V.width * V.height;
    const size_t plane = 3 * (size_t)V.pix_base + (size_t)ch * npix;
    load_halo(sx, image + plane, V.width, V.height, x0, y0);
    load_halo(sy, target + plane, V.width, V.height, x0, y0);
    __syncthreads();
    // horizontal window sums over the kE rows, for the kT output columns
    for (int i = threadIdx.x; i < kE * kT; i += blockDim.x) {
        const int r = i / kT, c = i - r * kT;
        float a = 0.f, b = 0.f, aa = 0.f, bb = 0.f, ab = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kR; k++) {
            const float wk = LV.win[k], xv = sx[r][c + k], yv = sy[r][c + k];
            a = fmaf(wk, xv, a);
            b = fmaf(wk, yv, b);
            aa = fmaf(wk, xv * xv, aa);
            bb = fmaf(wk, yv * yv, bb);
            ab = fmaf(wk, xv * yv, ab);
        }
        hx[r][c] = a;
        hy[r][c] = b;
        hxx[r][c] = aa;
        hyy[r][c] = bb;
        hxy[r][c] = ab;
    }
    __syncthreads();
    float contrib = 0.0f;
#pragma unroll
    for (int j = 0; j < kPPT; j++) {  // output pixels threadIdx.x + 256 j
        const int o = threadIdx.x + 256 * j;
        const int c = o & (kT - 1), r = o / kT;
        const int gx = x0 + c, gy = y0 + r;
        if (gx < V.width && gy < V.height) {
            float mx = 0.f, my = 0.f, exx = 0.f, eyy = 0.f, exy = 0.f;
#pragma unroll
            for (int k = 0; k <= 2 * kR; k++) {
                const float wk = LV.win[k];
                mx = fmaf(wk, hx[r + k][c], mx);
                my = fmaf(wk, hy[r + k][c], my);
                exx = fmaf(wk, hxx[r + k][c], exx);
                eyy = fmaf(wk, hyy[r + k][c], eyy);
                exy = fmaf(wk, hxy[r + k][c], exy);
            }
            const float A1 = 2.f * mx * my + kC1, A2 = 2.f * (exy - mx * my) + kC2;
            const float B1 = mx * mx + my * my + kC1, B2 = (exx - mx * mx) + (eyy - my * my) + kC2;
            const float D = B1 * B2;
            const float s = A1 * A2 / D;
            // partials of s at fixed (e_xx, e_xy) and the other image's moments
            const float s_mu = (2.f * my * (A2 - A1) - 2.f * mx * s * (B2 - B1)) / D;
            const float s_xx = -s / B2;
            const float s_xy = 2.f * A1 / D;
            const size_t p = (size_t)gy * V.width + gx;
            float* P = partials + 3 * plane;  // three planes per channel plane
            P[p] = s_mu;
            P[npix + p] = s_xx;
            P[2 * npix + p] = s_xy;
            const float xv = sx[r + kR][c + kR], yv = sy[r + kR][c + kR];
            contrib += fmaf(1.0f - lambda, fabsf(xv - yv), lambda * (1.0f - s));
        }
    }
    // fixed-order sums: FP32 over a warp's 128 pixels (FP64 runs at a small fraction of the
    // FP32 rate), then FP64 over the block's warps and, in loss_reduce_kernel, the tiles
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) contrib += __shfl_xor_sync(0xffffffffu, contrib, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)contrib;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < 8; i++) t += red[i];
        tile_loss[(size_t)ch * LV.total_tiles + tile] = t;
    }
}

__global__ void __launch_bounds__(256) ssim_grad_kernel(const __grid_constant__ LossViews LV,
                                                        const float* __restrict__ image,
                                                        const float* __restrict__ target, float lambda,
                                                        float inv_count, const float* __restrict__ partials,
                                                        float* __restrict__ dL_dimage) {
    __shared__ float sm[3][kE][kE + 1];
    __shared__ float hm[3][kE][kT + 1];
    const uint32_t tile = blockIdx.x;
    const int ch = blockIdx.y;
    const int vi = loss_view(LV, tile);
    const auto& V = LV.v[vi];
    const uint32_t local = tile - V.tile_base;
    const int ty = (int)(local / V.tiles_x), tx = (int)(local - (uint32_t)ty * V.tiles_x);
    const int x0 = tx * kT, y0 = ty * kT;
    const size_t npix = (size_t)V.width * V.height;
    const size_t plane = 3 * (size_t)V.pix_base + (size_t)ch * npix;
    const float* P = partials + 3 * plane;
#pragma unroll
    for (int m = 0; m < 3; m++) load_halo(sm[m], P + m * npix, V.width, V.height, x0, y0);
    __syncthreads();
    for (int i = threadIdx.x; i < kE * kT; i += blockDim.x) {
        const int r = i / kT, c = i - r * kT;
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kR; k++) {
            const float wk = LV.win[k];
            a0 = fmaf(wk, sm[0][r][c + k], a0);
            a1 = fmaf(wk, sm[1][r][c + k], a1);
            a2 = fmaf(wk, sm[2][r][c + k], a2);
        }
        hm[0][r][c] = a0;
        hm[1][r][c] = a1;
        hm[2][r][c] = a2;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kPPT; j++) {  // output pixels threadIdx.x + 256 j
        const int o = threadIdx.x + 256 * j;
        const int c = o & (kT - 1), r = o / kT;
        const int gx = x0 + c, gy = y0 + r;
        if (gx >= V.width || gy >= V.height) continue;
        float w0 = 0.f, w1 = 0.f, w2 = 0.f;
#pragma unroll
        for (int k = 0; k <= 2 * kR; k++) {
            const float wk = LV.win[k];
            w0 = fmaf(wk, hm[0][r + k][c], w0);
            w1 = fmaf(wk, hm[1][r + k][c], w1);
            w2 = fmaf(wk, hm[2][r + k][c], w2);
        }
        const size_t p = (size_t)gy * V.width + gx;
        const float xv = image[plane + p], yv = target[plane + p];
        const float dssim = w0 + 2.f * xv * w1 + yv * w2;
        const float sgn = (xv > yv) ? 1.f : ((xv < yv) ? -1.f : 0.f);
        dL_dimage[plane + p] = inv_count * ((1.0f - lambda) * sgn - lambda * dssim);
    }
}

// Sums the per-tile losses in a fixed order (one CTA) and writes the mean.
__global__ void __launch_bounds__(256) loss_reduce_kernel(const double* __restrict__ tile_loss, uint32_t count,
                                                          double inv_count, float* __restrict__ loss) {
    __shared__ double red[256];
    double t = 0.0;
    for (uint32_t i = threadIdx.x; i < count; i += blockDim.x) t += tile_loss[i];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = (float)(red[0] * inv_count);
}

// ------------------------------------------------------------------ Adam
// Kingma & Ba's update with bias correction, per element of every parameter
// group (blockIdx.y = group):
//   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
//   p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
// The step t lives on the device (adam_tick_kernel increments it first) so
// that a captured graph advances it on every replay; the learning rates are
// read from device memory for the same reason.
struct AdamGroup {
    float* p;
    float* m;
    float* v;
    const float* g;
    __nv_bfloat16* p_bf16;  // optional rounded copy of p
    int64_t count;
    int lr_index;
};
struct AdamGroups {
    AdamGroup grp[8];
    int n;
};

__global__ void adam_tick_kernel(int64_t* step, float b1, float b2, float* bias) {
    const int64_t t = ++(*step);
    bias[0] = 1.0f - powf(b1, (float)t);
    bias[1] = 1.0f - powf(b2, (float)t);
}

__global__ void __launch_bounds__(256) adam_update_kernel(const __grid_constant__ AdamGroups AG,
                                                          const float* __restrict__ lrs, float b1, float b2,
                                                          float eps, const float* __restrict__ bias) {
    const AdamGroup& G = AG.grp[blockIdx.y];
    const float lr = lrs[G.lr_index];
    const float ib1 = 1.0f / bias[0], ib2 = 1.0f / bias[1];
    auto update = [&](float g, float& m, float& v, float& p) {
        m = fmaf(b1, m, (1.0f - b1) * g);
        v = fmaf(b2, v, (1.0f - b2) * g * g);
        p = p - lr * (m * ib1) / (sqrtf(v * ib2) + eps);
    };
    // four elements per thread in 16-byte accesses when every array allows it (HBM-bound: four
    // float streams in, three out, plus the BF16 copy), then the remainder one by one
    const bool vec = ((reinterpret_cast<uintptr_t>(G.p) | reinterpret_cast<uintptr_t>(G.m) |
                       reinterpret_cast<uintptr_t>(G.v) | reinterpret_cast<uintptr_t>(G.g)) & 15u) == 0 &&
                     (reinterpret_cast<uintptr_t>(G.p_bf16) & 7u) == 0;
    const int64_t n4 = vec ? G.count / 4 : 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += stride) {
        const float4 g = reinterpret_cast<const float4*>(G.g)[q];
        float4 m = reinterpret_cast<const float4*>(G.m)[q];
        float4 v = reinterpret_cast<const float4*>(G.v)[q];
        float4 p = reinterpret_cast<const float4*>(G.p)[q];
        update(g.x, m.x, v.x, p.x);
        update(g.y, m.y, v.y, p.y);
        update(g.z, m.z, v.z, p.z);
        update(g.w, m.w, v.w, p.w);
        reinterpret_cast<float4*>(G.m)[q] = m;
        reinterpret_cast<float4*>(G.v)[q] = v;
        reinterpret_cast<float4*>(G.p)[q] = p;
        if (G.p_bf16) {
            __nv_bfloat162 lo = __floats2bfloat162_rn(p.x, p.y), hi = __floats2bfloat162_rn(p.z, p.w);
            uint2 packed;
            packed.x = *reinterpret_cast<uint32_t*>(&lo);
            packed.y = *reinterpret_cast<uint32_t*>(&hi);
            reinterpret_cast<uint2*>(G.p_bf16)[q] = packed;
        }
    }
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < G.count; i += stride) {
        float m = G.m[i], v = G.v[i], p = G.p[i];
        update(G.g[i], m, v, p);
        G.m[i] = m;
        G.v[i] = v;
        G.p[i] = p;
        if (G.p_bf16) G.p_bf16[i] = __float2bfloat16_rn(p);
    }
}

}  // namespace fgs4d

using namespace fgs4d;

namespace {

fgs4d_status make_loss_views(const fgs4d_view* views, int n_views, LossViews* LV, int64_t* total_pixels) {
    if (!views || n_views < 1 || n_views > FGS4D_MAX_VIEWS) return FGS4D_ERR_INVALID_ARG;
    double sum = 0.0;
    for (int i = 0; i <= 2 * kR; i++) sum += exp(-(double)((i - kR) * (i - kR)) / (2.0 * 1.5 * 1.5));
    for (int i = 0; i <= 2 * kR; i++) LV->win[i] = (float)(exp(-(double)((i - kR) * (i - kR)) / (2.0 * 1.5 * 1.5)) / sum);
    LV->n = (uint32_t)n_views;
    uint32_t tiles = 0;
    int64_t pix = 0;
    for (int i = 0; i < n_views; i++) {
        const int w = views[i].width, h = views[i].height;
        if (w < 1 || h < 1 || w > 16384 || h > 16384) return FGS4D_ERR_INVALID_ARG;
        auto& V = LV->v[i];
        V.tile_base = tiles;
        V.tiles_x = (uint32_t)((w + kT - 1) / kT);
        V.width = w;
        V.height = h;
        V.pix_base = pix;
        tiles += V.tiles_x * (uint32_t)((h + kT - 1) / kT);
        pix += (int64_t)w * h;
    }
    LV->total_tiles = tiles;
    *total_pixels = pix;
    return FGS4D_OK;
}

}  // namespace

extern "C" {

size_t fgs4d_loss_scratch_size(const fgs4d_view* views, int n_views) {
    LossViews LV;
    int64_t pix = 0;
    if (make_loss_views(views, n_views, &LV, &pix) != FGS4D_OK) return 0;
    const size_t partial = 9 * (size_t)pix * sizeof(float);
    const size_t tiles = 3 * (size_t)LV.total_tiles * sizeof(double);
    return ((partial + 255) / 256) * 256 + tiles;
}

fgs4d_status fgs4d_loss_l1_dssim(const fgs4d_view* views, int n_views, const float* image, const float* target,
                                 float lambda, float* loss, float* dL_dimage, void* scratch, size_t scratch_bytes,
                                 fgs4d_stream stream) {
    if (!image || !target || !loss || !dL_dimage || !scratch) return FGS4D_ERR_INVALID_ARG;
    if (!(lambda >= 0.0f && lambda <= 1.0f)) return FGS4D_ERR_INVALID_ARG;
    LossViews* LV = new LossViews;
    int64_t pix = 0;
    fgs4d_status s = make_loss_views(views, n_views, LV, &pix);
    if (s == FGS4D_OK && scratch_bytes < fgs4d_loss_scratch_size(views, n_views)) s = FGS4D_ERR_CAPACITY;
    if (s == FGS4D_OK && ((uintptr_t)scratch % 256 != 0)) s = FGS4D_ERR_INVALID_ARG;
    if (s == FGS4D_OK) {
        cudaError_t e = cudaSuccess;
        const size_t partial = ((9 * (size_t)pix * sizeof(float) + 255) / 256) * 256;
        float* parts = static_cast<float*>(scratch);
        double* tl = reinterpret_cast<double*>(static_cast<char*>(scratch) + partial);
        const cudaStream_t st = (cudaStream_t)stream;
        const double count = 3.0 * (double)pix;
        const dim3 grid(LV->total_tiles, 3);
        if (e == cudaSuccess) {
            ssim_moments_kernel<<<grid, 256, 0, st>>>(*LV, image, target, lambda, parts, tl);
            ssim_grad_kernel<<<grid, 256, 0, st>>>(*LV, image, target, lambda, (float)(1.0 / count), parts,
                                                   dL_dimage);
            loss_reduce_kernel<<<1, 256, 0, st>>>(tl, 3 * LV->total_tiles, 1.0 / count, loss);
            count_launches(3);
            e = cudaGetLastError();
        }
        s = e == cudaSuccess ? FGS4D_OK : FGS4D_ERR_CUDA;
    }
    delete LV;
    return s;
}

fgs4d_status fgs4d_adam_step(const fgs4d_adam_group* groups, int n_groups, const float* lrs, float beta1,
                             float beta2, float eps, int64_t* step, float* bias_scratch, fgs4d_stream stream) {
    if (!groups || n_groups < 1 || n_groups > 8 || !lrs || !step || !bias_scratch) return FGS4D_ERR_INVALID_ARG;
    if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f && eps > 0.0f)) return FGS4D_ERR_INVALID_ARG;
    AdamGroups AG;
    AG.n = n_groups;
    int64_t most = 0;
    for (int i = 0; i < n_groups; i++) {
        const fgs4d_adam_group& g = groups[i];
        if (g.count < 0 || g.lr_index < 0) return FGS4D_ERR_INVALID_ARG;
        if (g.count > 0 && (!g.param || !g.exp_avg || !g.exp_avg_sq || !g.grad)) return FGS4D_ERR_INVALID_ARG;
        AG.grp[i] = AdamGroup{g.param, g.exp_avg, g.exp_avg_sq, g.grad,
                              reinterpret_cast<__nv_bfloat16*>(g.param_bf16), g.count, g.lr_index};
        most = g.count > most ? g.count : most;
    }
    const cudaStream_t st = (cudaStream_t)stream;
    adam_tick_kernel<<<1, 1, 0, st>>>(step, beta1, beta2, bias_scratch);
    count_launches(1);
    if (most > 0) {
        int64_t blocks = (most / 4 + 255) / 256;
        if (blocks < 1) blocks = 1;
        if (blocks > 152 * 16) blocks = 152 * 16;
        adam_update_kernel<<<dim3((unsigned)blocks, (unsigned)n_groups), 256, 0, st>>>(AG, lrs, beta1, beta2, eps,
                                                                                      bias_scratch);
        count_launches(1);
    }
    return cudaGetLastError() == cudaSuccess ? FGS4D_OK : FGS4D_ERR_CUDA;
}

}  // extern "C"
