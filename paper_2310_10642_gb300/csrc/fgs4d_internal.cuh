// fgs4d_internal.cuh -- device-side data structures and math shared by the
// kernels of libfgs4d (slice/project, binning, compositing and their adjoint).
//
// Nothing here is visible through the C ABI.  The view set and the options
// travel to every kernel by value as a __grid_constant__ parameter, so a
// launch captured in a CUDA graph carries its own copy.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fgs4d.h"

namespace fgs4d {

constexpr int kTilePix = 256;                  // threads per compositing CTA
constexpr float kLog2e = 1.4426950408889634f;  // log2(e)
constexpr float kLn2 = 0.6931471805599453f;

// One view, pre-digested on the host.
struct DevView {
    float W[9];       // world -> camera rotation, row-major
    float tau[3];     // translation
    float campos[3];  // camera centre C = -W^T tau
    float fx, fy, cx, cy;
    float limx, limy;  // clamp of x/z, y/z inside the Jacobian (huge when off)
    float t;
    float bg[3];
    int width, height, tiles_x, tiles_y;  // binning tiles across and down
    uint32_t tile_base;  // first global binning tile id of this view
    uint32_t pix_base;   // first pixel (offset into final_T / n_last)
};

struct ViewSet {
    int n;
    uint32_t total_tiles;
    DevView v[FGS4D_MAX_VIEWS];
};

struct DevOpts {
    float p_min, near_z, alpha_min, alpha_max, T_min, dilation;
    float schur_cond, conic_cond;
    float ln_alpha_min;
    int record_fp16;
    int tile;   // compositing tile side: 16 or 32 (one thread block)
    int bin;    // binning tile side: 16, 32 or 64, a multiple of tile
    int batch;  // records staged per shared-memory batch while compositing: 32..256
    int aux;    // store per-splat depth and flow (fgs4d_render_aux)
    float flow_dt;
    int accumulate;  // backward: add to the gradient outputs instead of overwriting them
};

// Gaussian parameters (SoA) as the kernels see them.
struct DevGauss {
    const float* mu;
    const float* log_s;
    const float* ql;
    const float* qr;
    const float* logit;
    const void* shs;
    int n;
    int L;
    int K;
    float inv_period;
    int shs_bf16;
    int rot;  // fgs4d_rotation: how Sigma is formed and sliced (RotMode)
};

// fgs4d_rotation as a compile-time kernel parameter.  kRot4D: R = L(q_l) R(q_r)
// (Eq. 8) and the slice of Eq. 9-10.  kRotSpatial (No-4DRot): R =
// blockdiag(R3(q_l), 1), so Sigma is block-diagonal and the slice reduces to
// mu_{xyz|t} = mu_xyz, Sigma_{xyz|t} = Sigma_xyz, p(t) from s_t alone: no
// Schur complement, no velocity term.  kRotStatic (3D Gaussian splatting):
// as kRotSpatial with no time axis at all: mu_t and s_t are not read, p = 1
// and the 4DSH time basis is evaluated at dt = 0.
enum RotMode : int { kRot4D = 0, kRotSpatial = 1, kRotStatic = 2 };

// ---------------------------------------------------------------------------
// Per-frame state layout (byte offsets into the caller's state buffer).
// ---------------------------------------------------------------------------
struct StateLayout {
    size_t counters;       // uint32[16]: n_visible, n_pairs, status, capacity
    size_t records;        // SplatRecord[V*n]
    size_t tiles_touched;  // uint32[V*n]
    size_t depth_key;      // uint32[V*n]
    size_t sort_keys[2];   // uint32[V*n] double buffer (depth sort)
    size_t sort_vals[2];   // uint32[V*n]
    size_t offsets;        // uint32[V*n] pair offsets per depth-sorted splat
    size_t scan_tmp;       // uint32[kScanBlocksMax + 32]
    size_t hist;           // uint32[kMaxDigits * kSortBlocksMax + kMaxDigits]
    size_t ranges;         // uint2[total_tiles]
    size_t grad2d;         // float4[3 * V*n] per-splat 2D gradient
    size_t aux;            // float4[V*n] depth, flow u, flow v (0 when aux channels are off)
    size_t gsum;           // float[11][n] per-Gaussian sums of the projection adjoint
    size_t chunk_hist;     // uint32[total_tiles * chunks_per_view]: (tile, chunk) counts (counting path only)
    size_t pair_keys[2];   // uint32[capacity] double buffer (radix path only)
    size_t pair_vals[2];   // uint32[capacity] (the counting path uses pair_vals[0] alone)
    size_t fixed_bytes;    // everything above except the pair buffers
    size_t total;
    int64_t capacity;
    int64_t n_splats;      // V * n
    uint32_t record_bytes;
    // Pair binning by a stable counting sort over (tile, chunk) counts when
    // every view has at most kCountTilesMax binning tiles; otherwise by a
    // radix sort of the pairs on their tile id.
    int count_sort;
    uint32_t chunk;            // visible splats per chunk (a power of two)
    uint32_t chunks_per_view;  // ceil(n / chunk): a view has at most n visible splats (chunks in use: device)
    uint32_t view_tiles_max;   // binning tiles of the largest view
};

constexpr int kScanBlocksMax = 1024;
constexpr int kSortBlocksMax = 1024;
constexpr int kMaxDigits = 512;  // radix digits of at most 9 bits
constexpr uint32_t kCountTilesMax = 4096;  // binning tiles per view for the counting path
constexpr int kCountWarps = 4;              // warps per block of the counting kernels, one chunk each
constexpr uint32_t kCountBuf = 1024;        // pairs a warp of the scatter stages per round of 32 splats

// Splat record (FP32): 48 bytes, three 16-byte vectors.
//   r0 = (u, v, conic_a, conic_b)   r1 = (conic_c, alpha_eff, R, G)
//   r2 = (B, depth, hx, hy)         half extents of the support box
struct __align__(16) SplatRecord {
    float4 r0, r1, r2;
};

// Splat record (mixed precision): 32 bytes, two 16-byte vectors.
//   (u, v, alpha_eff, R, G, B) fp32; the conic Q = [[a, b], [b, c]] as its
//   Cholesky factor Q = L L^T, L = [[l11, 0], [l21, l22]], in 16 bits per
//   entry: int16 mantissas m with one shared exponent, l = m 2^-e, e chosen
//   so that the largest |m| lies in [2^14, 2^15).  The quadratic form
//   d^T Q d = (l11 dx + l21 dy)^2 + (l22 dy)^2 is then a sum of squares whose
//   relative error is ~2^-14: rounding (a, b, c) instead ruins it along the long
//   axis of an elongated splat, where a dx^2 + 2 b dx dy + c dy^2 cancels, and
//   IEEE fp16's 11-bit significands perturb alpha by ~1e-3 relative, enough to
//   flip alpha_min decisions that cost up to alpha_min T per splat.  The
//   support box is not stored; it follows from L wherever the record is
//   decoded, so binning and compositing use the same, conservative box.
struct __align__(16) SplatRecordH {
    float u, v, alpha_eff, R;
    float G, B;
    short m11, m21, m22;
    short e;
};
static_assert(sizeof(SplatRecordH) == 32, "mixed-precision record must be 32 bytes");

// conic (a, b, c) and the 2D covariance's S11 -> Cholesky factor of the conic:
// l11 = sqrt(a), l21 = b / l11, l22 = sqrt(c - l21^2) = 1 / sqrt(S11)
// (the last form needs no subtraction).
__device__ __forceinline__ SplatRecordH encode_record_h(float u, float v, const float* conic, float S11,
                                                        float alpha_eff, const float* col) {
    SplatRecordH r;
    r.u = u;
    r.v = v;
    r.alpha_eff = alpha_eff;
    r.R = col[0];
    r.G = col[1];
    r.B = col[2];
    const float l11 = sqrtf(conic[0]);
    const float l21 = conic[1] / l11;
    const float l22 = rsqrtf(S11);
    int e = 0;
    frexpf(fmaxf(fmaxf(l11, fabsf(l21)), l22), &e);  // max = f 2^e, f in [0.5, 1)
    const int sh = 15 - e;                            // max 2^sh in [2^14, 2^15)
    auto q = [sh](float x) { return (short)fminf(fmaxf(rintf(ldexpf(x, sh)), -32767.0f), 32767.0f); };
    r.m11 = q(l11);
    r.m21 = q(l21);
    r.m22 = q(l22);
    r.e = (short)sh;
    return r;
}

// Decoded view of either record type.  (a, b, c) is the conic; for the
// mixed-precision record (l11, l21, l22) is its Cholesky factor, from which
// (a, b, c) was formed.
struct SplatView {
    float u, v, a, b, c, alpha_eff, R, G, B, hx, hy;
    float l11, l21, l22;
};
__device__ __forceinline__ SplatView decode_record(const SplatRecord& r, float) {
    return SplatView{r.r0.x, r.r0.y, r.r0.z, r.r0.w, r.r1.x, r.r1.y, r.r1.z, r.r1.w, r.r2.x, r.r2.z, r.r2.w,
                     0.0f,   0.0f,   0.0f};
}
// Hardware approximations (about one to two ulp) for the support ellipse's
// set-up (ellipse_rows): its spans carry half a pixel (and k 0.2%) of slack,
// far above their error, and every kernel rounds them alike.  (The support
// box of decode_record keeps the IEEE forms: with them the adjoint raster
// kernel, which decodes every staged record, schedules faster.)
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// natural log through the hardware base-2 log
__device__ __forceinline__ float ln_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return __fmul_rn(y, 0.69314718055994531f);
}
// k = 2 ln(alpha_eff / alpha_min), 0 when alpha_eff <= alpha_min
__device__ __forceinline__ float support_k(float alpha_eff, float ln_alpha_min) {
    return 2.0f * fmaxf(__fsub_rn(ln_approx(alpha_eff), ln_alpha_min), 0.0f);
}

// ln_alpha_min = log(alpha_min).  With Sigma = Q^-1: Sigma_11 = 1 / l22^2 and
// Sigma_00 = (l21^2 + l22^2) / (l11 l22)^2, so the support box
// |dx| <= sqrt(k Sigma_00), |dy| <= sqrt(k Sigma_11), k = 2 ln(alpha_eff /
// alpha_min) (plus half a pixel, as in project_view) needs no subtraction.
__device__ __forceinline__ SplatView decode_record(const SplatRecordH& r, float ln_alpha_min) {
    const float s = ldexpf(1.0f, -(int)r.e);
    SplatView o;
    o.u = r.u;
    o.v = r.v;
    o.l11 = (float)r.m11 * s;
    o.l21 = (float)r.m21 * s;
    o.l22 = (float)r.m22 * s;
    o.a = o.l11 * o.l11;
    o.b = o.l11 * o.l21;
    o.c = fmaf(o.l21, o.l21, o.l22 * o.l22);
    o.alpha_eff = r.alpha_eff;
    o.R = r.R;
    o.G = r.G;
    o.B = r.B;
    const float sk = sqrtf(2.0f * fmaxf(logf(o.alpha_eff) - ln_alpha_min, 0.0f));
    const bool ok = o.l11 > 0.0f && o.l22 > 0.0f;
    o.hx = ok ? sk * sqrtf(fmaf(o.l21, o.l21, o.l22 * o.l22)) / (o.l11 * o.l22) + 0.5f : -1.0f;
    o.hy = ok ? sk / o.l22 + 0.5f : -1.0f;
    return o;
}

// ---------------------------------------------------------------------------
// Small math helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Real spherical harmonics, degree <= 3, Cartesian form on the unit sphere
// (Condon-Shortley phase; index j = l^2 + l + m).  Constants are
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the factors of the Cartesian
// polynomials.
__device__ __forceinline__ void sh_eval(int L, float x, float y, float z, float* Y) {
    Y[0] = 0.28209479177387814f;
    if (L < 1) return;
    Y[1] = -0.4886025119029199f * y;
    Y[2] = 0.4886025119029199f * z;
    Y[3] = -0.4886025119029199f * x;
    if (L < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, yz = y * z, xz = x * z;
    Y[4] = 1.0925484305920792f * xy;
    Y[5] = -1.0925484305920792f * yz;
    Y[6] = 0.31539156525252005f * (2.0f * zz - xx - yy);
    Y[7] = -1.0925484305920792f * xz;
    Y[8] = 0.5462742152960396f * (xx - yy);
    if (L < 3) return;
    Y[9] = -0.5900435899266435f * y * (3.0f * xx - yy);
    Y[10] = 2.890611442640554f * xy * z;
    Y[11] = -0.4570457994644658f * y * (4.0f * zz - xx - yy);
    Y[12] = 0.3731763325901154f * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
    Y[13] = -0.4570457994644658f * x * (4.0f * zz - xx - yy);
    Y[14] = 1.445305721320277f * z * (xx - yy);
    Y[15] = -0.5900435899266435f * x * (xx - 3.0f * yy);
}

// Gradient of sum_j w_j Y_j (as polynomials in x, y, z) -> (gx, gy, gz).
__device__ __forceinline__ void sh_grad(int L, float x, float y, float z, const float* w, float& gx, float& gy,
                                        float& gz) {
    gx = gy = gz = 0.0f;
    if (L < 1) return;
    gy += -0.4886025119029199f * w[1];
    gz += 0.4886025119029199f * w[2];
    gx += -0.4886025119029199f * w[3];
    if (L < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    {
        const float c0 = 1.0925484305920792f, c2 = 0.31539156525252005f, c4 = 0.5462742152960396f;
        gx += c0 * y * w[4];
        gy += c0 * x * w[4];
        gy += -c0 * z * w[5];
        gz += -c0 * y * w[5];
        gx += c2 * (-2.0f * x) * w[6];
        gy += c2 * (-2.0f * y) * w[6];
        gz += c2 * (4.0f * z) * w[6];
        gx += -c0 * z * w[7];
        gz += -c0 * x * w[7];
        gx += c4 * (2.0f * x) * w[8];
        gy += c4 * (-2.0f * y) * w[8];
    }
    if (L < 3) return;
    {
        const float a = -0.5900435899266435f, b = 2.890611442640554f, c = -0.4570457994644658f;
        const float d = 0.3731763325901154f, e = 1.445305721320277f;
        // Y9 = a y (3xx - yy)
        gx += a * 6.0f * x * y * w[9];
        gy += a * (3.0f * xx - 3.0f * yy) * w[9];
        // Y10 = b x y z
        gx += b * y * z * w[10];
        gy += b * x * z * w[10];
        gz += b * x * y * w[10];
        // Y11 = c y (4zz - xx - yy)
        gx += c * y * (-2.0f * x) * w[11];
        gy += c * (4.0f * zz - xx - 3.0f * yy) * w[11];
        gz += c * y * 8.0f * z * w[11];
        // Y12 = d z (2zz - 3xx - 3yy)
        gx += d * z * (-6.0f * x) * w[12];
        gy += d * z * (-6.0f * y) * w[12];
        gz += d * (6.0f * zz - 3.0f * xx - 3.0f * yy) * w[12];
        // Y13 = c x (4zz - xx - yy)
        gx += c * (4.0f * zz - 3.0f * xx - yy) * w[13];
        gy += c * x * (-2.0f * y) * w[13];
        gz += c * x * 8.0f * z * w[13];
        // Y14 = e z (xx - yy)
        gx += e * z * 2.0f * x * w[14];
        gy += e * z * (-2.0f * y) * w[14];
        gz += e * (xx - yy) * w[14];
        // Y15 = a x (xx - 3yy)
        gx += a * (3.0f * xx - 3.0f * yy) * w[15];
        gy += a * x * (-6.0f * y) * w[15];
    }
}

__device__ __forceinline__ float to_float(float x) { return x; }
__device__ __forceinline__ float to_float(__nv_bfloat16 x) { return __bfloat162float(x); }


// ---------------------------------------------------------------------------
// Per-Gaussian, view-independent part: activations, R = L(q_l) R(q_r),
// M = R S, Sigma = M M^T (Eq. 7, Eq. 8).
// ---------------------------------------------------------------------------
struct Core {
    float mu[4];
    float s[4];
    float alpha;
    float qln[4], qrn[4];
    float nl, nr;
    float R[16];
    float M[16];
    float S[16];  // full symmetric Sigma
    bool ok;
};

__device__ __forceinline__ void left_matrix(const float* q, float* L) {
    const float a = q[0], b = q[1], c = q[2], d = q[3];
    L[0] = a;  L[1] = -b; L[2] = -c;  L[3] = -d;
    L[4] = b;  L[5] = a;  L[6] = -d;  L[7] = c;
    L[8] = c;  L[9] = d;  L[10] = a;  L[11] = -b;
    L[12] = d; L[13] = -c; L[14] = b; L[15] = a;
}
__device__ __forceinline__ void right_matrix(const float* q, float* R) {
    const float p = q[0], qq = q[1], r = q[2], s = q[3];
    R[0] = p;   R[1] = -qq; R[2] = -r;  R[3] = -s;
    R[4] = qq;  R[5] = p;   R[6] = s;   R[7] = -r;
    R[8] = r;   R[9] = -s;  R[10] = p;  R[11] = qq;
    R[12] = s;  R[13] = r;  R[14] = -qq; R[15] = p;
}

// blockdiag(R3(q), 1): the rotation of x, y, z by the unit quaternion
// q = (w, x, y, z) in the usual convention, t fixed (the No-4DRot variant).
template <class T>
__device__ __forceinline__ void spatial_rotation(const T* q, T* R) {
    const T w = q[0], x = q[1], y = q[2], z = q[3];
    const T one = T(1), two = T(2);
    R[0] = one - two * (y * y + z * z); R[1] = two * (x * y - w * z);       R[2] = two * (x * z + w * y);       R[3] = T(0);
    R[4] = two * (x * y + w * z);       R[5] = one - two * (x * x + z * z); R[6] = two * (y * z - w * x);       R[7] = T(0);
    R[8] = two * (x * z - w * y);       R[9] = two * (y * z + w * x);       R[10] = one - two * (x * x + y * y); R[11] = T(0);
    R[12] = T(0);                       R[13] = T(0);                       R[14] = T(0);                       R[15] = one;
}

template <int kMode>
__device__ __forceinline__ void load_core(const DevGauss& G, int g, Core& c) {
    constexpr bool k4D = kMode == kRot4D, kStatic = kMode == kRotStatic;
    const size_t n = (size_t)G.n;
    float ls[4], ql[4], qr[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        // a static Gaussian has no time axis: mu_t and s_t are not read
        c.mu[i] = (kStatic && i == 3) ? 0.0f : __ldg(G.mu + i * n + g);
        ls[i] = (kStatic && i == 3) ? 0.0f : __ldg(G.log_s + i * n + g);
        ql[i] = __ldg(G.ql + i * n + g);
        qr[i] = k4D ? __ldg(G.qr + i * n + g) : (i == 0 ? 1.0f : 0.0f);
    }
    const float logit = __ldg(G.logit + g);
    c.alpha = 1.0f / (1.0f + expf(-logit));
    const float nl2 = ql[0] * ql[0] + ql[1] * ql[1] + ql[2] * ql[2] + ql[3] * ql[3];
    const float nr2 = qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2] + qr[3] * qr[3];
    c.nl = sqrtf(nl2);
    c.nr = sqrtf(nr2);
    bool finite = isfinite(logit) && isfinite(nl2) && isfinite(nr2);
#pragma unroll
    for (int i = 0; i < 4; i++) {
        c.s[i] = expf(ls[i]);
        finite = finite && isfinite(c.mu[i]) && isfinite(c.s[i]) && c.s[i] > 0.0f;
        c.qln[i] = ql[i] / c.nl;
        c.qrn[i] = qr[i] / c.nr;
    }
    c.ok = finite && nl2 > 1e-24f && nr2 > 1e-24f;
    if constexpr (!k4D) {
        // Sigma = blockdiag(R3 diag(s_xyz^2) R3^T, s_t^2): the 3x3 block only
        spatial_rotation(c.qln, c.R);
#pragma unroll
        for (int i = 0; i < 16; i++) c.M[i] = 0.0f;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) c.M[i * 4 + j] = c.R[i * 4 + j] * c.s[j];
        c.M[15] = kStatic ? 0.0f : c.s[3];
#pragma unroll
        for (int i = 0; i < 16; i++) c.S[i] = 0.0f;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = i; j < 3; j++) {
                const float acc = fmaf(c.M[i * 4 + 0], c.M[j * 4 + 0],
                                       fmaf(c.M[i * 4 + 1], c.M[j * 4 + 1], c.M[i * 4 + 2] * c.M[j * 4 + 2]));
                c.S[i * 4 + j] = acc;
                c.S[j * 4 + i] = acc;
            }
        c.S[15] = c.M[15] * c.M[15];
    } else {
        float Lm[16], Rm[16];
        left_matrix(c.qln, Lm);
        right_matrix(c.qrn, Rm);
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = 0; j < 4; j++) {
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k < 4; k++) acc = fmaf(Lm[i * 4 + k], Rm[k * 4 + j], acc);
                c.R[i * 4 + j] = acc;
                c.M[i * 4 + j] = acc * c.s[j];
            }
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
            for (int j = i; j < 4; j++) {
                float acc = 0.0f;
#pragma unroll
                for (int k = 0; k < 4; k++) acc = fmaf(c.M[i * 4 + k], c.M[j * 4 + k], acc);
                c.S[i * 4 + j] = acc;
                c.S[j * 4 + i] = acc;
            }
    }
}

// Same Sigma in double precision (fallback for ill-conditioned slices of
// the 4D rotation; the block-diagonal modes form no Schur complement).
static __device__ __noinline__ void core_sigma_f64(const DevGauss& G, int g, double* Sd) {
    const size_t n = (size_t)G.n;
    double ql[4], qr[4], s[4], nl = 0.0, nr = 0.0;
    for (int i = 0; i < 4; i++) {
        ql[i] = (double)G.ql[i * n + g];
        qr[i] = (double)G.qr[i * n + g];
        s[i] = exp((double)G.log_s[i * n + g]);
        nl += ql[i] * ql[i];
        nr += qr[i] * qr[i];
    }
    nl = sqrt(nl);
    nr = sqrt(nr);
    for (int i = 0; i < 4; i++) {
        ql[i] /= nl;
        qr[i] /= nr;
    }
    double M[16];
    const double a = ql[0], b = ql[1], c = ql[2], d = ql[3];
    const double Lm[16] = {a, -b, -c, -d, b, a, -d, c, c, d, a, -b, d, -c, b, a};
    const double p = qr[0], q = qr[1], r = qr[2], t = qr[3];
    const double Rm[16] = {p, -q, -r, -t, q, p, t, -r, r, -t, p, q, t, r, -q, p};
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            double acc = 0.0;
            for (int k = 0; k < 4; k++) acc += Lm[i * 4 + k] * Rm[k * 4 + j];
            M[i * 4 + j] = acc * s[j];
        }
    for (int i = 0; i < 4; i++)
        for (int j = 0; j < 4; j++) {
            double acc = 0.0;
            for (int k = 0; k < 4; k++) acc += M[i * 4 + k] * M[j * 4 + k];
            Sd[i * 4 + j] = acc;
        }
}

// ---------------------------------------------------------------------------
// Per-view slice (Eq. 9, Eq. 10) and projection (Eq. 3, Eq. 4).
// ---------------------------------------------------------------------------
struct ViewGeom {
    float p;         // marginal p(t)
    float dt;        // t - mu_t
    float mu3[3];    // conditional mean
    float S3[6];     // conditional covariance (00, 01, 02, 11, 12, 22)
    float xc[3];     // camera-space mean
    float T[6];      // J W (2x3)
    bool clx, cly;   // Jacobian clamp active
    float cov[3];    // 2D covariance (00, 01, 11) incl. dilation
    float conic[3];  // (a, b, c)
    float u, v;
    float alpha_eff;
    float hx, hy;    // half extents of the support box (pixels)
    int rect[4];     // inclusive tile rect: x0, y0, x1, y1
    int tiles;       // number of touched tiles (0 = invisible)
};

template <int kMode>
__device__ __forceinline__ void slice_view(const Core& c, const DevView& V, const DevOpts& O, const DevGauss& G, int g,
                                           ViewGeom& w, bool allow_f64) {
    if constexpr (kMode != kRot4D) {
        // block-diagonal Sigma: nothing to condition on; p(t) from s_t alone (static: p = 1)
        w.dt = kMode == kRotStatic ? 0.0f : V.t - c.mu[3];
        w.p = kMode == kRotStatic ? 1.0f : expf(-0.5f * w.dt * w.dt / c.S[15]);
        w.mu3[0] = c.mu[0];
        w.mu3[1] = c.mu[1];
        w.mu3[2] = c.mu[2];
        w.S3[0] = c.S[0];
        w.S3[1] = c.S[1];
        w.S3[2] = c.S[2];
        w.S3[3] = c.S[5];
        w.S3[4] = c.S[6];
        w.S3[5] = c.S[10];
        return;
    }
    const float sig = c.S[15];
    w.dt = V.t - c.mu[3];
    w.p = expf(-0.5f * w.dt * w.dt / sig);
    const float inv = 1.0f / sig;
    const float b0 = c.S[3], b1 = c.S[7], b2 = c.S[11];
    const float k = w.dt * inv;
    w.mu3[0] = fmaf(b0, k, c.mu[0]);
    w.mu3[1] = fmaf(b1, k, c.mu[1]);
    w.mu3[2] = fmaf(b2, k, c.mu[2]);
    w.S3[0] = c.S[0] - b0 * b0 * inv;
    w.S3[1] = c.S[1] - b0 * b1 * inv;
    w.S3[2] = c.S[2] - b0 * b2 * inv;
    w.S3[3] = c.S[5] - b1 * b1 * inv;
    w.S3[4] = c.S[6] - b1 * b2 * inv;
    w.S3[5] = c.S[10] - b2 * b2 * inv;
    // Conditioning test: strong cancellation in the Schur complement.
    if (allow_f64 && (w.S3[0] < O.schur_cond * c.S[0] || w.S3[3] < O.schur_cond * c.S[5] ||
                      w.S3[5] < O.schur_cond * c.S[10])) {
        double Sd[16];
        core_sigma_f64(G, g, Sd);
        const double sd = Sd[15];
        const double dtd = (double)V.t - (double)c.mu[3];
        const double bd[3] = {Sd[3], Sd[7], Sd[11]};
        for (int i = 0; i < 3; i++) w.mu3[i] = (float)((double)c.mu[i] + bd[i] * dtd / sd);
        w.S3[0] = (float)(Sd[0] - bd[0] * bd[0] / sd);
        w.S3[1] = (float)(Sd[1] - bd[0] * bd[1] / sd);
        w.S3[2] = (float)(Sd[2] - bd[0] * bd[2] / sd);
        w.S3[3] = (float)(Sd[5] - bd[1] * bd[1] / sd);
        w.S3[4] = (float)(Sd[6] - bd[1] * bd[2] / sd);
        w.S3[5] = (float)(Sd[10] - bd[2] * bd[2] / sd);
        w.p = (float)exp(-0.5 * dtd * dtd / sd);
    }
}

// Tiles touched by the support box |x - u| <= hx, |y - v| <= hy of a splat:
// the pixels it covers, clamped to the image, and the tiles containing them
// (inclusive rect x0, y0, x1, y1).  Returns the tile count, 0 when the box
// misses the image.  The one place that turns a box into tiles, for both the
// count (slice/project) and the emitted pairs (bin_sort).
__device__ __forceinline__ int box_tiles(float u, float v, float hx, float hy, const DevView& V, int tile, int* rect) {
    const float fx0 = fmaxf(ceilf(u - hx), 0.0f);
    const float fx1 = fminf(floorf(u + hx), (float)(V.width - 1));
    const float fy0 = fmaxf(ceilf(v - hy), 0.0f);
    const float fy1 = fminf(floorf(v + hy), (float)(V.height - 1));
    if (!(fx0 <= fx1 && fy0 <= fy1)) return 0;
    const int sh = __ffs(tile) - 1;  // tile is a power of two; the pixel bounds are >= 0
    rect[0] = (int)fx0 >> sh;
    rect[1] = (int)fy0 >> sh;
    rect[2] = (int)fx1 >> sh;
    rect[3] = (int)fy1 >> sh;
    return (rect[2] - rect[0] + 1) * (rect[3] - rect[1] + 1);
}

// Tile binning by the support ellipse (reading R7 made tight).  alpha >=
// alpha_min needs d^T Q d <= k, k = 2 ln(alpha_eff / alpha_min), Q the conic.
// With rx = sqrt(k Sigma_00), ry = sqrt(k Sigma_11) (the box half extents
// without their margin) the ellipse's left edge at height dy is
//   x_l(dy) = -(b/a) dy - sqrt(k (1 - dy^2 / ry^2) / a)
// (and x_r with + sqrt), convex (concave) in dy, extreme at
// dy = +-(b/c) rx.  Over the pixel rows of tile row ty the reached columns
// therefore run from x_l at the clamped leftmost dy to x_r at the clamped
// rightmost dy.  k gets 0.2% and x, y half a pixel of slack, so every pixel
// whose single-precision alpha can reach alpha_min lies in a counted tile.
// Both the tile count (slice/project) and the emitted pairs (bin_sort) come
// from this one function on the same record values.
struct EllipseRows {
    float u, v, ba, ia, ks, rys, irys, dyl;
    bool exact;  // false: degenerate shape, every tile of the box rect is kept
};

__device__ __forceinline__ EllipseRows ellipse_rows(const SplatView& r, float ln_alpha_min) {
    EllipseRows e;
    e.u = r.u;
    e.v = r.v;
    constexpr float kSlack = 1.002f;
    constexpr float kSqrtSlack = 1.0009995f;  // sqrt(kSlack)
    const float k = support_k(r.alpha_eff, ln_alpha_min);
    const float rx = r.hx - 0.5f, ry = r.hy - 0.5f;
    e.exact = r.a > 0.0f && r.c > 0.0f && rx > 0.0f && ry > 0.0f && k > 0.0f;
    e.ia = e.exact ? rcp_approx(r.a) : 0.0f;
    e.ba = e.exact ? __fmul_rn(r.b, e.ia) : 0.0f;
    e.ks = __fmul_rn(k, kSlack);
    e.rys = __fmul_rn(ry, kSqrtSlack);
    e.irys = e.exact ? rcp_approx(e.rys) : 0.0f;
    e.dyl = e.exact ? __fmul_rn(__fmul_rn(__fmul_rn(r.b, rcp_approx(r.c)), rx), kSqrtSlack) : 0.0f;
    return e;
}

// Pixel columns [*px0, *px1] reached by the ellipse over the pixel rows
// row_lo..row_hi (integers, within the image), clamped to the image; false
// when it reaches none of them.  Needs e.exact.
__device__ __forceinline__ bool ellipse_row_span(const EllipseRows& e, const DevView& V, float row_lo, float row_hi,
                                                 float* px0, float* px1) {
    const float lo = fmaxf(row_lo - 0.5f - e.v, -e.rys), hi = fminf(row_hi + 0.5f - e.v, e.rys);
    if (!(lo <= hi)) return false;
    const float yl = fminf(fmaxf(e.dyl, lo), hi), yr = fminf(fmaxf(-e.dyl, lo), hi);
    const float ql = yl * e.irys, qr = yr * e.irys;
    // explicit fused operations: every kernel that walks these spans (the
    // pair count, the pair scatter, the raster masks) rounds them alike
    const float xl = __fmaf_rn(-e.ba, yl, -sqrt_approx(fmaxf(e.ks * __fmaf_rn(-ql, ql, 1.0f), 0.0f) * e.ia));
    const float xr = __fmaf_rn(-e.ba, yr, sqrt_approx(fmaxf(e.ks * __fmaf_rn(-qr, qr, 1.0f), 0.0f) * e.ia));
    *px0 = fmaxf(ceilf(e.u + xl - 0.5f), 0.0f);
    *px1 = fminf(floorf(e.u + xr + 0.5f), (float)(V.width - 1));
    return *px0 <= *px1;
}

// Tiles [*tx0, *tx0 + count) of tile row ty reached by the ellipse, within
// the box rect (x0, y0, x1, y1).  tile is 16, 32 or 64.
__device__ __forceinline__ int ellipse_row_tiles(const EllipseRows& e, const DevView& V, int tile, const int* rect,
                                                 int ty, int* tx0) {
    *tx0 = rect[0];
    if (!e.exact) return rect[2] - rect[0] + 1;
    const int sh = __ffs(tile) - 1;
    const float row_lo = (float)(ty << sh), row_hi = (float)min((ty << sh) + tile - 1, V.height - 1);
    float px0, px1;
    if (!ellipse_row_span(e, V, row_lo, row_hi, &px0, &px1)) return 0;
    const int t0 = max((int)px0 >> sh, rect[0]), t1 = min((int)px1 >> sh, rect[2]);
    *tx0 = t0;
    return max(t1 - t0 + 1, 0);
}

__device__ __forceinline__ int ellipse_tiles(const SplatView& r, float ln_alpha_min, const DevView& V, int tile,
                                             const int* rect) {
    const EllipseRows e = ellipse_rows(r, ln_alpha_min);
    int n = 0;
    for (int ty = rect[1]; ty <= rect[3]; ty++) {
        int tx0;
        n += ellipse_row_tiles(e, V, tile, rect, ty, &tx0);
    }
    return n;
}

// Camera transform, Jacobian, 2D covariance, conic, support box and tile rect.
// Returns false when the splat is culled (near plane, alpha_eff, empty rect).
__device__ __forceinline__ bool project_view(const Core& c, const DevView& V, const DevOpts& O, ViewGeom& w,
                                             bool allow_f64) {
    w.tiles = 0;
#pragma unroll
    for (int i = 0; i < 3; i++)
        w.xc[i] = fmaf(V.W[i * 3 + 0], w.mu3[0], fmaf(V.W[i * 3 + 1], w.mu3[1], fmaf(V.W[i * 3 + 2], w.mu3[2], V.tau[i])));
    const float Z = w.xc[2];
    if (!(Z >= O.near_z)) return false;
    const float iz = 1.0f / Z;
    float tx = w.xc[0] * iz, ty = w.xc[1] * iz;
    w.u = fmaf(V.fx, tx, V.cx);
    w.v = fmaf(V.fy, ty, V.cy);
    w.clx = false;
    w.cly = false;
    if (tx < -V.limx) { tx = -V.limx; w.clx = true; }
    if (tx > V.limx) { tx = V.limx; w.clx = true; }
    if (ty < -V.limy) { ty = -V.limy; w.cly = true; }
    if (ty > V.limy) { ty = V.limy; w.cly = true; }
    const float J00 = V.fx * iz, J02 = -V.fx * tx * iz, J11 = V.fy * iz, J12 = -V.fy * ty * iz;
#pragma unroll
    for (int k = 0; k < 3; k++) {
        w.T[k] = fmaf(J00, V.W[0 * 3 + k], J02 * V.W[2 * 3 + k]);
        w.T[3 + k] = fmaf(J11, V.W[1 * 3 + k], J12 * V.W[2 * 3 + k]);
    }
    // Sigma_2d = T Sigma3 T^T + delta I
    const float* S = w.S3;
    float TS[2][3];
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const float* t = &w.T[3 * r];
        TS[r][0] = t[0] * S[0] + t[1] * S[1] + t[2] * S[2];
        TS[r][1] = t[0] * S[1] + t[1] * S[3] + t[2] * S[4];
        TS[r][2] = t[0] * S[2] + t[1] * S[4] + t[2] * S[5];
    }
    w.cov[0] = TS[0][0] * w.T[0] + TS[0][1] * w.T[1] + TS[0][2] * w.T[2] + O.dilation;
    w.cov[1] = TS[0][0] * w.T[3] + TS[0][1] * w.T[4] + TS[0][2] * w.T[5];
    w.cov[2] = TS[1][0] * w.T[3] + TS[1][1] * w.T[4] + TS[1][2] * w.T[5] + O.dilation;
    float det = w.cov[0] * w.cov[2] - w.cov[1] * w.cov[1];
    if (allow_f64 && det < O.conic_cond * w.cov[0] * w.cov[2]) {
        // ill-conditioned 2x2: recompute covariance, determinant and inverse in FP64
        double Td[6], Sd[6];
        for (int i = 0; i < 6; i++) { Td[i] = w.T[i]; Sd[i] = w.S3[i]; }
        double TSd[2][3];
        for (int r = 0; r < 2; r++) {
            const double* t = &Td[3 * r];
            TSd[r][0] = t[0] * Sd[0] + t[1] * Sd[1] + t[2] * Sd[2];
            TSd[r][1] = t[0] * Sd[1] + t[1] * Sd[3] + t[2] * Sd[4];
            TSd[r][2] = t[0] * Sd[2] + t[1] * Sd[4] + t[2] * Sd[5];
        }
        const double c00 = TSd[0][0] * Td[0] + TSd[0][1] * Td[1] + TSd[0][2] * Td[2] + (double)O.dilation;
        const double c01 = TSd[0][0] * Td[3] + TSd[0][1] * Td[4] + TSd[0][2] * Td[5];
        const double c11 = TSd[1][0] * Td[3] + TSd[1][1] * Td[4] + TSd[1][2] * Td[5] + (double)O.dilation;
        const double dd = c00 * c11 - c01 * c01;
        if (!(dd > 0.0)) return false;
        w.cov[0] = (float)c00;
        w.cov[1] = (float)c01;
        w.cov[2] = (float)c11;
        w.conic[0] = (float)(c11 / dd);
        w.conic[1] = (float)(-c01 / dd);
        w.conic[2] = (float)(c00 / dd);
        det = (float)dd;
    } else {
        if (!(det > 0.0f)) return false;
        const float idet = 1.0f / det;
        w.conic[0] = w.cov[2] * idet;
        w.conic[1] = -w.cov[1] * idet;
        w.conic[2] = w.cov[0] * idet;
    }
    w.alpha_eff = c.alpha * w.p;
    if (!(w.alpha_eff >= O.alpha_min)) return false;
    // Support box: alpha_eff * G >= alpha_min needs d^T Sigma2d^-1 d <= 2 ln(alpha_eff /
    // alpha_min) =: k, and d^T Sigma2d^-1 d >= dx^2 / Sigma2d_00 (Cauchy-Schwarz), so
    // |dx| <= sqrt(k Sigma2d_00) and |dy| <= sqrt(k Sigma2d_11), plus half a pixel margin.
    const float k2 = 2.0f * fmaxf(logf(w.alpha_eff) - O.ln_alpha_min, 0.0f);
    w.hx = sqrtf(k2 * w.cov[0]) + 0.5f;
    w.hy = sqrtf(k2 * w.cov[2]) + 0.5f;
    w.tiles = box_tiles(w.u, w.v, w.hx, w.hy, V, O.bin, w.rect);
    return w.tiles > 0;
}

// Unit view direction from the camera centre to the conditional mean.
__device__ __forceinline__ float view_dir(const ViewGeom& w, const DevView& V, float* d) {
    const float e0 = w.mu3[0] - V.campos[0], e1 = w.mu3[1] - V.campos[1], e2 = w.mu3[2] - V.campos[2];
    const float nrm = sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
    const float inv = 1.0f / nrm;
    d[0] = e0 * inv;
    d[1] = e1 * inv;
    d[2] = e2 * inv;
    return nrm;
}

// ---------------------------------------------------------------------------
// Host launchers (defined in the .cu files, called by the C ABI in api.cu).
// ---------------------------------------------------------------------------
cudaError_t launch_slice_project(const DevGauss& G, const ViewSet& VS, const DevOpts& O, const StateLayout& lay,
                                 char* state, uint32_t capacity, cudaStream_t st);
cudaError_t launch_bin_sort(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state, int sm_count,
                            cudaStream_t st, int* out_buf);
cudaError_t launch_render(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state, int pair_buf,
                          float* image, float* final_T, int32_t* n_last, cudaStream_t st);
cudaError_t launch_sample_split(const DevGauss& G, const int64_t* index, const float* z, int64_t m, float* out,
                                cudaStream_t st);
cudaError_t launch_render_aux(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state, int pair_buf,
                              float* aux_image, cudaStream_t st);
cudaError_t launch_render_stats(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state,
                                int pair_buf, float* image, float* final_T, int32_t* n_last,
                                unsigned long long* stats, cudaStream_t st);
cudaError_t launch_render_backward(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state,
                                   int pair_buf, const float* final_T, const int32_t* n_last, const float* dL_dimage,
                                   cudaStream_t st);
cudaError_t launch_project_backward(const DevGauss& G, const ViewSet& VS, const DevOpts& O, const StateLayout& lay,
                                    char* state, const fgs4d_gaussian_grads& grads, cudaStream_t st);

// number of radix passes etc. needed by the host to know which buffer holds the result
int pair_sort_bits(uint32_t total_tiles);
int radix_passes(int bits);

// Variants of the two backward launchers that take the per-splat 2D gradient
// buffer explicitly instead of the state's section.
cudaError_t launch_render_backward_into(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state,
                                        int pair_buf, const float* final_T, const int32_t* n_last,
                                        const float* dL_dimage, float4* g2, cudaStream_t st);
cudaError_t launch_project_backward_from(const DevGauss& G, const ViewSet& VS, const DevOpts& O,
                                         const StateLayout& lay, char* state, float4* g2, uint32_t* list,
                                         uint32_t* list_count, uint32_t* scan_tmp,
                                         const fgs4d_gaussian_grads& grads, cudaStream_t st);

// Gaussian-major list (g, then view) of the splats with tiles_touched > 0, as
// splat ids v n + g; its length goes to *count.  scan_tmp: kScanBlocksMax + 32 words.
cudaError_t compact_visible_gaussian_major(const uint32_t* tiles, uint32_t n, uint32_t V, uint32_t* list,
                                           uint32_t* count, uint32_t* scan_tmp, int sm_count, cudaStream_t st);

// Host-side count of kernel launches issued by this library (all threads).
void count_launches(unsigned k);

}  // namespace fgs4d
