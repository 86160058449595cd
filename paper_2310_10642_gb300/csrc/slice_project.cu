// slice_project.cu -- per-Gaussian kernels of the 4DGS rendering routine.
//
// slice_project_kernel (forward): for each Gaussian and each view of the
// batch, Eq. 7-8 (covariance from the quaternion pair), Eq. 9-10 (conditional
// 3D Gaussian, marginal p(t) and the p(t) < p_min filter of Sec. 4.2),
// Eq. 11 (4D spherindrical-harmonic colour) and Eq. 3-4 (EWA projection),
// written as one splat record per (view, Gaussian) (48 bytes, or 32 with
// 16-bit conics).  One thread per Gaussian over all views; a block stages its
// Gaussians' 4DSH coefficients in shared memory for the views to share.
//
// project_backward_kernel (adjoint): the chain rule from the per-splat 2D
// gradient (written by the compositing adjoint) back to the raw parameters,
// one thread per visible splat of a Gaussian-major list; the splats of one
// Gaussian sum their contributions over the warp and its first lane runs
// Eq. 7-8 backwards once.  sh_backward_kernel then forms the 4DSH
// coefficient gradients, one thread per (Gaussian, channel), from the colour
// cotangents the adjoint leaves per splat.
#include <algorithm>

#include "fgs4d_internal.cuh"

namespace fgs4d {

// One coefficient: from global memory through the read-only data cache, or
// (kShared) a plain load from the shared-memory copy.
template <bool kShared, class T>
__device__ __forceinline__ float load_coef(const T* p) {
    if constexpr (kShared)
        return to_float(*p);
    else
        return to_float(__ldg(p));
}

// Coefficients of Gaussian g: row r at sh[r * n]; one address increment per
// row (row stride n), the storage type resolved outside the loops.
template <int L, bool kShared, class T>
__device__ __forceinline__ void color_sum(const T* __restrict__ sh, size_t n, int K, float dt_scaled, const float* Y,
                                          float* raw) {
    constexpr int NB = (L + 1) * (L + 1);
    raw[0] = raw[1] = raw[2] = 0.0f;
    for (int f = 0; f <= K; f++) {
        const float cf = cospif((float)f * dt_scaled);
        const T* row = sh + (size_t)(f * NB * 3) * n;
#pragma unroll
        for (int j = 0; j < NB; j++) {
            const float b = cf * Y[j];
            raw[0] = fmaf(b, load_coef<kShared>(row), raw[0]);
            raw[1] = fmaf(b, load_coef<kShared>(row + n), raw[1]);
            raw[2] = fmaf(b, load_coef<kShared>(row + 2 * n), raw[2]);
            row += 3 * n;
        }
    }
}

constexpr int kSliceThreads = 128;
// A block stages its Gaussians' 4DSH coefficients in shared memory (one
// column per thread, rows as in global memory) when they fit in this many
// bytes, so that the views after the first read them on chip.
constexpr int kSliceStageBytes = 48 * 1024;

// staged: the coefficients of this thread's Gaussian are column threadIdx.x
// of a [rows][kSliceThreads] array in shared memory.
template <int L>
__device__ __forceinline__ void color_forward(const DevGauss& G, int g, const ViewGeom& w, const DevView& V,
                                              const void* staged, float* raw) {
    float d[3];
    view_dir(w, V, d);
    float Y[16];
    sh_eval(L, d[0], d[1], d[2], Y);
    const float dts = 2.0f * w.dt * G.inv_period;
    if (staged) {
        if (G.shs_bf16)
            color_sum<L, true>(reinterpret_cast<const __nv_bfloat16*>(staged) + threadIdx.x, (size_t)kSliceThreads,
                               G.K, dts, Y, raw);
        else
            color_sum<L, true>(reinterpret_cast<const float*>(staged) + threadIdx.x, (size_t)kSliceThreads, G.K, dts,
                               Y, raw);
    } else if (G.shs_bf16) {
        color_sum<L, false>(reinterpret_cast<const __nv_bfloat16*>(G.shs) + g, (size_t)G.n, G.K, dts, Y, raw);
    } else {
        color_sum<L, false>(reinterpret_cast<const float*>(G.shs) + g, (size_t)G.n, G.K, dts, Y, raw);
    }
}

// Copies the coefficient rows of Gaussian g into column threadIdx.x of dst
// (coalesced: row r of the block's Gaussians is contiguous in global memory).
template <class T>
__device__ __forceinline__ void stage_coefficients(const T* __restrict__ src, size_t n, int rows, T* dst) {
    for (int r = 0; r < rows; r++) dst[r * kSliceThreads] = src[(size_t)r * n];
}

// Colour part of the adjoint for one splat (Eq. 11): per channel the raw
// colour, its clamp, the cotangent graw, and the sums wsum_j = sum_ch graw P_j
// (P_j = sum_f cos_f k_fj) and ddt = sum_ch graw sum_f dcos_f/ddt kY_f that the
// direction and time gradients need.  cos/sin of the orders by angle addition.
template <int L, class T>
__device__ __forceinline__ void color_adjoint(const T* __restrict__ sh, size_t n, int K, float c1, float s1,
                                              float inv_period, const float* Y, const float* dcol, float* wsum,
                                              float& ddt, float* graws) {
    constexpr int NB = (L + 1) * (L + 1);
    for (int ch = 0; ch < 3; ch++) {
        float P[16];
#pragma unroll
        for (int j = 0; j < NB; j++) P[j] = 0.0f;
        float Q = 0.0f;
        float cf = 1.0f, sf = 0.0f;
        const T* row = sh + (size_t)ch * n;
        for (int f = 0; f <= K; f++) {
            const float om = 6.283185307179586f * (float)f * inv_period;
            float kY = 0.0f;
#pragma unroll
            for (int j = 0; j < NB; j++) {
                const float k = to_float(__ldg(row));
                row += 3 * n;
                P[j] = fmaf(cf, k, P[j]);
                kY = fmaf(k, Y[j], kY);
            }
            Q = fmaf(-om * sf, kY, Q);
            const float cn = fmaf(cf, c1, -sf * s1);
            sf = fmaf(sf, c1, cf * s1);
            cf = cn;
        }
        float raw = 0.0f;
#pragma unroll
        for (int j = 0; j < NB; j++) raw = fmaf(P[j], Y[j], raw);
        const float graw = (raw + 0.5f > 0.0f) ? dcol[ch] : 0.0f;
        graws[ch] = graw;
        if (graw != 0.0f) {
#pragma unroll
            for (int j = 0; j < NB; j++) wsum[j] = fmaf(graw, P[j], wsum[j]);
            ddt = fmaf(graw, Q, ddt);
        }
    }
}

// 5 blocks per SM (96 registers, no spills): one more than 128 registers allow
template <int L, int kMode>
__global__ void __launch_bounds__(kSliceThreads, 5) slice_project_kernel(
    const DevGauss G, const __grid_constant__ ViewSet VS, const DevOpts O, SplatRecord* __restrict__ rec,  // or SplatRecordH
    uint32_t* __restrict__ tiles_touched, uint32_t* __restrict__ depth_key, uint32_t* __restrict__ counters,
    float4* __restrict__ aux, int stage) {
    extern __shared__ __align__(16) unsigned char s_coef[];  // [rows][kSliceThreads] when stage != 0
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G.n) return;  // no barrier below: a thread reads only its own column
    const size_t n = (size_t)G.n;
    const void* staged = nullptr;
    if (stage) {
        const int rows = 3 * (L + 1) * (L + 1) * (G.K + 1);
        if (G.shs_bf16)
            stage_coefficients(reinterpret_cast<const __nv_bfloat16*>(G.shs) + g, n, rows,
                               reinterpret_cast<__nv_bfloat16*>(s_coef) + threadIdx.x);
        else
            stage_coefficients(reinterpret_cast<const float*>(G.shs) + g, n, rows,
                               reinterpret_cast<float*>(s_coef) + threadIdx.x);
        staged = s_coef;
    }
    Core c;
    load_core<kMode>(G, g, c);
    if (!c.ok) {
        atomicOr(&counters[2], FGS4D_STATUS_NONFINITE);
        for (int v = 0; v < VS.n; v++) tiles_touched[(size_t)v * n + g] = 0u;
        return;
    }
    for (int v = 0; v < VS.n; v++) {
        const DevView& V = VS.v[v];
        const size_t idx = (size_t)v * n + g;
        ViewGeom w;
        slice_view<kMode>(c, V, O, G, g, w, true);
        const bool vis = (w.p >= O.p_min) && project_view(c, V, O, w, true);
        if (!vis) {
            tiles_touched[idx] = 0u;
            continue;
        }
        float raw[3];
        color_forward<L>(G, g, w, V, staged, raw);
        float col[3];
#pragma unroll
        for (int ch = 0; ch < 3; ch++) col[ch] = fmaxf(raw[ch] + 0.5f, 0.0f);
        // tiles_touched here is the support box's tile count: the visibility flag of the
        // compaction; bin_sort replaces it by the support ellipse's count for the visible splats
        if (O.record_fp16) {
            const SplatRecordH h = encode_record_h(w.u, w.v, w.conic, w.cov[2], w.alpha_eff, col);
            // the box of the stored (16-bit) conic, exactly as bin_sort will decode it
            const SplatView d = decode_record(h, O.ln_alpha_min);
            w.tiles = box_tiles(d.u, d.v, d.hx, d.hy, V, O.bin, w.rect);
            if (w.tiles == 0) {
                tiles_touched[idx] = 0u;
                continue;
            }
            reinterpret_cast<SplatRecordH*>(rec)[idx] = h;
        } else {
            SplatRecord r;
            r.r0 = make_float4(w.u, w.v, w.conic[0], w.conic[1]);
            r.r1 = make_float4(w.conic[2], w.alpha_eff, col[0], col[1]);
            r.r2 = make_float4(col[2], w.xc[2], w.hx, w.hy);
            rec[idx] = r;
        }
        tiles_touched[idx] = (uint32_t)w.tiles;
        depth_key[idx] = __float_as_uint(w.xc[2]);
        if (aux && kMode != kRot4D) {  // block-diagonal Sigma: the conditional mean does not move
            aux[idx] = make_float4(w.xc[2], 0.0f, 0.0f, 0.0f);
        } else if (aux) {
            // Eq. 9: mu_{xyz|t} moves by Sigma_{xyz,t} / Sigma_tt per unit of t; the flow is the
            // displacement of its projection over flow_dt (0 where the moved mean is behind the camera)
            const float k = O.flow_dt / c.S[15];
            float xm[3];
#pragma unroll
            for (int i = 0; i < 3; i++) {
                const float m = fmaf(c.S[4 * i + 3], k, w.mu3[i]);
                xm[i] = m;
            }
            float xc2[3];
#pragma unroll
            for (int i = 0; i < 3; i++)
                xc2[i] = fmaf(V.W[i * 3 + 0], xm[0], fmaf(V.W[i * 3 + 1], xm[1], fmaf(V.W[i * 3 + 2], xm[2], V.tau[i])));
            float fu = 0.0f, fv = 0.0f;
            if (xc2[2] > 0.0f) {
                fu = fmaf(V.fx, xc2[0] / xc2[2], V.cx) - w.u;
                fv = fmaf(V.fy, xc2[1] / xc2[2], V.cy) - w.v;
            }
            aux[idx] = make_float4(w.xc[2], fu, fv, 0.0f);
        }
    }
}

// ---------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------
constexpr int kBwdThreads = 128;

// Sum of x over the caller's segment of contiguous lanes; the result is exact
// in the segment's first lane (seg_last = last lane of the segment).
__device__ __forceinline__ float segment_sum(float x, int lane, int seg_last) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float y = __shfl_down_sync(0xffffffffu, x, off);
        if (lane + off <= seg_last) x += y;
    }
    return x;
}

// Geometry part of the adjoint, one thread per visible (Gaussian, view) splat
// taken from a Gaussian-major list, so that lanes do not idle on views where
// their Gaussian is invisible.  The splats of one Gaussian sit in adjacent
// lanes; their contributions to dL/dSigma (4x4), dL/dmu, dL/dalpha are summed
// over the segment and its first lane runs Eq. 7-8 backwards once and adds the
// result to the (pre-zeroed) outputs.  Each splat's 2D-gradient slot is
// replaced by its colour cotangent, read by sh_backward_kernel:
//   slot[0] = (view direction d, dt),  slot[1] = (dL/draw_R, dL/draw_G, dL/draw_B, 0)
// where dL/draw is dL/dcolour with the colour clamp max(raw + 0.5, 0) applied.
// Eq. 7-8 backwards for one Gaussian: Sigma = M M^T, M = R S, R = L(q_l) R(q_r)
// (or blockdiag(R3(q_l), 1) without 4D rotation).  GS: dL/dSigma with its
// upper triangle filled (symmetrised here); galpha: dL/dsigmoid(logit).
// Writes the gradients of log s, q_l, q_r and the opacity logit.
template <int kMode>
__device__ __forceinline__ void covariance_chain(const DevGauss& G, const Core& cl, float* GS, float galpha,
                                                 float* gls, float* gql, float* gqr, float& glogit) {
#pragma unroll
    for (int i = 0; i < 4; i++) gls[i] = gql[i] = gqr[i] = 0.0f;
    // symmetrise the accumulator (only the upper triangle was written)
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < i; j++) GS[i * 4 + j] = GS[j * 4 + i];
    if constexpr (kMode != kRot4D) {
        // Sigma = blockdiag(M3 M3^T, s_t^2), M3 = R3(q) diag(s_xyz): the 3x3 block,
        // then dL/dlog s_t = 2 s_t^2 dL/dSigma_tt (zero without a time axis)
        float dR[9];
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int k = 0; k < 3; k++) {
                const float dM = 2.0f * fmaf(GS[i * 4 + 0], cl.M[0 * 4 + k],
                                             fmaf(GS[i * 4 + 1], cl.M[1 * 4 + k], GS[i * 4 + 2] * cl.M[2 * 4 + k]));
                dR[i * 3 + k] = dM * cl.s[k];
                gls[k] = fmaf(dM, cl.R[i * 4 + k], gls[k]);
            }
#pragma unroll
        for (int k = 0; k < 3; k++) gls[k] *= cl.s[k];
        gls[3] = kMode == kRotStatic ? 0.0f : 2.0f * GS[15] * cl.M[15] * cl.M[15];
        const float w = cl.qln[0], x = cl.qln[1], y = cl.qln[2], z = cl.qln[3];
        const float* d = dR;  // row-major 3x3
        const float gw = 2.0f * (-z * d[1] + y * d[2] + z * d[3] - x * d[5] - y * d[6] + x * d[7]);
        const float gx = 2.0f * (y * d[1] + z * d[2] + y * d[3] - 2.0f * x * d[4] - w * d[5] + z * d[6] +
                                 w * d[7] - 2.0f * x * d[8]);
        const float gy = 2.0f * (-2.0f * y * d[0] + x * d[1] + w * d[2] + x * d[3] + z * d[5] - w * d[6] +
                                 z * d[7] - 2.0f * y * d[8]);
        const float gz = 2.0f * (-2.0f * z * d[0] - w * d[1] + x * d[2] + w * d[3] - 2.0f * z * d[4] +
                                 y * d[5] + x * d[6] + y * d[7]);
        const float gq[4] = {gw, gx, gy, gz};
        float dq = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; i++) dq = fmaf(gq[i], cl.qln[i], dq);
#pragma unroll
        for (int i = 0; i < 4; i++) gql[i] = (gq[i] - dq * cl.qln[i]) / cl.nl;
        glogit = galpha * cl.alpha * (1.0f - cl.alpha);
        return;
    }
    float dR[16];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int k = 0; k < 4; k++) {
            float acc = 0.0f;
#pragma unroll
            for (int j = 0; j < 4; j++) acc = fmaf(GS[i * 4 + j], cl.M[j * 4 + k], acc);
            const float dM = 2.0f * acc;
            dR[i * 4 + k] = dM * cl.s[k];
            gls[k] = fmaf(dM, cl.R[i * 4 + k], gls[k]);
        }
#pragma unroll
    for (int k = 0; k < 4; k++) gls[k] *= cl.s[k];
    float Lm[16], Rm[16];
    left_matrix(cl.qln, Lm);
    right_matrix(cl.qrn, Rm);
    float D[16], E[16];  // D = dR Rm^T, E = Lm^T dR
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) {
            float x = 0.0f, y = 0.0f;
#pragma unroll
            for (int k = 0; k < 4; k++) {
                x = fmaf(dR[i * 4 + k], Rm[j * 4 + k], x);
                y = fmaf(Lm[k * 4 + i], dR[k * 4 + j], y);
            }
            D[i * 4 + j] = x;
            E[i * 4 + j] = y;
        }
    const float gl[4] = {D[0] + D[5] + D[10] + D[15], -D[1] + D[4] - D[11] + D[14],
                         -D[2] + D[7] + D[8] - D[13], -D[3] - D[6] + D[9] + D[12]};
    const float gr[4] = {E[0] + E[5] + E[10] + E[15], -E[1] + E[4] + E[11] - E[14],
                         -E[2] - E[7] + E[8] + E[13], -E[3] + E[6] - E[9] + E[12]};
    float dl = 0.0f, dr = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        dl = fmaf(gl[i], cl.qln[i], dl);
        dr = fmaf(gr[i], cl.qrn[i], dr);
    }
#pragma unroll
    for (int i = 0; i < 4; i++) {
        gql[i] = (gl[i] - dl * cl.qln[i]) / cl.nl;
        gqr[i] = (gr[i] - dr * cl.qrn[i]) / cl.nr;
    }
    glogit = galpha * cl.alpha * (1.0f - cl.alpha);
}

// Rows of the per-Gaussian scratch the deferred chain reads: the ten upper
// entries of dL/dSigma (row i of kGsumEntry: Sigma element index) and
// dL/dsigmoid(logit) in row 10.
constexpr int kGsumRows = 11;
__device__ constexpr int kGsumEntry[10] = {0, 1, 2, 3, 5, 6, 7, 10, 11, 15};

// kDefer: add the per-Gaussian sums to gsum ([kGsumRows][n], zeroed) and
// leave Eq. 7-8 to covariance_chain_kernel; else each segment's first lane
// runs it (gsum unused).
template <int L, bool kDefer, int kMode>
__global__ void __launch_bounds__(kBwdThreads, 4) project_backward_kernel(
    const DevGauss G, const __grid_constant__ ViewSet VS, const DevOpts O, float4* __restrict__ grad2d,
    const uint32_t* __restrict__ list, const uint32_t* __restrict__ list_count, const fgs4d_gaussian_grads out,
    float* __restrict__ gsum) {
    constexpr int NB = (L + 1) * (L + 1);
    const uint32_t count = *list_count;
    const int lane = threadIdx.x & 31;
    const uint32_t warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    const size_t n = (size_t)G.n;
    for (uint32_t base = warp0 * 32; base < count; base += n_warps * 32) {  // warp-uniform
        const uint32_t e = base + lane;
        const bool active = e < count;
        const uint32_t sid = active ? list[e] : 0u;
        const int g = (int)(sid % (uint32_t)n);
        const int v = (int)(sid / (uint32_t)n);
        const uint32_t key = active ? (uint32_t)g : (0x80000000u | (uint32_t)lane);
        const uint32_t peers = __match_any_sync(0xffffffffu, key);
        const int seg_first = __ffs(peers) - 1, seg_last = 31 - __clz(peers);

        float gmu[4] = {0, 0, 0, 0};
        float GS[16];
#pragma unroll
        for (int i = 0; i < 16; i++) GS[i] = 0.0f;
        float galpha = 0.0f, m2d = 0.0f, mt = 0.0f;
        Core c;
        c.ok = false;
        if (active) load_core<kMode>(G, g, c);
        if (active && c.ok) {
            const float sig = c.S[15];
            const size_t idx = sid;
            const DevView& V = VS.v[v];
            ViewGeom w;
            slice_view<kMode>(c, V, O, G, g, w, true);
            if (!project_view(c, V, O, w, true)) {  // cannot happen for a binned splat; keep the slot defined
                grad2d[3 * idx + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                const float4 q0 = grad2d[3 * idx + 0];
                const float4 q1 = grad2d[3 * idx + 1];
                const float4 q2 = grad2d[3 * idx + 2];
                const float du = q0.x, dv = q0.y, da = q0.z, db = q0.w, dc = q1.x, dae = q1.y;
                const float dcol[3] = {q1.z, q1.w, q2.x};
                m2d += sqrtf(du * du + dv * dv);

                // ---- colour (Eq. 11) ----
                float d[3];
                const float nrm = view_dir(w, V, d);
                float Y[16];
                sh_eval(L, d[0], d[1], d[2], Y);
                float wsum[16];
    #pragma unroll
                for (int j = 0; j < NB; j++) wsum[j] = 0.0f;
                float ddt = 0.0f;
                float graws[3];
                const float arg1 = 2.0f * w.dt * G.inv_period;  // 0 for a static Gaussian
                const float c1 = cospif(arg1), s1 = sinpif(arg1);
                if (G.shs_bf16)
                    color_adjoint<L>(reinterpret_cast<const __nv_bfloat16*>(G.shs) + g, n, G.K, c1, s1,
                                     G.inv_period, Y, dcol, wsum, ddt, graws);
                else
                    color_adjoint<L>(reinterpret_cast<const float*>(G.shs) + g, n, G.K, c1, s1, G.inv_period, Y,
                                     dcol, wsum, ddt, graws);
                // colour cotangent for the coefficient gradients (sh_backward_kernel)
                grad2d[3 * idx + 0] = make_float4(d[0], d[1], d[2], w.dt);
                grad2d[3 * idx + 1] = make_float4(graws[0], graws[1], graws[2], 0.0f);
                float gd[3];
                sh_grad(L, d[0], d[1], d[2], wsum, gd[0], gd[1], gd[2]);
                const float gdd = gd[0] * d[0] + gd[1] * d[1] + gd[2] * d[2];
                float dmu3[3];
                const float inrm = 1.0f / nrm;
    #pragma unroll
                for (int i = 0; i < 3; i++) dmu3[i] = (gd[i] - gdd * d[i]) * inrm;

                // ---- conic -> 2D covariance: G2 = -Q Gc Q ----
                const float a = w.conic[0], bq = w.conic[1], cq = w.conic[2];
                const float g00 = da, g01 = 0.5f * db, g11 = dc;
                // QG = Q * Gc
                const float qg00 = a * g00 + bq * g01, qg01 = a * g01 + bq * g11;
                const float qg10 = bq * g00 + cq * g01, qg11 = bq * g01 + cq * g11;
                const float G200 = -(qg00 * a + qg01 * bq);
                const float G201 = -(qg00 * bq + qg01 * cq);
                const float G211 = -(qg10 * bq + qg11 * cq);

                // ---- Eq. 4: dSigma3 = T^T G2 T, dT = 2 G2 T Sigma3 ----
                const float* T = w.T;
                float GT[2][3];
    #pragma unroll
                for (int k = 0; k < 3; k++) {
                    GT[0][k] = G200 * T[k] + G201 * T[3 + k];
                    GT[1][k] = G201 * T[k] + G211 * T[3 + k];
                }
                float G3[6];  // 00 01 02 11 12 22
                G3[0] = T[0] * GT[0][0] + T[3] * GT[1][0];
                G3[1] = T[0] * GT[0][1] + T[3] * GT[1][1];
                G3[2] = T[0] * GT[0][2] + T[3] * GT[1][2];
                G3[3] = T[1] * GT[0][1] + T[4] * GT[1][1];
                G3[4] = T[1] * GT[0][2] + T[4] * GT[1][2];
                G3[5] = T[2] * GT[0][2] + T[5] * GT[1][2];
                const float* S3 = w.S3;
                float dT[2][3];
    #pragma unroll
                for (int r = 0; r < 2; r++) {
                    dT[r][0] = 2.0f * (GT[r][0] * S3[0] + GT[r][1] * S3[1] + GT[r][2] * S3[2]);
                    dT[r][1] = 2.0f * (GT[r][0] * S3[1] + GT[r][1] * S3[3] + GT[r][2] * S3[4]);
                    dT[r][2] = 2.0f * (GT[r][0] * S3[2] + GT[r][1] * S3[4] + GT[r][2] * S3[5]);
                }
                // dJ = dT W^T
                float dJ[2][3];
    #pragma unroll
                for (int r = 0; r < 2; r++)
    #pragma unroll
                    for (int m = 0; m < 3; m++)
                        dJ[r][m] = dT[r][0] * V.W[m * 3 + 0] + dT[r][1] * V.W[m * 3 + 1] + dT[r][2] * V.W[m * 3 + 2];

                // ---- J and the projected mean w.r.t. camera coordinates ----
                const float X = w.xc[0], Yc = w.xc[1], Z = w.xc[2];
                const float iz = 1.0f / Z, iz2 = iz * iz;
                float tx = X * iz, ty = Yc * iz;
                tx = fminf(fmaxf(tx, -V.limx), V.limx);
                ty = fminf(fmaxf(ty, -V.limy), V.limy);
                float dxc[3] = {0.0f, 0.0f, 0.0f};
                dxc[2] += dJ[0][0] * (-V.fx * iz2) + dJ[1][1] * (-V.fy * iz2);
                dxc[2] += dJ[0][2] * (V.fx * tx * iz2) + dJ[1][2] * (V.fy * ty * iz2);
                if (!w.clx) {
                    dxc[0] += dJ[0][2] * (-V.fx * iz2);
                    dxc[2] += dJ[0][2] * (V.fx * X * iz2 * iz);
                }
                if (!w.cly) {
                    dxc[1] += dJ[1][2] * (-V.fy * iz2);
                    dxc[2] += dJ[1][2] * (V.fy * Yc * iz2 * iz);
                }
                dxc[0] += du * V.fx * iz;
                dxc[1] += dv * V.fy * iz;
                dxc[2] += -du * V.fx * X * iz2 - dv * V.fy * Yc * iz2;
    #pragma unroll
                for (int i = 0; i < 3; i++)
                    dmu3[i] += V.W[0 * 3 + i] * dxc[0] + V.W[1 * 3 + i] * dxc[1] + V.W[2 * 3 + i] * dxc[2];

                // ---- Eq. 9, Eq. 10 ----
                const float dp = dae * c.alpha;
                galpha += dae * w.p;
                if constexpr (kMode == kRot4D) {
                    const float b[3] = {c.S[3], c.S[7], c.S[11]};
                    const float isig = 1.0f / sig;
                    float G3b[3];
                    G3b[0] = G3[0] * b[0] + G3[1] * b[1] + G3[2] * b[2];
                    G3b[1] = G3[1] * b[0] + G3[3] * b[1] + G3[4] * b[2];
                    G3b[2] = G3[2] * b[0] + G3[4] * b[1] + G3[5] * b[2];
                    const float mb = dmu3[0] * b[0] + dmu3[1] * b[1] + dmu3[2] * b[2];
                    const float bGb = b[0] * G3b[0] + b[1] * G3b[1] + b[2] * G3b[2];
                    const float dt = w.dt;
                    const float dsig = (-mb * dt + bGb + dp * w.p * 0.5f * dt * dt) * isig * isig;
                    ddt += mb * isig - dp * w.p * dt * isig;
    #pragma unroll
                    for (int i = 0; i < 3; i++) {
                        const float dbi = (dmu3[i] * dt - 2.0f * G3b[i]) * isig;
                        GS[i * 4 + 3] += 0.5f * dbi;
                    }
                    GS[15] += dsig;
                } else if constexpr (kMode == kRotSpatial) {
                    // no coupling: the mean and the spatial covariance do not depend on t;
                    // p = exp(-dt^2 / (2 s_t^2)) alone carries the time
                    const float isig = 1.0f / sig, dt = w.dt;
                    GS[15] += dp * w.p * 0.5f * dt * dt * isig * isig;
                    ddt += -dp * w.p * dt * isig;
                } else {
                    ddt = 0.0f;  // static: no time axis
                }
                mt = fabsf(ddt);  // this view's |dL/dmu_t|
    #pragma unroll
                for (int i = 0; i < 3; i++) gmu[i] += dmu3[i];
                gmu[3] -= ddt;
                GS[0] += G3[0];
                GS[1] += G3[1];
                GS[2] += G3[2];
                GS[5] += G3[3];
                GS[6] += G3[4];
                GS[10] += G3[5];
            }
        }
        // ---- sum the segment (all visible views of this Gaussian in this warp) ----
        gmu[0] = segment_sum(gmu[0], lane, seg_last);
        gmu[1] = segment_sum(gmu[1], lane, seg_last);
        gmu[2] = segment_sum(gmu[2], lane, seg_last);
        gmu[3] = segment_sum(gmu[3], lane, seg_last);
        GS[0] = segment_sum(GS[0], lane, seg_last);
        GS[1] = segment_sum(GS[1], lane, seg_last);
        GS[2] = segment_sum(GS[2], lane, seg_last);
        GS[3] = segment_sum(GS[3], lane, seg_last);
        GS[5] = segment_sum(GS[5], lane, seg_last);
        GS[6] = segment_sum(GS[6], lane, seg_last);
        GS[7] = segment_sum(GS[7], lane, seg_last);
        GS[10] = segment_sum(GS[10], lane, seg_last);
        GS[11] = segment_sum(GS[11], lane, seg_last);
        GS[15] = segment_sum(GS[15], lane, seg_last);
        galpha = segment_sum(galpha, lane, seg_last);
        m2d = segment_sum(m2d, lane, seg_last);
        mt = segment_sum(mt, lane, seg_last);
        if (!(active && c.ok && lane == seg_first)) continue;
        if constexpr (kDefer) {
            // add the segment's sums; Eq. 7-8 runs once per Gaussian, with every lane busy, in
            // covariance_chain_kernel (the sums of a Gaussian split over two warps add up there)
#pragma unroll
            for (int i = 0; i < 10; i++) atomicAdd(&gsum[i * n + g], GS[kGsumEntry[i]]);
            atomicAdd(&gsum[10 * n + g], galpha);
#pragma unroll
            for (int i = 0; i < 4; i++) atomicAdd(&out.mu[i * n + g], gmu[i]);
            if (out.mean2d_abs) atomicAdd(&out.mean2d_abs[g], m2d);
            if (out.mu_t_abs) atomicAdd(&out.mu_t_abs[g], mt);
            continue;  // the rest is not compiled into this instance
        }
        // The leader rebuilds the rotation chain from the parameters, so that R, M and the
        // quaternions are not live across the per-splat part above.
        Core cl;
        load_core<kMode>(G, g, cl);

        // ---- Eq. 7-8 once per Gaussian: Sigma = M M^T, M = R S, R = L(q_l) R(q_r) ----
        float gls[4] = {0, 0, 0, 0}, gql[4] = {0, 0, 0, 0}, gqr[4] = {0, 0, 0, 0}, glogit = 0.0f;
        if (c.ok) {
            covariance_chain<kMode>(G, cl, GS, galpha, gls, gql, gqr, glogit);
        } else {
    #pragma unroll
            for (int i = 0; i < 4; i++) gmu[i] = 0.0f;
        }
        // a Gaussian whose views straddle two warps is completed by two leaders: add, do not store
#pragma unroll
        for (int i = 0; i < 4; i++) {
            atomicAdd(&out.mu[i * n + g], gmu[i]);
            atomicAdd(&out.log_scale[i * n + g], gls[i]);
            atomicAdd(&out.q_left[i * n + g], gql[i]);
            if (kMode == kRot4D) atomicAdd(&out.q_right[i * n + g], gqr[i]);
        }
        atomicAdd(&out.opacity_logit[g], glogit);
        if (out.mean2d_abs) atomicAdd(&out.mean2d_abs[g], m2d);
        if (out.mu_t_abs) atomicAdd(&out.mu_t_abs[g], mt);
    }
}

// Eq. 7-8 backwards, one thread per Gaussian, from the sums the projection
// adjoint left in gsum (all zero: no visible splat, gradients stay zero).
// The outputs were zeroed (or hold the sums to add to) and each Gaussian has
// one thread.
template <int kMode>
__global__ void __launch_bounds__(256) covariance_chain_kernel(const DevGauss G, const float* __restrict__ gsum,
                                                               const fgs4d_gaussian_grads out, int accumulate) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G.n) return;
    const size_t n = (size_t)G.n;
    float GS[16];
    bool any = false;
#pragma unroll
    for (int i = 0; i < 10; i++) {
        GS[kGsumEntry[i]] = gsum[i * n + g];
        any = any || GS[kGsumEntry[i]] != 0.0f;
    }
    const float galpha = gsum[10 * n + g];
    if (!any && galpha == 0.0f) return;
    Core cl;
    load_core<kMode>(G, g, cl);
    if (!cl.ok) return;
    float gls[4], gql[4], gqr[4], glogit;
    covariance_chain<kMode>(G, cl, GS, galpha, gls, gql, gqr, glogit);
    // one thread per Gaussian: plain stores, or atomic adds when accumulating (calls on
    // other states may add into the same outputs concurrently)
    auto put = [accumulate](float* p, float v) {
        if (accumulate)
            atomicAdd(p, v);
        else
            *p = v;
    };
#pragma unroll
    for (int i = 0; i < 4; i++) {
        put(&out.log_scale[i * n + g], gls[i]);
        put(&out.q_left[i * n + g], gql[i]);
        if (kMode == kRot4D) put(&out.q_right[i * n + g], gqr[i]);
    }
    put(&out.opacity_logit[g], glogit);
}

// Coefficient part of the adjoint (Eq. 11): dL/dk[f][j][ch] = sum over the
// visible views of dL/draw_ch cos(2 pi f dt / T) Y_j(d), from the colour
// cotangents left by project_backward_kernel.  One thread per (Gaussian,
// channel) keeps the (K+1) (L+1)^2 sums in registers; consecutive threads take
// consecutive Gaussians, so every load and store is coalesced.
template <int L, int K1>
__global__ void __launch_bounds__(256, 4) sh_backward_kernel(int n, int n_views, float inv_period,
                                                          const float4* __restrict__ grad2d, float* __restrict__ gshs,
                                                          int accumulate) {
    constexpr int NB = (L + 1) * (L + 1);
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int ch = blockIdx.y;
    if (g >= n) return;
    float acc[K1][NB];
#pragma unroll
    for (int f = 0; f < K1; f++)
#pragma unroll
        for (int j = 0; j < NB; j++) acc[f][j] = 0.0f;
    // The 2D-gradient record of every splat is zeroed before the adjoint, and
    // only the splats it reached get a non-zero colour cotangent, so the
    // cotangent alone says which views to take (the loads of several views
    // are in flight together).
#pragma unroll 4
    for (int v = 0; v < n_views; v++) {
        const size_t idx = (size_t)v * n + g;
        const float4 gr = grad2d[3 * idx + 1];
        const float graw = ch == 0 ? gr.x : (ch == 1 ? gr.y : gr.z);
        if (graw == 0.0f) continue;
        const float4 dd = grad2d[3 * idx + 0];
        float Y[16];
        sh_eval(L, dd.x, dd.y, dd.z, Y);
#pragma unroll
        for (int f = 0; f < K1; f++) {
            const float gc = graw * cospif(2.0f * (float)f * dd.w * inv_period);
#pragma unroll
            for (int j = 0; j < NB; j++) acc[f][j] = fmaf(gc, Y[j], acc[f][j]);
        }
    }
#pragma unroll
    for (int f = 0; f < K1; f++)
#pragma unroll
        for (int j = 0; j < NB; j++) {
            float* dst = gshs + (size_t)((f * NB + j) * 3 + ch) * n + g;
            if (!accumulate)
                *dst = acc[f][j];
            else if (acc[f][j] != 0.0f)
                atomicAdd(dst, acc[f][j]);
        }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
__global__ void init_counters_kernel(uint32_t* counters, uint32_t capacity) {
    counters[0] = 0u;  // visible splats
    counters[1] = 0u;  // pairs
    counters[2] = 0u;  // status bits
    counters[3] = capacity;
}

cudaError_t launch_slice_project(const DevGauss& G, const ViewSet& VS, const DevOpts& O, const StateLayout& lay,
                                 char* state, uint32_t capacity, cudaStream_t st) {
    uint32_t* counters = reinterpret_cast<uint32_t*>(state + lay.counters);
    init_counters_kernel<<<1, 1, 0, st>>>(counters, capacity);
    count_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (G.n == 0) return cudaSuccess;
    const int threads = kSliceThreads;
    const int blocks = (G.n + threads - 1) / threads;
    // stage the coefficients on chip when more than one view reads them and they fit
    const size_t stage_bytes = (size_t)3 * (G.L + 1) * (G.L + 1) * (G.K + 1) * threads *
                               (G.shs_bf16 ? sizeof(__nv_bfloat16) : sizeof(float));
    const int stage = VS.n > 1 && stage_bytes <= (size_t)kSliceStageBytes;
    const size_t smem = stage ? stage_bytes : 0;
    auto* rec = reinterpret_cast<SplatRecord*>(state + lay.records);
    auto* tt = reinterpret_cast<uint32_t*>(state + lay.tiles_touched);
    auto* dk = reinterpret_cast<uint32_t*>(state + lay.depth_key);
    auto* aux = O.aux ? reinterpret_cast<float4*>(state + lay.aux) : nullptr;
    auto go = [&](auto kernel) { kernel<<<blocks, threads, smem, st>>>(G, VS, O, rec, tt, dk, counters, aux, stage); };
    switch (G.L * 3 + G.rot) {
        case 0: go(slice_project_kernel<0, kRot4D>); break;
        case 1: go(slice_project_kernel<0, kRotSpatial>); break;
        case 2: go(slice_project_kernel<0, kRotStatic>); break;
        case 3: go(slice_project_kernel<1, kRot4D>); break;
        case 4: go(slice_project_kernel<1, kRotSpatial>); break;
        case 5: go(slice_project_kernel<1, kRotStatic>); break;
        case 6: go(slice_project_kernel<2, kRot4D>); break;
        case 7: go(slice_project_kernel<2, kRotSpatial>); break;
        case 8: go(slice_project_kernel<2, kRotStatic>); break;
        case 9: go(slice_project_kernel<3, kRot4D>); break;
        case 10: go(slice_project_kernel<3, kRotSpatial>); break;
        default: go(slice_project_kernel<3, kRotStatic>); break;
    }
    count_launches(1);
    return cudaGetLastError();
}

template <int L, int K1>
static void launch_sh(const DevGauss& G, int n_views, const float4* g2, float* gshs, int acc, cudaStream_t st) {
    const dim3 grid((G.n + 255) / 256, 3);
    sh_backward_kernel<L, K1><<<grid, 256, 0, st>>>(G.n, n_views, G.inv_period, g2, gshs, acc);
}

template <int L>
static void launch_sh_k(const DevGauss& G, int n_views, const float4* g2, float* gshs, int acc, cudaStream_t st) {
    switch (G.K) {
        case 0: launch_sh<L, 1>(G, n_views, g2, gshs, acc, st); break;
        case 1: launch_sh<L, 2>(G, n_views, g2, gshs, acc, st); break;
        case 2: launch_sh<L, 3>(G, n_views, g2, gshs, acc, st); break;
        case 3: launch_sh<L, 4>(G, n_views, g2, gshs, acc, st); break;
        default: launch_sh<L, 5>(G, n_views, g2, gshs, acc, st); break;
    }
}

static int local_sm_count() {
    static int count = 0;
    if (count == 0) {
        int dev = 0, c = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && c > 0)
            count = c;
        else
            return 152;
    }
    return count;
}

// Adjoint of slice/project/4DSH: Gaussian-major list of the visible splats,
// geometry kernel over that list (outputs accumulated, so cleared first),
// then the coefficient kernel.
template <int L, int kMode>
static cudaError_t launch_pb(const DevGauss& G, const ViewSet& VS, const DevOpts& O, const uint32_t* tt, float4* g2,
                            uint32_t* list, uint32_t* list_count, uint32_t* scan_tmp, float* gsum,
                            const fgs4d_gaussian_grads& grads, cudaStream_t st) {
    const size_t n = (size_t)G.n;
    cudaError_t e = cudaSuccess;
    if (!O.accumulate) {  // accumulating: the outputs hold the sums to add to
        float* outs[5] = {grads.mu, grads.log_scale, grads.q_left, grads.q_right, grads.opacity_logit};
        const size_t rows[5] = {4, 4, 4, 4, 1};
        for (int i = 0; i < 5 && e == cudaSuccess; i++)
            e = cudaMemsetAsync(outs[i], 0, rows[i] * n * sizeof(float), st);
        if (e == cudaSuccess && grads.mean2d_abs) e = cudaMemsetAsync(grads.mean2d_abs, 0, n * sizeof(float), st);
        if (e == cudaSuccess && grads.mu_t_abs) e = cudaMemsetAsync(grads.mu_t_abs, 0, n * sizeof(float), st);
    }
    if (e == cudaSuccess && gsum) e = cudaMemsetAsync(gsum, 0, kGsumRows * n * sizeof(float), st);
    if (e != cudaSuccess) return e;
    const int sms = local_sm_count();
    e = compact_visible_gaussian_major(tt, (uint32_t)n, (uint32_t)VS.n, list, list_count, scan_tmp, sms, st);
    if (e != cudaSuccess) return e;
    const uint64_t S = (uint64_t)n * VS.n;
    const int blocks = (int)std::max<uint64_t>(1, std::min<uint64_t>((S + kBwdThreads - 1) / kBwdThreads, 16ull * sms));
    if (gsum) {
        project_backward_kernel<L, true, kMode>
            <<<blocks, kBwdThreads, 0, st>>>(G, VS, O, g2, list, list_count, grads, gsum);
        covariance_chain_kernel<kMode><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(G, gsum, grads, O.accumulate);
        count_launches(1);
    } else {
        project_backward_kernel<L, false, kMode>
            <<<blocks, kBwdThreads, 0, st>>>(G, VS, O, g2, list, list_count, grads, nullptr);
    }
    launch_sh_k<L>(G, VS.n, g2, grads.shs, O.accumulate, st);
    count_launches(2);
    return cudaGetLastError();
}

static cudaError_t launch_pb_any(const DevGauss& G, const ViewSet& VS, const DevOpts& O, const uint32_t* tt,
                                 float4* g2, uint32_t* list, uint32_t* list_count, uint32_t* scan_tmp, float* gsum,
                                 const fgs4d_gaussian_grads& grads, cudaStream_t st) {
#define FGS4D_PB(l, m) return launch_pb<l, m>(G, VS, O, tt, g2, list, list_count, scan_tmp, gsum, grads, st)
    switch (G.L * 3 + G.rot) {
        case 0: FGS4D_PB(0, kRot4D);
        case 1: FGS4D_PB(0, kRotSpatial);
        case 2: FGS4D_PB(0, kRotStatic);
        case 3: FGS4D_PB(1, kRot4D);
        case 4: FGS4D_PB(1, kRotSpatial);
        case 5: FGS4D_PB(1, kRotStatic);
        case 6: FGS4D_PB(2, kRot4D);
        case 7: FGS4D_PB(2, kRotSpatial);
        case 8: FGS4D_PB(2, kRotStatic);
        case 9: FGS4D_PB(3, kRot4D);
        case 10: FGS4D_PB(3, kRotSpatial);
        default: FGS4D_PB(3, kRotStatic);
    }
#undef FGS4D_PB
}

// The list of visible splats goes to the state's pair-offset section (free
// once the tiles are binned) and its length to counters[4].
cudaError_t launch_project_backward(const DevGauss& G, const ViewSet& VS, const DevOpts& O, const StateLayout& lay,
                                    char* state, const fgs4d_gaussian_grads& grads, cudaStream_t st) {
    if (G.n == 0) return cudaSuccess;
    auto* tt = reinterpret_cast<const uint32_t*>(state + lay.tiles_touched);
    auto* g2 = reinterpret_cast<float4*>(state + lay.grad2d);
    auto* list = reinterpret_cast<uint32_t*>(state + lay.offsets);
    auto* cnt = reinterpret_cast<uint32_t*>(state + lay.counters) + 4;
    auto* scan_tmp = reinterpret_cast<uint32_t*>(state + lay.scan_tmp);
    auto* gsum = reinterpret_cast<float*>(state + lay.gsum);
    return launch_pb_any(G, VS, O, tt, g2, list, cnt, scan_tmp, gsum, grads, st);
}

// Same as launch_project_backward with the per-splat 2D gradient, the list,
// its length and the scan scratch supplied by the caller (used by the
// allocation-free backward entry point, which does not write the state).
cudaError_t launch_project_backward_from(const DevGauss& G, const ViewSet& VS, const DevOpts& O,
                                         const StateLayout& lay, char* state, float4* g2, uint32_t* list,
                                         uint32_t* list_count, uint32_t* scan_tmp,
                                         const fgs4d_gaussian_grads& grads, cudaStream_t st) {
    if (G.n == 0) return cudaSuccess;
    auto* tt = reinterpret_cast<const uint32_t*>(state + lay.tiles_touched);
    // the state is input only on this path: each segment's first lane runs Eq. 7-8 itself
    return launch_pb_any(G, VS, O, tt, g2, list, list_count, scan_tmp, nullptr, grads, st);
}

// Split sampling in 4D (Sec. 3.4): new means drawn from a Gaussian's own 4D
// density, x = mu + M z with M = R diag(s) (so that M M^T = Sigma, Eq. 7-8)
// and z ~ N(0, I) supplied by the caller.  One thread per sample; index[j]
// names the Gaussian, z and out are [4][m].  A Gaussian with non-finite or
// zero-norm parameters yields NaN.
template <int kMode>
__global__ void __launch_bounds__(256) sample_split_kernel(const DevGauss G, const int64_t* __restrict__ index,
                                                           const float* __restrict__ z, int64_t m,
                                                           float* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const int64_t gi = index[j];
    if (gi < 0 || gi >= G.n) {
#pragma unroll
        for (int i = 0; i < 4; i++) out[i * m + j] = __int_as_float(0x7fc00000);
        return;
    }
    Core c;
    load_core<kMode>(G, (int)gi, c);
    float zz[4];
#pragma unroll
    for (int k = 0; k < 4; k++) zz[k] = z[k * m + j];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        float x = c.mu[i];
#pragma unroll
        for (int k = 0; k < 4; k++) x = fmaf(c.M[i * 4 + k], zz[k], x);
        out[i * m + j] = c.ok ? x : __int_as_float(0x7fc00000);
    }
}

cudaError_t launch_sample_split(const DevGauss& G, const int64_t* index, const float* z, int64_t m, float* out,
                                cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((m + 255) / 256);
    if (G.rot == kRot4D)
        sample_split_kernel<kRot4D><<<blocks, 256, 0, st>>>(G, index, z, m, out);
    else if (G.rot == kRotSpatial)
        sample_split_kernel<kRotSpatial><<<blocks, 256, 0, st>>>(G, index, z, m, out);
    else
        sample_split_kernel<kRotStatic><<<blocks, 256, 0, st>>>(G, index, z, m, out);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace fgs4d
