// api.cu -- the C ABI of libfgs4d (declared in include/fgs4d.h).
//
// Host-side argument checking, the per-frame state layout, the view set
// passed by value to every kernel, and the launch sequence of each entry
// point.  No entry point allocates device memory or synchronises, except
// fgs4d_read_counters.
#include <float.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "fgs4d_internal.cuh"

using namespace fgs4d;

namespace fgs4d {
static std::atomic<uint64_t> g_launches{0};
void count_launches(unsigned k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace fgs4d

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

fgs4d_status check_options(const fgs4d_options* o) {
    if (!o) return FGS4D_ERR_INVALID_ARG;
    const float vals[] = {o->p_min, o->near_z, o->alpha_min, o->alpha_max, o->T_min, o->dilation, o->clamp_fov,
                          o->schur_cond, o->conic_cond};
    for (float v : vals)
        if (!isfinite(v) || v < 0.0f) return FGS4D_ERR_INVALID_ARG;
    if (!(o->alpha_min > 0.0f && o->alpha_min <= o->alpha_max && o->alpha_max < 1.0f)) return FGS4D_ERR_INVALID_ARG;
    if (!(o->near_z > 0.0f) || o->p_min > 1.0f || o->T_min >= 1.0f) return FGS4D_ERR_INVALID_ARG;
    if (o->record_fp16 != 0 && o->record_fp16 != 1) return FGS4D_ERR_INVALID_ARG;
    if (o->tile_size != 16 && o->tile_size != 32) return FGS4D_ERR_INVALID_ARG;
    if (o->bin_size != 0 && ((o->bin_size != 16 && o->bin_size != 32 && o->bin_size != 64) ||
                             o->bin_size % o->tile_size != 0))
        return FGS4D_ERR_INVALID_ARG;
    if (o->batch_depth != 32 && o->batch_depth != 64 && o->batch_depth != 128 && o->batch_depth != 256)
        return FGS4D_ERR_INVALID_ARG;
    if (o->aux_channels != 0 && o->aux_channels != 1) return FGS4D_ERR_INVALID_ARG;
    if (!isfinite(o->flow_dt)) return FGS4D_ERR_INVALID_ARG;
    if (o->accumulate_grads != 0 && o->accumulate_grads != 1) return FGS4D_ERR_INVALID_ARG;
    return FGS4D_OK;
}

DevOpts dev_options(const fgs4d_options* o) {
    DevOpts d;
    d.p_min = o->p_min;
    d.near_z = o->near_z;
    d.alpha_min = o->alpha_min;
    d.alpha_max = o->alpha_max;
    d.T_min = o->T_min;
    d.dilation = o->dilation;
    d.schur_cond = o->schur_cond;
    d.conic_cond = o->conic_cond;
    d.ln_alpha_min = logf(o->alpha_min);
    d.record_fp16 = o->record_fp16;
    d.tile = o->tile_size;
    d.bin = o->bin_size ? o->bin_size : o->tile_size;
    d.batch = o->batch_depth;
    d.aux = o->aux_channels;
    d.flow_dt = o->flow_dt;
    d.accumulate = o->accumulate_grads;
    return d;
}

// Builds the view set; checks sizes.  clamp_fov from the options.
fgs4d_status make_views(const fgs4d_view* views, int n_views, const fgs4d_options* o, ViewSet* VS) {
    if (!views || n_views < 1 || n_views > FGS4D_MAX_VIEWS) return FGS4D_ERR_INVALID_ARG;
    memset(VS, 0, sizeof(*VS));
    VS->n = n_views;
    uint64_t tiles = 0, pix = 0;
    for (int i = 0; i < n_views; i++) {
        const fgs4d_view& h = views[i];
        DevView& d = VS->v[i];
        if (h.width < 1 || h.height < 1 || h.width > 16384 || h.height > 16384) return FGS4D_ERR_INVALID_ARG;
        for (int k = 0; k < 12; k++)
            if (!isfinite(h.viewmat[k])) return FGS4D_ERR_INVALID_ARG;
        if (!(isfinite(h.fx) && isfinite(h.fy) && isfinite(h.cx) && isfinite(h.cy) && isfinite(h.t)) ||
            !(h.fx > 0.0f && h.fy > 0.0f))
            return FGS4D_ERR_INVALID_ARG;
        for (int r = 0; r < 3; r++) {
            for (int c = 0; c < 3; c++) d.W[r * 3 + c] = h.viewmat[r * 4 + c];
            d.tau[r] = h.viewmat[r * 4 + 3];
        }
        for (int c = 0; c < 3; c++) {
            double acc = 0.0;
            for (int r = 0; r < 3; r++) acc -= (double)d.W[r * 3 + c] * (double)d.tau[r];
            d.campos[c] = (float)acc;
            d.bg[c] = h.bg[c];
        }
        d.fx = h.fx;
        d.fy = h.fy;
        d.cx = h.cx;
        d.cy = h.cy;
        d.t = h.t;
        if (o->clamp_fov > 0.0f) {
            d.limx = o->clamp_fov * 0.5f * (float)h.width / h.fx;
            d.limy = o->clamp_fov * 0.5f * (float)h.height / h.fy;
        } else {
            d.limx = FLT_MAX;
            d.limy = FLT_MAX;
        }
        d.width = h.width;
        d.height = h.height;
        const int bin = o->bin_size ? o->bin_size : o->tile_size;
        d.tiles_x = (h.width + bin - 1) / bin;
        d.tiles_y = (h.height + bin - 1) / bin;
        d.tile_base = (uint32_t)tiles;
        d.pix_base = (uint32_t)pix;
        tiles += (uint64_t)d.tiles_x * d.tiles_y;
        pix += (uint64_t)h.width * h.height;
    }
    if (tiles > 0x7fffffffull || pix > 0x7fffffffull) return FGS4D_ERR_INVALID_ARG;
    VS->total_tiles = (uint32_t)tiles;
    return FGS4D_OK;
}

// Lays out the state for n Gaussians and the views; capacity < 0 means
// "derive it from state_bytes".
fgs4d_status make_layout(int64_t n, const ViewSet& VS, int record_fp16, int aux, int64_t capacity,
                         size_t state_bytes, StateLayout* L) {
    if (n < 0) return FGS4D_ERR_INVALID_ARG;
    const int64_t S = n * (int64_t)VS.n;
    if (S >= 0x7fffffffll) return FGS4D_ERR_INVALID_ARG;
    memset(L, 0, sizeof(*L));
    L->n_splats = S;
    L->record_bytes = record_fp16 ? sizeof(SplatRecordH) : sizeof(SplatRecord);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    const size_t s = (size_t)S;
    L->counters = take(16 * sizeof(uint32_t));
    L->records = take(s * L->record_bytes);
    L->tiles_touched = take(s * 4);
    L->depth_key = take(s * 4);
    L->sort_keys[0] = take(s * 4);
    L->sort_keys[1] = take(s * 4);
    L->sort_vals[0] = take(s * 4);
    L->sort_vals[1] = take(s * 4);
    L->offsets = take(s * 4);
    L->scan_tmp = take((kScanBlocksMax + 32) * 4);
    L->hist = take(((size_t)kMaxDigits * kSortBlocksMax + kMaxDigits) * 4);
    L->ranges = take((size_t)VS.total_tiles * 8);
    L->grad2d = take(s * 48);
    L->aux = aux ? take(s * 16) : 0;
    L->gsum = take((size_t)n * 11 * sizeof(float));
    // Pair binning path: the counting sort keeps one uint32 counter per
    // (binning tile, chunk of a view's depth-ordered visible splats) and one
    // pair array; the radix path keys and values, double-buffered.
    uint32_t tmax = 0;
    for (int i = 0; i < VS.n; i++) tmax = std::max(tmax, (uint32_t)(VS.v[i].tiles_x * VS.v[i].tiles_y));
    L->view_tiles_max = tmax;
    L->count_sort = n > 0 && tmax <= kCountTilesMax;
    if (L->count_sort) {
        // chunks of 256 splats unless the counters would pass 2^26 entries
        uint32_t C = 256;
        while ((uint64_t)VS.total_tiles * (uint64_t)((n + C - 1) / C) > (1ull << 26) && C < (1u << 20)) C <<= 1;
        L->chunk = C;
        L->chunks_per_view = (uint32_t)((n + C - 1) / C);
        if ((uint64_t)VS.total_tiles * L->chunks_per_view >= (1ull << 31)) L->count_sort = 0;  // 32-bit scan
        else L->chunk_hist = take((size_t)VS.total_tiles * L->chunks_per_view * 4);
    }
    L->fixed_bytes = off;
    const int arrays = L->count_sort ? 1 : 4;  // uint32 arrays of `capacity`
    if (capacity < 0) {
        if (state_bytes < L->fixed_bytes) return FGS4D_ERR_CAPACITY;
        // each array padded to the alignment
        int64_t cap = (int64_t)((state_bytes - L->fixed_bytes) / (4 * arrays));
        while (cap > 0 && L->fixed_bytes + arrays * align_up((size_t)cap * 4) > state_bytes) cap--;
        capacity = cap;
    }
    if (capacity > 0xffffffffll) capacity = 0xffffffffll;
    L->capacity = capacity;
    const size_t pb = align_up((size_t)capacity * 4);
    if (L->count_sort) {
        L->pair_keys[0] = L->pair_keys[1] = L->pair_vals[0] = L->pair_vals[1] = off;
        L->total = off + pb;
    } else {
        L->pair_keys[0] = off;
        L->pair_keys[1] = off + pb;
        L->pair_vals[0] = off + 2 * pb;
        L->pair_vals[1] = off + 3 * pb;
        L->total = off + 4 * pb;
    }
    return FGS4D_OK;
}

fgs4d_status check_gaussians(const fgs4d_gaussians* g, DevGauss* d) {
    if (!g) return FGS4D_ERR_INVALID_ARG;
    if (g->n < 0 || g->n >= 0x7fffffffll) return FGS4D_ERR_INVALID_ARG;
    if (g->sh_degree < 0 || g->sh_degree > FGS4D_MAX_SH_DEGREE || g->n_freq < 0 || g->n_freq > FGS4D_MAX_FREQ)
        return FGS4D_ERR_INVALID_ARG;
    if (!(g->period > 0.0f) || !isfinite(g->period)) return FGS4D_ERR_INVALID_ARG;
    if (g->shs_dtype != FGS4D_F32 && g->shs_dtype != FGS4D_BF16) return FGS4D_ERR_INVALID_ARG;
    if (g->rotation != FGS4D_ROT_4D && g->rotation != FGS4D_ROT_SPATIAL && g->rotation != FGS4D_ROT_STATIC)
        return FGS4D_ERR_INVALID_ARG;
    if (g->n > 0) {
        const void* ptrs[] = {g->mu, g->log_scale, g->q_left, g->opacity_logit, g->shs};
        for (const void* p : ptrs)
            if (!p || !aligned(p, 16)) return FGS4D_ERR_INVALID_ARG;
        if (g->rotation == FGS4D_ROT_4D && (!g->q_right || !aligned(g->q_right, 16))) return FGS4D_ERR_INVALID_ARG;
    }
    d->mu = g->mu;
    d->log_s = g->log_scale;
    d->ql = g->q_left;
    d->qr = g->q_right;
    d->logit = g->opacity_logit;
    d->shs = g->shs;
    d->n = (int)g->n;
    d->L = g->sh_degree;
    d->K = g->n_freq;
    d->inv_period = 1.0f / g->period;
    d->shs_bf16 = g->shs_dtype == FGS4D_BF16;
    d->rot = g->rotation;
    return FGS4D_OK;
}

struct Prepared {
    ViewSet VS;
    DevOpts O;
    StateLayout L;
};

fgs4d_status prepare(int64_t n, const fgs4d_view* views, int n_views, const fgs4d_options* opt, void* state,
                     size_t state_bytes, Prepared* P) {
    fgs4d_status s = check_options(opt);
    if (s != FGS4D_OK) return s;
    if (!state || !aligned(state, kAlign)) return FGS4D_ERR_INVALID_ARG;
    if ((s = make_views(views, n_views, opt, &P->VS)) != FGS4D_OK) return s;
    if ((s = make_layout(n, P->VS, opt->record_fp16, opt->aux_channels, -1, state_bytes, &P->L)) != FGS4D_OK)
        return s;
    P->O = dev_options(opt);
    return FGS4D_OK;
}

int sm_count_cached() {
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

fgs4d_status cuda_status(cudaError_t e) { return e == cudaSuccess ? FGS4D_OK : FGS4D_ERR_CUDA; }

}  // namespace

extern "C" {

int fgs4d_abi_version(void) { return FGS4D_ABI_VERSION; }

uint64_t fgs4d_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

const char* fgs4d_status_string(fgs4d_status s) {
    switch (s) {
        case FGS4D_OK: return "ok";
        case FGS4D_ERR_INVALID_ARG: return "invalid argument";
        case FGS4D_ERR_CAPACITY: return "state too small or pair capacity exceeded";
        case FGS4D_ERR_CUDA: return "CUDA error";
        case FGS4D_ERR_TIMEOUT: return "timeout";
        case FGS4D_ERR_NONFINITE: return "non-finite input or zero-norm quaternion";
    }
    return "unknown status";
}

void fgs4d_default_options(fgs4d_options* o) {
    if (!o) return;
    o->p_min = 0.05f;
    o->near_z = 0.2f;
    o->alpha_min = 1.0f / 255.0f;
    o->alpha_max = 0.99f;
    o->T_min = 1e-4f;
    o->dilation = 0.3f;
    o->clamp_fov = 1.3f;
    o->record_fp16 = 0;
    o->schur_cond = 1e-3f;
    o->conic_cond = 1e-4f;
    o->tile_size = FGS4D_TILE;
    o->batch_depth = 256;
    o->aux_channels = 0;
    o->flow_dt = 1.0f / 300.0f;
    o->bin_size = 0;
    o->accumulate_grads = 0;
}

int64_t fgs4d_total_pixels(const fgs4d_view* views, int n_views) {
    if (!views || n_views < 0) return -1;
    int64_t p = 0;
    for (int i = 0; i < n_views; i++) p += (int64_t)views[i].width * views[i].height;
    return p;
}

fgs4d_status fgs4d_state_size(int64_t n, const fgs4d_view* views, int n_views, int64_t pair_capacity,
                              const fgs4d_options* opt, size_t* bytes) {
    if (!bytes || pair_capacity < 0 || pair_capacity > 0xffffffffll) return FGS4D_ERR_INVALID_ARG;
    fgs4d_status s = check_options(opt);
    if (s != FGS4D_OK) return s;
    ViewSet VS;
    s = make_views(views, n_views, opt, &VS);
    StateLayout L;
    if (s == FGS4D_OK) s = make_layout(n, VS, opt->record_fp16, opt->aux_channels, pair_capacity, 0, &L);
    if (s != FGS4D_OK) return s;
    *bytes = L.total;
    return FGS4D_OK;
}

fgs4d_status fgs4d_slice_project(const fgs4d_gaussians* g, const fgs4d_view* views, int n_views,
                                 const fgs4d_options* opt, void* state, size_t state_bytes, fgs4d_stream stream) {
    DevGauss G;
    fgs4d_status s = check_gaussians(g, &G);
    if (s != FGS4D_OK) return s;
    Prepared prep;
    Prepared* P = &prep;
    s = prepare(g->n, views, n_views, opt, state, state_bytes, P);
    if (s == FGS4D_OK) {
        char* st = static_cast<char*>(state);
        cudaError_t e = launch_slice_project(G, P->VS, P->O, P->L, st, (uint32_t)P->L.capacity,
                                             (cudaStream_t)stream);
        s = cuda_status(e);
    }
    return s;
}

fgs4d_status fgs4d_bin_sort(int64_t n, const fgs4d_view* views, int n_views, const fgs4d_options* opt, void* state,
                            size_t state_bytes, fgs4d_stream stream) {
    Prepared prep;
    Prepared* P = &prep;
    fgs4d_status s = prepare(n, views, n_views, opt, state, state_bytes, P);
    if (s == FGS4D_OK) {
        int buf = 0;
        s = cuda_status(launch_bin_sort(P->VS, P->O, P->L, static_cast<char*>(state), sm_count_cached(),
                                        (cudaStream_t)stream, &buf));
    }
    return s;
}

static int pair_buffer(const Prepared& P) {
    if (P.L.capacity == 0 || P.L.count_sort) return 0;
    return radix_passes(pair_sort_bits(P.VS.total_tiles + 1)) & 1;
}

fgs4d_status fgs4d_render(int64_t n, const fgs4d_view* views, int n_views, const fgs4d_options* opt, void* state,
                          size_t state_bytes, float* image, float* final_T, int32_t* n_last, fgs4d_stream stream) {
    if (!image || !final_T || !n_last) return FGS4D_ERR_INVALID_ARG;
    if (!aligned(image, 4) || !aligned(final_T, 4) || !aligned(n_last, 4)) return FGS4D_ERR_INVALID_ARG;
    Prepared prep;
    Prepared* P = &prep;
    fgs4d_status s = prepare(n, views, n_views, opt, state, state_bytes, P);
    if (s == FGS4D_OK)
        s = cuda_status(launch_render(P->VS, P->O, P->L, static_cast<char*>(state), pair_buffer(*P), image, final_T,
                                      n_last, (cudaStream_t)stream));
    return s;
}

fgs4d_status fgs4d_sample_split(const fgs4d_gaussians* g, const int64_t* index, const float* z, int64_t m,
                                float* out_mu, fgs4d_stream stream) {
    DevGauss G;
    fgs4d_status s = check_gaussians(g, &G);
    if (s != FGS4D_OK) return s;
    if (m < 0 || (m > 0 && (!index || !z || !out_mu))) return FGS4D_ERR_INVALID_ARG;
    if (!aligned(index, 8) || !aligned(z, 4) || !aligned(out_mu, 4)) return FGS4D_ERR_INVALID_ARG;
    return cuda_status(launch_sample_split(G, index, z, m, out_mu, (cudaStream_t)stream));
}

fgs4d_status fgs4d_render_aux(int64_t n, const fgs4d_view* views, int n_views, const fgs4d_options* opt, void* state,
                              size_t state_bytes, float* aux_image, fgs4d_stream stream) {
    if (!aux_image || !aligned(aux_image, 4) || !opt || opt->aux_channels != 1) return FGS4D_ERR_INVALID_ARG;
    Prepared prep;
    Prepared* P = &prep;
    fgs4d_status s = prepare(n, views, n_views, opt, state, state_bytes, P);
    if (s == FGS4D_OK)
        s = cuda_status(launch_render_aux(P->VS, P->O, P->L, static_cast<char*>(state), pair_buffer(*P), aux_image,
                                          (cudaStream_t)stream));
    return s;
}

fgs4d_status fgs4d_render_stats(int64_t n, const fgs4d_view* views, int n_views, const fgs4d_options* opt,
                                void* state, size_t state_bytes, float* image, float* final_T, int32_t* n_last,
                                uint64_t* stats, fgs4d_stream stream) {
    if (!image || !final_T || !n_last || !stats) return FGS4D_ERR_INVALID_ARG;
    if (!aligned(image, 4) || !aligned(final_T, 4) || !aligned(n_last, 4) || !aligned(stats, 8))
        return FGS4D_ERR_INVALID_ARG;
    Prepared prep;
    Prepared* P = &prep;
    fgs4d_status s = prepare(n, views, n_views, opt, state, state_bytes, P);
    if (s == FGS4D_OK)
        s = cuda_status(launch_render_stats(P->VS, P->O, P->L, static_cast<char*>(state), pair_buffer(*P), image,
                                            final_T, n_last, reinterpret_cast<unsigned long long*>(stats),
                                            (cudaStream_t)stream));
    return s;
}

static fgs4d_status check_grads(const fgs4d_gaussians* g, const fgs4d_gaussian_grads* grads) {
    if (!grads) return FGS4D_ERR_INVALID_ARG;
    if (g->n > 0) {
        const void* ptrs[] = {grads->mu, grads->log_scale, grads->q_left, grads->q_right, grads->opacity_logit,
                              grads->shs};
        for (const void* p : ptrs)
            if (!p || !aligned(p, 4)) return FGS4D_ERR_INVALID_ARG;
    }
    return FGS4D_OK;
}

fgs4d_status fgs4d_render_backward(const fgs4d_gaussians* g, const fgs4d_view* views, int n_views,
                                   const fgs4d_options* opt, void* state, size_t state_bytes, const float* final_T,
                                   const int32_t* n_last, const float* dL_dimage, fgs4d_gaussian_grads* grads,
                                   fgs4d_stream stream) {
    DevGauss G;
    fgs4d_status s = check_gaussians(g, &G);
    if (s != FGS4D_OK) return s;
    if (!final_T || !n_last || !dL_dimage) return FGS4D_ERR_INVALID_ARG;
    if ((s = check_grads(g, grads)) != FGS4D_OK) return s;
    Prepared prep;
    Prepared* P = &prep;
    s = prepare(g->n, views, n_views, opt, state, state_bytes, P);
    if (s == FGS4D_OK) {
        char* st = static_cast<char*>(state);
        cudaError_t e = launch_render_backward(P->VS, P->O, P->L, st, pair_buffer(*P), final_T, n_last, dL_dimage,
                                               (cudaStream_t)stream);
        if (e == cudaSuccess) e = launch_project_backward(G, P->VS, P->O, P->L, st, *grads, (cudaStream_t)stream);
        s = cuda_status(e);
    }
    return s;
}

fgs4d_status fgs4d_render_backward_2d(int64_t n, const fgs4d_view* views, int n_views, const fgs4d_options* opt,
                                      void* state, size_t state_bytes, const float* final_T, const int32_t* n_last,
                                      const float* dL_dimage, fgs4d_stream stream) {
    if (!final_T || !n_last || !dL_dimage) return FGS4D_ERR_INVALID_ARG;
    if (!aligned(final_T, 4) || !aligned(n_last, 4) || !aligned(dL_dimage, 4)) return FGS4D_ERR_INVALID_ARG;
    Prepared prep;
    Prepared* P = &prep;
    fgs4d_status s = prepare(n, views, n_views, opt, state, state_bytes, P);
    if (s == FGS4D_OK)
        s = cuda_status(launch_render_backward(P->VS, P->O, P->L, static_cast<char*>(state), pair_buffer(*P), final_T,
                                               n_last, dL_dimage, (cudaStream_t)stream));
    return s;
}

fgs4d_status fgs4d_project_backward(const fgs4d_gaussians* g, const fgs4d_view* views, int n_views,
                                    const fgs4d_options* opt, void* state, size_t state_bytes,
                                    fgs4d_gaussian_grads* grads, fgs4d_stream stream) {
    DevGauss G;
    fgs4d_status s = check_gaussians(g, &G);
    if (s != FGS4D_OK) return s;
    if ((s = check_grads(g, grads)) != FGS4D_OK) return s;
    Prepared prep;
    Prepared* P = &prep;
    s = prepare(g->n, views, n_views, opt, state, state_bytes, P);
    if (s == FGS4D_OK)
        s = cuda_status(launch_project_backward(G, P->VS, P->O, P->L, static_cast<char*>(state), *grads,
                                                (cudaStream_t)stream));
    return s;
}

fgs4d_status fgs4d_state_layout(int64_t n, const fgs4d_view* views, int n_views, const fgs4d_options* opt,
                                size_t state_bytes, fgs4d_state_layout_info* out) {
    if (!out) return FGS4D_ERR_INVALID_ARG;
    fgs4d_status s = check_options(opt);
    if (s != FGS4D_OK) return s;
    Prepared prep;
    Prepared* P = &prep;
    s = make_views(views, n_views, opt, &P->VS);
    if (s == FGS4D_OK) s = make_layout(n, P->VS, opt->record_fp16, opt->aux_channels, -1, state_bytes, &P->L);
    if (s == FGS4D_OK) {
        out->counters = P->L.counters;
        out->records = P->L.records;
        out->tiles_touched = P->L.tiles_touched;
        out->ranges = P->L.ranges;
        out->pair_vals = P->L.pair_vals[pair_buffer(*P)];
        out->record_bytes = P->L.record_bytes;
        out->n_splats = (uint64_t)P->L.n_splats;
        out->total_tiles = P->VS.total_tiles;
        out->pair_capacity = (uint64_t)P->L.capacity;
        out->grad2d = P->L.grad2d;
    }
    return s;
}

fgs4d_status fgs4d_read_counters(const void* state, fgs4d_counters* out, fgs4d_stream stream) {
    if (!state || !out || !aligned(state, kAlign)) return FGS4D_ERR_INVALID_ARG;
    uint32_t h[4];
    cudaError_t e = cudaMemcpyAsync(h, state, sizeof(h), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return FGS4D_ERR_CUDA;
    out->n_visible = h[0];
    out->n_pairs = h[1];
    out->status = h[2];
    out->pair_capacity = h[3];
    return FGS4D_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// fgs4d_render_backward_noalloc: the backward pass without caller scratch.
//
// Some callers cannot call cudaMalloc at the moment they need the backward
// pass: real-time render loops that reserve every byte of device memory once
// at start-up and forbid later allocations, and plugins hosted by an engine
// that owns the device allocator.  This entry point keeps its scratch -- the
// per-splat 2D gradient (three float4 per (view, Gaussian) splat), the list
// of visible splats (one word per splat), its length and the scan's block
// sums -- in a static device array of this library instead of the caller's
// state.  The state from the forward pass is only read.  The array holds
// FGS4D_NOALLOC_MAX_SPLATS splats (13 MiB) and every GPU that loads this
// library keeps it until the process exits.  The host side allocates
// nothing either: the per-call view set and layout live on the stack.
// ---------------------------------------------------------------------------
#include <mutex>

constexpr size_t kNoallocGrad = 3 * (size_t)FGS4D_NOALLOC_MAX_SPLATS;   // float4: 2D gradients
constexpr size_t kNoallocList = (size_t)FGS4D_NOALLOC_MAX_SPLATS / 4;   // float4: splat list words
constexpr size_t kNoallocMisc = (kScanBlocksMax + 32 + 16) / 4;          // float4: scan sums, list length
static __device__ __align__(256) float4 g_noalloc_grad2d[kNoallocGrad + kNoallocList + kNoallocMisc];

namespace {

constexpr int kNoallocMaxDevices = 256;
std::mutex g_noalloc_mu;
float4* g_noalloc_ptr[kNoallocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device with that device current.  The host-side name of the array is
// only a stand-in: kernels must get this address, never the symbol itself.
cudaError_t noalloc_scratch(float4** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_grad2d);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = static_cast<float4*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" fgs4d_status fgs4d_render_backward_noalloc(const fgs4d_gaussians* g, const fgs4d_view* views,
                                                      int n_views, const fgs4d_options* opt, void* state,
                                                      size_t state_bytes, const float* final_T,
                                                      const int32_t* n_last, const float* dL_dimage,
                                                      fgs4d_gaussian_grads* grads, fgs4d_stream stream) {
    DevGauss G;
    fgs4d_status s = check_gaussians(g, &G);
    if (s != FGS4D_OK) return s;
    if (!final_T || !n_last || !dL_dimage || !grads) return FGS4D_ERR_INVALID_ARG;
    if (g->n > 0) {
        const void* ptrs[] = {grads->mu, grads->log_scale, grads->q_left, grads->q_right, grads->opacity_logit,
                              grads->shs};
        for (const void* p : ptrs)
            if (!p || !aligned(p, 4)) return FGS4D_ERR_INVALID_ARG;
    }
    if (n_views >= 1 && g->n * (int64_t)n_views > (int64_t)FGS4D_NOALLOC_MAX_SPLATS) return FGS4D_ERR_CAPACITY;
    Prepared prep;
    Prepared* P = &prep;
    s = prepare(g->n, views, n_views, opt, state, state_bytes, P);
    if (s == FGS4D_OK) {
        float4* g2 = nullptr;
        cudaError_t e = noalloc_scratch(&g2);
        char* st = static_cast<char*>(state);
        if (e == cudaSuccess)
            e = launch_render_backward_into(P->VS, P->O, P->L, st, pair_buffer(*P), final_T, n_last, dL_dimage, g2,
                                            (cudaStream_t)stream);
        uint32_t* list = reinterpret_cast<uint32_t*>(g2 + kNoallocGrad);
        uint32_t* misc = reinterpret_cast<uint32_t*>(g2 + kNoallocGrad + kNoallocList);
        if (e == cudaSuccess)
            e = launch_project_backward_from(G, P->VS, P->O, P->L, st, g2, list, misc + kScanBlocksMax + 32, misc,
                                             *grads, (cudaStream_t)stream);
        s = cuda_status(e);
    }
    return s;
}
