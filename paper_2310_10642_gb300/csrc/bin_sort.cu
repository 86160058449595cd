// bin_sort.cu -- tile binning with a depth order, on the device.
//
// "Tile" here is a binning tile (bin_size pixels square).  Each tile's list
// must be ordered by (depth, Gaussian index) (Sec. 3.1: splats are blended in
// depth order; ties broken by index).  Instead of one radix sort of 64-bit
// (tile | depth) keys over all (splat, tile) pairs, the visible splats are
// sorted once by depth and the pairs are then placed by tile keeping that
// order:
//   1. compact the visible (view, Gaussian) splats in index order
//   2. stable LSD radix sort of the compacted splats by depth (32-bit keys)
//   3. counting path (every view has at most kCountTilesMax binning tiles):
//      a stable pass by view, per-chunk tile counts, one scan of them, and
//      an ordered scatter of the splat ids into the tiles' lists (see
//      "Counting-sort binning" below); or
//   3'. radix path (larger views): count the tiles each visible splat's
//      support ellipse reaches, scan the counts in depth order into pair
//      offsets, emit one (global tile id, splat id) pair per reached tile,
//      stable LSD radix sort of the pairs by tile id (only the bits in use)
//   4. per-tile [start, end) ranges
// Stability makes each tile's list come out in (depth, index) order on both
// paths.
//
// All counts that depend on the data (visible splats, pairs) stay on the
// device; grids are sized from capacities and every block derives its share
// from the device count, so the whole pipeline is graph-capturable.
#include "fgs4d_internal.cuh"

namespace fgs4d {

constexpr int kThreads = 256;
constexpr int kItems = 8;
constexpr int kTileItems = kThreads * kItems;  // 2048
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t device_count(const uint32_t* d_n, uint32_t n_max) {
    return d_n ? min(*d_n, n_max) : n_max;
}

// Contiguous chunk [begin, end) of a block, in whole tiles of kTileItems.
__device__ __forceinline__ void block_chunk(uint32_t n, int G, uint32_t& begin, uint32_t& end) {
    uint64_t per = ((uint64_t)n + G - 1) / G;
    per = (per + kTileItems - 1) / kTileItems * kTileItems;
    const uint64_t b = (uint64_t)blockIdx.x * per;
    begin = (uint32_t)(b < (uint64_t)n ? b : (uint64_t)n);
    end = (uint32_t)(b + per < (uint64_t)n ? b + per : (uint64_t)n);
}

// Exclusive scan of one value per thread over the block (blockDim % 32 == 0).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t x, uint32_t* s_warp, uint32_t& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) s_warp[wid] = v;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += y;
        }
        s_warp[lane] = w;
    }
    __syncthreads();
    const uint32_t prefix = (wid > 0 ? s_warp[wid - 1] : 0u) + v - x;
    total = s_warp[nw - 1];
    __syncthreads();
    return prefix;
}

// ---------------------------------------------------------------------------
// Device-wide exclusive scan: reduce -> scan of block sums -> apply.
// ---------------------------------------------------------------------------
struct LoadVisible {  // 1 for a splat that touches a tile
    const uint32_t* tiles;
    __device__ uint32_t operator()(uint32_t i) const { return tiles[i] > 0u ? 1u : 0u; }
};
struct StoreCompact {  // visible splat -> (depth key, splat id) at its rank
    const uint32_t* tiles;
    const uint32_t* depth_key;
    uint32_t* keys;
    uint32_t* vals;
    __device__ void operator()(uint32_t i, uint32_t prefix, uint32_t x) const {
        if (x) {
            keys[prefix] = depth_key[i];
            vals[prefix] = i;
        }
    }
};
struct LoadTilesSorted {  // tile count of the i-th splat in depth order
    const uint32_t* tiles;
    const uint32_t* sorted;
    __device__ uint32_t operator()(uint32_t i) const { return tiles[sorted[i]]; }
};
struct StoreOffset {
    uint32_t* offsets;
    __device__ void operator()(uint32_t i, uint32_t prefix, uint32_t) const { offsets[i] = prefix; }
};

template <class Load>
__global__ void __launch_bounds__(kThreads) scan_reduce_kernel(Load ld, const uint32_t* d_n, uint32_t n_max,
                                                               uint32_t* block_sums) {
    __shared__ uint32_t s_warp[32];
    const uint32_t n = device_count(d_n, n_max);
    uint32_t begin, end;
    block_chunk(n, gridDim.x, begin, end);
    uint32_t sum = 0;
    for (uint32_t i = begin + threadIdx.x; i < end; i += kThreads) sum += ld(i);
    uint32_t total;
    block_exclusive_scan(sum, s_warp, total);
    if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_blocks_kernel(uint32_t* block_sums, int G, uint32_t* total_out) {
    __shared__ uint32_t s_warp[32];
    const uint32_t x = threadIdx.x < G ? block_sums[threadIdx.x] : 0u;
    uint32_t total;
    const uint32_t p = block_exclusive_scan(x, s_warp, total);
    if (threadIdx.x < G) block_sums[threadIdx.x] = p;
    if (threadIdx.x == 0 && total_out) *total_out = total;
}

template <class Load, class Store>
__global__ void __launch_bounds__(kThreads) scan_apply_kernel(Load ld, Store stv, const uint32_t* d_n, uint32_t n_max,
                                                              const uint32_t* block_sums) {
    __shared__ uint32_t s_warp[32];
    const uint32_t n = device_count(d_n, n_max);
    uint32_t begin, end;
    block_chunk(n, gridDim.x, begin, end);
    uint32_t running = block_sums[blockIdx.x];
    for (uint32_t tile = begin; tile < end; tile += kTileItems) {
        const uint32_t my = tile + threadIdx.x * kItems;
        uint32_t x[kItems];
        uint32_t local = 0;
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            x[k] = (my + k < end) ? ld(my + k) : 0u;
            local += x[k];
        }
        uint32_t total;
        uint32_t p = running + block_exclusive_scan(local, s_warp, total);
#pragma unroll
        for (int k = 0; k < kItems; k++) {
            if (my + k < end) stv(my + k, p, x[k]);
            p += x[k];
        }
        running += total;
    }
}

template <class Load, class Store>
static cudaError_t device_scan(Load ld, Store stv, const uint32_t* d_n, uint32_t n_max, uint32_t* block_sums,
                               uint32_t* total_out, int G, cudaStream_t st) {
    scan_reduce_kernel<Load><<<G, kThreads, 0, st>>>(ld, d_n, n_max, block_sums);
    scan_blocks_kernel<<<1, 1024, 0, st>>>(block_sums, G, total_out);
    scan_apply_kernel<Load, Store><<<G, kThreads, 0, st>>>(ld, stv, d_n, n_max, block_sums);
    count_launches(3);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (uint32 key, uint32 value) with RB-bit digits
// (RB = 8 or 9, chosen per sort so that the passes cover the key bits with
// as few passes as possible).  Per pass: upsweep (per-block digit counts),
// scan (one block per digit over the blocks), downsweep (stable rank within
// each block tile by warp match_any, reorder in shared memory, write out).
// ---------------------------------------------------------------------------
template <int RB>
__global__ void __launch_bounds__(kThreads) radix_upsweep_kernel(const uint32_t* __restrict__ keys, const uint32_t* d_n,
                                                                 uint32_t n_max, int shift, uint32_t* hist) {
    constexpr uint32_t D = 1u << RB, DPT = D / kThreads;
    __shared__ uint32_t s_h[kThreads / 32][D];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int w = 0; w < kThreads / 32; w++)
        for (uint32_t k = 0; k < DPT; k++) s_h[w][tid * DPT + k] = 0u;
    __syncthreads();
    const uint32_t n = device_count(d_n, n_max);
    uint32_t begin, end;
    block_chunk(n, gridDim.x, begin, end);
    (void)lane;
    // 16-byte loads (chunks start at multiples of kTileItems of a 256-byte
    // aligned array), one shared atomic per key into the warp's histogram
    const uint32_t n4 = (end - begin) / 4;
    const uint4* k4 = reinterpret_cast<const uint4*>(keys + begin);
    uint32_t* h = s_h[wid];
    for (uint32_t i = tid; i < n4; i += kThreads) {
        const uint4 q = k4[i];
        atomicAdd(&h[(q.x >> shift) & (D - 1)], 1u);
        atomicAdd(&h[(q.y >> shift) & (D - 1)], 1u);
        atomicAdd(&h[(q.z >> shift) & (D - 1)], 1u);
        atomicAdd(&h[(q.w >> shift) & (D - 1)], 1u);
    }
    for (uint32_t i = begin + 4 * n4 + tid; i < end; i += kThreads) atomicAdd(&h[(keys[i] >> shift) & (D - 1)], 1u);
    __syncthreads();
    for (uint32_t k = 0; k < DPT; k++) {
        const uint32_t d = tid * DPT + k;
        uint32_t sum = 0;
        for (int w = 0; w < kThreads / 32; w++) sum += s_h[w][d];
        hist[d * gridDim.x + blockIdx.x] = sum;
    }
}

// One block per digit: exclusive scan over the blocks, digit totals.
__global__ void __launch_bounds__(1024) radix_scan_kernel(uint32_t* hist, int G, uint32_t* digit_total) {
    __shared__ uint32_t s_warp[32];
    const int d = blockIdx.x;
    uint32_t running = 0;
    for (int b0 = 0; b0 < G; b0 += 1024) {
        const int b = b0 + threadIdx.x;
        const uint32_t x = b < G ? hist[d * G + b] : 0u;
        uint32_t total;
        const uint32_t p = block_exclusive_scan(x, s_warp, total);
        if (b < G) hist[d * G + b] = running + p;
        running += total;
    }
    if (threadIdx.x == 0) digit_total[d] = running;
}

template <int RB>
__global__ void __launch_bounds__(kThreads) radix_downsweep_kernel(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, const uint32_t* d_n, uint32_t n_max, int shift, const uint32_t* __restrict__ hist,
    const uint32_t* __restrict__ digit_total) {
    constexpr uint32_t D = 1u << RB, DPT = D / kThreads;
    __shared__ uint32_t s_global[D];
    __shared__ uint32_t s_tile_start[D];
    __shared__ uint32_t s_wcnt[kThreads / 32][D];
    __shared__ uint32_t s_keys[kTileItems];
    __shared__ uint32_t s_vals[kTileItems];
    __shared__ uint32_t s_warp[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t n = device_count(d_n, n_max);
    uint32_t begin, end;
    block_chunk(n, gridDim.x, begin, end);
    if (begin >= end) return;  // uniform across the block
    {
        // this thread owns digits tid*DPT .. tid*DPT + DPT - 1
        uint32_t own[DPT], sum = 0;
        for (uint32_t k = 0; k < DPT; k++) {
            own[k] = digit_total[tid * DPT + k];
            sum += own[k];
        }
        uint32_t tot;
        uint32_t start = block_exclusive_scan(sum, s_warp, tot);
        for (uint32_t k = 0; k < DPT; k++) {
            const uint32_t d = tid * DPT + k;
            s_global[d] = start + hist[d * gridDim.x + blockIdx.x];
            start += own[k];
        }
    }
    const uint32_t lt = lanemask_lt();
    for (uint32_t tile = begin; tile < end; tile += kTileItems) {
        for (int w = 0; w < kThreads / 32; w++)
            for (uint32_t k = 0; k < DPT; k++) s_wcnt[w][tid * DPT + k] = 0u;
        __syncthreads();
        uint32_t k[kItems], val[kItems], dig[kItems], rank[kItems];
#pragma unroll
        for (int i = 0; i < kItems; i++) {
            const uint32_t idx = tile + wid * (32 * kItems) + i * 32 + lane;
            const bool valid = idx < end;
            k[i] = valid ? keys_in[idx] : 0u;
            val[i] = valid ? vals_in[idx] : 0u;
            dig[i] = valid ? (k[i] >> shift) & (D - 1) : D;
        }
#pragma unroll
        for (int i = 0; i < kItems; i++) {
            const uint32_t peers = __match_any_sync(kFull, dig[i]);
            const uint32_t base = dig[i] < D ? s_wcnt[wid][dig[i]] : 0u;
            __syncwarp();
            if (dig[i] < D && lane == __ffs(peers) - 1) s_wcnt[wid][dig[i]] = base + __popc(peers);
            __syncwarp();
            rank[i] = base + __popc(peers & lt);
        }
        __syncthreads();
        uint32_t tile_cnt[DPT], sum = 0;
        for (uint32_t kk = 0; kk < DPT; kk++) {
            const uint32_t d = tid * DPT + kk;
            uint32_t run = 0;
            for (int w = 0; w < kThreads / 32; w++) {
                const uint32_t c = s_wcnt[w][d];
                s_wcnt[w][d] = run;
                run += c;
            }
            tile_cnt[kk] = run;
            sum += run;
        }
        uint32_t tile_total;
        uint32_t ts = block_exclusive_scan(sum, s_warp, tile_total);
        for (uint32_t kk = 0; kk < DPT; kk++) {
            s_tile_start[tid * DPT + kk] = ts;
            ts += tile_cnt[kk];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kItems; i++) {
            if (dig[i] < D) {
                const uint32_t pos = s_tile_start[dig[i]] + s_wcnt[wid][dig[i]] + rank[i];
                s_keys[pos] = k[i];
                s_vals[pos] = val[i];
            }
        }
        __syncthreads();
        const uint32_t tile_n = min((uint32_t)kTileItems, end - tile);
        for (uint32_t j = tid; j < tile_n; j += kThreads) {
            const uint32_t kk = s_keys[j];
            const uint32_t d = (kk >> shift) & (D - 1);
            const uint32_t out = s_global[d] + (j - s_tile_start[d]);
            keys_out[out] = kk;
            vals_out[out] = s_vals[j];
        }
        __syncthreads();
        for (uint32_t kk = 0; kk < DPT; kk++) s_global[tid * DPT + kk] += tile_cnt[kk];
        __syncthreads();
    }
}

// Number of passes and digit width for a sort over `bits` key bits.
static void radix_plan(int bits, int& passes, int& rb) {
    passes = (bits + 8) / 9;  // ceil(bits / 9)
    if (passes < 1) passes = 1;
    rb = ((bits + passes - 1) / passes) > 8 ? 9 : 8;
}

int radix_passes(int bits) {
    int p, rb;
    radix_plan(bits, p, rb);
    return p;
}

// Sorts keys[0]/vals[0] over `bits` low key bits; result in buffer (passes % 2).
static cudaError_t radix_sort(uint32_t* keys[2], uint32_t* vals[2], const uint32_t* d_n, uint32_t n_max, int bits,
                              uint32_t* hist, uint32_t* digit_total, int G, cudaStream_t st, int* out_buf) {
    int passes, rb;
    radix_plan(bits, passes, rb);
    int cur = 0;
    for (int pass = 0; pass < passes; pass++) {
        const int shift = pass * rb;
        if (rb == 9) {
            radix_upsweep_kernel<9><<<G, kThreads, 0, st>>>(keys[cur], d_n, n_max, shift, hist);
            radix_scan_kernel<<<512, 1024, 0, st>>>(hist, G, digit_total);
            radix_downsweep_kernel<9><<<G, kThreads, 0, st>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], d_n,
                                                              n_max, shift, hist, digit_total);
        } else {
            radix_upsweep_kernel<8><<<G, kThreads, 0, st>>>(keys[cur], d_n, n_max, shift, hist);
            radix_scan_kernel<<<256, 1024, 0, st>>>(hist, G, digit_total);
            radix_downsweep_kernel<8><<<G, kThreads, 0, st>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], d_n,
                                                              n_max, shift, hist, digit_total);
        }
        cur ^= 1;
        count_launches(3);
    }
    *out_buf = cur;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pair emission and tile ranges
// ---------------------------------------------------------------------------
// Pair emission, one thread per visible splat in depth order: the thread
// walks its splat's tile rows (the same ellipse_row_tiles calls as the
// count, so exactly tiles[sid] pairs) and writes (tile, splat) pairs from
// the splat's offset on, through its warp's shared buffer.  With 64-pixel binning tiles a splat reaches ~10
// tiles, and a warp-cooperative walk (32 lanes over one splat's box tiles,
// ballot-packed) spent more on broadcasting each splat than on its pairs.
// Should the rows ever disagree with the count, surplus slots get the dump
// tile id VS.total_tiles, which no block renders.
constexpr int kEmitStage = 512;  // pairs a warp gathers in shared memory before writing them out

__global__ void __launch_bounds__(256) emit_pairs_kernel(
    const __grid_constant__ ViewSet VS, uint32_t n_gauss, const uint32_t* __restrict__ sorted_splats,
    const uint32_t* __restrict__ offsets, const uint32_t* __restrict__ tiles, const void* __restrict__ rec,
    int rec_fp16, float ln_alpha_min, uint32_t n_max, uint32_t* counters, uint32_t capacity, int tile,
    uint32_t* __restrict__ pair_keys, uint32_t* __restrict__ pair_vals) {
    constexpr unsigned F = 0xffffffffu;
    // A warp takes 32 consecutive splats, whose pairs fill one contiguous
    // range of the output (their offsets are consecutive in depth order):
    // each thread writes its splat's pairs into the warp's shared buffer, then
    // the warp copies the range out with coalesced stores.  A range larger
    // than the buffer is written directly.
    __shared__ uint32_t s_key[256 / 32][kEmitStage];
    __shared__ uint32_t s_val[256 / 32][kEmitStage];
    const uint32_t n_vis = min(counters[0], n_max);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * blockDim.x) >> 5;
    bool overflow = false;
    for (uint32_t base = warp0 * 32; base < n_vis; base += n_warps * 32) {  // warp-uniform
        const uint32_t p = base + lane;
        uint32_t sid = 0, cnt = 0, o = 0;
        if (p < n_vis) {
            sid = sorted_splats[p];
            cnt = tiles[sid];
            o = offsets[p];
        }
        const uint32_t o_first = __shfl_sync(F, o, 0);
        const uint32_t total = __shfl_sync(F, o + cnt, (int)min(31u, n_vis - 1 - base)) - o_first;
        const bool staged = total <= (uint32_t)kEmitStage;  // warp-uniform
        // pair number `at` of the output: into the warp's buffer (its capacity is checked on the
        // way out), or straight to the pair arrays
        auto put = [&](uint32_t at, uint32_t key, uint32_t val) {
            if (staged) {
                s_key[w][at - o_first] = key;
                s_val[w][at - o_first] = val;
            } else if (at >= capacity) {
                overflow = true;
            } else {
                pair_keys[at] = key;
                pair_vals[at] = val;
            }
        };
        if (cnt > 0) {
            const DevView& V = VS.v[sid / n_gauss];
            const SplatView r = rec_fp16
                                    ? decode_record(reinterpret_cast<const SplatRecordH*>(rec)[sid], ln_alpha_min)
                                    : decode_record(reinterpret_cast<const SplatRecord*>(rec)[sid], ln_alpha_min);
            int rect[4];
            uint32_t written = 0;
            if (box_tiles(r.u, r.v, r.hx, r.hy, V, tile, rect) > 0) {
                const EllipseRows e = ellipse_rows(r, ln_alpha_min);
                for (int ty = rect[1]; ty <= rect[3]; ty++) {
                    int tx0;
                    const int nr = ellipse_row_tiles(e, V, tile, rect, ty, &tx0);
                    const uint32_t row_key = V.tile_base + (uint32_t)ty * (uint32_t)V.tiles_x + (uint32_t)tx0;
                    for (int i = 0; i < nr && written < cnt; i++, written++) put(o + written, row_key + (uint32_t)i, sid);
                }
            }
            // the count came from the same rows, so this never runs; it keeps every slot
            // defined (the dump tile id VS.total_tiles sorts last and no block renders it)
            for (; written < cnt; written++) put(o + written, VS.total_tiles, sid);
        }
        if (staged) {
            __syncwarp();
            for (uint32_t k = (uint32_t)lane; k < total; k += 32) {
                const uint32_t at = o_first + k;
                if (at >= capacity) {
                    overflow = true;
                    break;
                }
                pair_keys[at] = s_key[w][k];
                pair_vals[at] = s_val[w][k];
            }
            __syncwarp();
        }
    }
    if (overflow) atomicOr(&counters[2], FGS4D_STATUS_PAIR_OVERFLOW);
}

// Exact tile count of each visible splat (the support ellipse's rows, as
// emit_pairs_kernel will write them), replacing the box count that
// slice/project left as the visibility flag.  One thread per visible splat.
__global__ void __launch_bounds__(256) ellipse_count_kernel(const __grid_constant__ ViewSet VS, uint32_t n_gauss,
                                                            const uint32_t* __restrict__ sorted_splats,
                                                            const void* __restrict__ rec, int rec_fp16,
                                                            float ln_alpha_min, uint32_t n_max,
                                                            const uint32_t* counters, int tile,
                                                            uint32_t* __restrict__ tiles) {
    const uint32_t n_vis = min(counters[0], n_max);
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n_vis; p += gridDim.x * blockDim.x) {
        const uint32_t sid = sorted_splats[p];
        const DevView& V = VS.v[sid / n_gauss];
        const SplatView r = rec_fp16 ? decode_record(reinterpret_cast<const SplatRecordH*>(rec)[sid], ln_alpha_min)
                                     : decode_record(reinterpret_cast<const SplatRecord*>(rec)[sid], ln_alpha_min);
        int rect[4];
        const int box = box_tiles(r.u, r.v, r.hx, r.hy, V, tile, rect);
        tiles[sid] = box > 0 ? (uint32_t)ellipse_tiles(r, ln_alpha_min, V, tile, rect) : 0u;
    }
}

// Each thread takes four consecutive sorted keys (one 16-byte load; the key
// buffer is 256-byte aligned) and its two neighbours; a tile's range starts
// where its key differs from the previous one and ends where it differs from
// the next.
__global__ void __launch_bounds__(256) tile_ranges_kernel(const uint32_t* __restrict__ keys, const uint32_t* counters,
                                                          uint32_t capacity, uint32_t total_tiles,
                                                          uint2* __restrict__ ranges) {
    const uint32_t n = min(counters[1], capacity);
    const uint32_t n4 = (n + 3) / 4;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n4; q += gridDim.x * blockDim.x) {
        const uint32_t i0 = 4 * q;
        uint32_t k[4];
        if (i0 + 4 <= n) {
            const uint4 v = reinterpret_cast<const uint4*>(keys)[q];
            k[0] = v.x;
            k[1] = v.y;
            k[2] = v.z;
            k[3] = v.w;
        } else {
#pragma unroll
            for (int j = 0; j < 4; j++) k[j] = i0 + j < n ? keys[i0 + j] : 0xffffffffu;
        }
        const uint32_t prev = i0 > 0 ? keys[i0 - 1] : 0xffffffffu;
        const uint32_t next = i0 + 4 < n ? keys[i0 + 4] : 0xffffffffu;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const uint32_t i = i0 + j;
            const uint32_t kj = k[j];
            if (i >= n || kj >= total_tiles) continue;  // past the end, or the dump tile (sorts last)
            const uint32_t left = j == 0 ? prev : k[j - 1];
            const uint32_t right = j == 3 ? next : k[j + 1];
            if (i == 0 || left != kj) ranges[kj].x = i;
            if (i == n - 1 || right != kj) ranges[kj].y = i + 1;
        }
    }
}

// ---------------------------------------------------------------------------
// Counting-sort binning (views of at most kCountTilesMax binning tiles).
// The visible splats are ordered by (view, depth, index); each view's run is
// cut into chunks of `chunk` splats, one warp per chunk.  The histogram
// kernel counts, per chunk, the pairs of each binning tile of its view; an
// exclusive scan of the counts laid out tile-major (per view, (tile, chunk)
// at tile * chunks + chunk after the earlier views' entries) gives every
// (tile, chunk) the first slot of its run in the tile-major pair array.
// The scatter kernel re-walks each chunk in order and writes every splat id
// to its slot.  Chunks of a tile follow each other in depth order and a warp
// keeps its chunk's order, so each tile's list comes out in (depth, index)
// order, as with the radix path.  The scatter's 4-byte stores land all over
// the pair array and their sectors are re-read from DRAM when they leave L2
// incomplete: 256-splat chunks (shorter-lived warps, shorter runs per tile)
// read 559 MB for 132 MB of output at ten views, 1024-splat chunks 835 MB.
// ---------------------------------------------------------------------------

// Splat ids in (depth, index) order -> their view, the key of the stable
// pass that groups the list by view.
__global__ void __launch_bounds__(256) view_keys_kernel(const uint32_t* __restrict__ sorted, const uint32_t* counters,
                                                        uint32_t n_max, uint32_t n_gauss,
                                                        uint32_t* __restrict__ keys) {
    const uint32_t n = min(counters[0], n_max);
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        keys[i] = sorted[i] / n_gauss;
}

// Where chunk c of view v lies.  view_count[] holds the visible splats per
// view, whose runs follow each other in view order in the sorted list; the
// chunk is positions [b, e) of it (empty past the view's end).  The view's
// (tile, chunk) counts take entries [off, off + tiles * chunks) of H, entry
// (t, c) at off + t * chunks + c, with chunks = ceil(visible / chunk): views
// in order, so that H is tile-major over all views.  Called by a whole warp.
struct ChunkPlace {
    uint32_t b, e, off, chunks;
};
__device__ __forceinline__ ChunkPlace chunk_place(const ViewSet& VS, const uint32_t* view_count, uint32_t v,
                                                  uint32_t c, uint32_t chunk) {
    const int lane = threadIdx.x & 31;
    uint32_t before = 0, off = 0;
    for (int i = lane; i < (int)v; i += 32) {
        const uint32_t n = view_count[i];
        before += n;
        off += (uint32_t)(VS.v[i].tiles_x * VS.v[i].tiles_y) * ((n + chunk - 1) / chunk);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        before += __shfl_xor_sync(kFull, before, o);
        off += __shfl_xor_sync(kFull, off, o);
    }
    const uint32_t cnt = view_count[v];
    ChunkPlace P;
    const uint32_t lo = min(c * chunk, cnt), hi = min(lo + chunk, cnt);
    P.b = before + lo;
    P.e = before + hi;
    P.off = off;
    P.chunks = (cnt + chunk - 1) / chunk;
    return P;
}

// Calls f(local tile index ty * tiles_x + tx, k) for the k-th binning tile
// (k = 0, 1, ...) of view V that the splat's support ellipse reaches, in row
// order, at most `limit` times; returns the number of calls.  The same box
// and ellipse rows as the pair count of the radix path.
template <class F>
__device__ __forceinline__ uint32_t for_each_tile(const SplatView& r, const DevView& V, int bin, float ln_alpha_min,
                                                  uint32_t limit, F&& f) {
    int rect[4];
    uint32_t n = 0;
    if (box_tiles(r.u, r.v, r.hx, r.hy, V, bin, rect) > 0) {
        const EllipseRows e = ellipse_rows(r, ln_alpha_min);
        for (int ty = rect[1]; ty <= rect[3] && n < limit; ty++) {
            int tx0;
            const int nr = ellipse_row_tiles(e, V, bin, rect, ty, &tx0);
            const uint32_t row = (uint32_t)ty * (uint32_t)V.tiles_x + (uint32_t)tx0;
            for (int i = 0; i < nr && n < limit; i++, n++) f(row + (uint32_t)i, n);
        }
    }
    return n;
}

__device__ __forceinline__ SplatView load_record(const void* rec, int rec_fp16, uint32_t sid, float ln_alpha_min) {
    return rec_fp16 ? decode_record(reinterpret_cast<const SplatRecordH*>(rec)[sid], ln_alpha_min)
                    : decode_record(reinterpret_cast<const SplatRecord*>(rec)[sid], ln_alpha_min);
}

// Per (view, chunk) warp: pairs per binning tile of the view, into H at
// the chunk's entries (chunk_place); also each visible splat's exact tile
// count, as the radix path's count kernel leaves it.  Warp 0 also stores
// the number of entries of H in use to *n_entries.
__global__ void __launch_bounds__(kCountWarps * 32) count_hist_kernel(
    const __grid_constant__ ViewSet VS, const uint32_t* __restrict__ sorted,
    const uint32_t* __restrict__ view_count, const void* __restrict__ rec, int rec_fp16, float ln_alpha_min, int bin,
    uint32_t chunk, uint32_t chunks_per_view, uint32_t tiles_max, uint32_t* __restrict__ tiles,
    uint32_t* __restrict__ H, uint32_t* __restrict__ n_entries) {
    extern __shared__ uint32_t s_count[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t gw = blockIdx.x * kCountWarps + (uint32_t)w;
    if (gw >= (uint32_t)VS.n * chunks_per_view) return;  // warp-uniform; the kernel has no block barrier
    const uint32_t v = gw / chunks_per_view, c = gw - v * chunks_per_view;
    if (gw == 0) {
        const ChunkPlace L = chunk_place(VS, view_count, (uint32_t)VS.n - 1, 0, chunk);
        if (lane == 0) n_entries[0] = L.off + (uint32_t)(VS.v[VS.n - 1].tiles_x * VS.v[VS.n - 1].tiles_y) * L.chunks;
    }
    const ChunkPlace P = chunk_place(VS, view_count, v, c, chunk);
    if (c >= P.chunks) return;  // warp-uniform: past the view's last chunk
    const DevView& V = VS.v[v];
    const uint32_t nt = (uint32_t)(V.tiles_x * V.tiles_y);
    uint32_t* cnt = s_count + (size_t)w * tiles_max;
    for (uint32_t t = lane; t < nt; t += 32) cnt[t] = 0u;
    __syncwarp();
    for (uint32_t p = P.b + lane; p < P.e; p += 32) {
        const uint32_t sid = sorted[p];
        const SplatView r = load_record(rec, rec_fp16, sid, ln_alpha_min);
        tiles[sid] =
            for_each_tile(r, V, bin, ln_alpha_min, 0xffffffffu, [&](uint32_t t, uint32_t) { atomicAdd(&cnt[t], 1u); });
    }
    __syncwarp();
    for (uint32_t t = lane; t < nt; t += 32) H[P.off + t * P.chunks + c] = cnt[t];
}

// Per (view, chunk) warp, after the exclusive scan of H: writes the chunk's
// splat ids to their slots of the tile-major pair array.  Per round of 32
// splats, each lane walks its splat's tiles into the warp's buffer, as
// (tile << 5 | lane), and sets its bit in each tile's lane mask (shared
// atomic OR); the warp then takes the buffer 32 entries at a time: a
// splat's slot in tile t is the tile's next free slot plus the number of
// lower lanes (earlier splats) in the mask, and the entry of the mask's
// lowest lane advances the tile by the mask's population and clears it.  So
// every tile's slots are taken in list order.  A round with more pairs than
// the buffer holds goes through it in runs of consecutive lanes; a splat
// with more pairs than the buffer holds walks them alone.
__global__ void __launch_bounds__(kCountWarps * 32) count_scatter_kernel(
    const __grid_constant__ ViewSet VS, const uint32_t* __restrict__ sorted,
    const uint32_t* __restrict__ view_count, const void* __restrict__ rec, int rec_fp16, float ln_alpha_min, int bin,
    uint32_t chunk, uint32_t chunks_per_view, uint32_t tiles_max, const uint32_t* __restrict__ tiles,
    const uint32_t* __restrict__ H, uint32_t capacity, uint32_t* counters, uint32_t* __restrict__ pair_vals) {
    extern __shared__ uint32_t s_count[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t gw = blockIdx.x * kCountWarps + (uint32_t)w;
    if (gw >= (uint32_t)VS.n * chunks_per_view) return;  // warp-uniform
    const uint32_t v = gw / chunks_per_view, c = gw - v * chunks_per_view;
    const ChunkPlace P = chunk_place(VS, view_count, v, c, chunk);
    if (c >= P.chunks) return;  // warp-uniform: past the view's last chunk
    const uint32_t b = P.b, e = P.e;
    const DevView& V = VS.v[v];
    const uint32_t nt = (uint32_t)(V.tiles_x * V.tiles_y);
    uint32_t* next = s_count + (size_t)w * (2 * tiles_max + kCountBuf);  // next free slot of each tile
    uint32_t* mask = next + tiles_max;                                   // lanes of the run reaching each tile
    uint32_t* buf = mask + tiles_max;
    for (uint32_t t = lane; t < nt; t += 32) {
        next[t] = H[P.off + t * P.chunks + c];
        mask[t] = 0u;
    }
    __syncwarp();
    const uint32_t lt = lanemask_lt(), bit = 1u << lane;
    for (uint32_t p0 = b; p0 < e; p0 += 32) {  // warp-uniform
        const uint32_t p = p0 + lane;
        uint32_t sid = 0, n_t = 0;
        if (p < e) {
            sid = sorted[p];
            n_t = tiles[sid];
        }
        uint32_t incl = n_t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        for (int l0 = 0; l0 < 32;) {  // warp-uniform
            const uint32_t base = __shfl_sync(kFull, incl - n_t, l0);
            const uint32_t fit = __ballot_sync(kFull, lane >= l0 && incl - base <= kCountBuf);
            if (fit == 0u) {  // lane l0 alone holds more pairs than the buffer: it walks them by itself
                if (lane == l0) {
                    const SplatView r = load_record(rec, rec_fp16, sid, ln_alpha_min);
                    for_each_tile(r, V, bin, ln_alpha_min, n_t, [&](uint32_t t, uint32_t) {
                        const uint32_t at_slot = next[t]++;
                        if (at_slot < capacity) pair_vals[at_slot] = sid;
                        else atomicOr(&counters[2], FGS4D_STATUS_PAIR_OVERFLOW);
                    });
                }
                __syncwarp();
                l0++;
                continue;
            }
            const int l1 = 32 - __clz(fit);  // lanes l0 .. l1 - 1 (fit is contiguous from l0)
            const uint32_t total = __shfl_sync(kFull, incl, l1 - 1) - base;
            if (lane >= l0 && lane < l1 && n_t > 0) {
                const uint32_t at0 = incl - n_t - base;
                const uint32_t tag = (uint32_t)lane;
                const SplatView r = load_record(rec, rec_fp16, sid, ln_alpha_min);
                const uint32_t got = for_each_tile(r, V, bin, ln_alpha_min, n_t, [&](uint32_t t, uint32_t k) {
                    buf[at0 + k] = t << 5 | tag;
                    atomicOr(&mask[t], bit);
                });
                for (uint32_t k = got; k < n_t; k++) buf[at0 + k] = 0xffffffffu;  // never: the walk repeats the count
            }
            __syncwarp();
            // the run's entries 32 at a time: slot of (tile t, owner lane o) = next[t] + lanes below o in the mask
            for (uint32_t q0 = 0; q0 < total; q0 += 32) {  // warp-uniform
                const uint32_t q = q0 + (uint32_t)lane;
                const uint32_t ent = q < total ? buf[q] : 0xffffffffu;
                const uint32_t t = ent >> 5, o = ent & 31u;
                const uint32_t src = __shfl_sync(kFull, sid, (int)o);
                if (t < nt) {
                    const uint32_t at_slot = next[t] + __popc(mask[t] & ((1u << o) - 1u));
                    if (at_slot < capacity) pair_vals[at_slot] = src;
                    else atomicOr(&counters[2], FGS4D_STATUS_PAIR_OVERFLOW);
                }
            }
            __syncwarp();
            // the entry of each mask's lowest lane advances its tile and clears the mask (another
            // entry of the tile reads either the mask, whose lowest lane it is not, or zero)
            for (uint32_t q0 = 0; q0 < total; q0 += 32) {  // warp-uniform
                const uint32_t q = q0 + (uint32_t)lane;
                const uint32_t ent = q < total ? buf[q] : 0xffffffffu;
                const uint32_t t = ent >> 5, o = ent & 31u;
                if (t < nt) {
                    const uint32_t m = mask[t];
                    if (m != 0u && (uint32_t)(__ffs(m) - 1) == o) {
                        next[t] += __popc(m);
                        mask[t] = 0u;
                    }
                }
            }
            __syncwarp();
            l0 = l1;
        }
    }
}

__device__ __forceinline__ int find_view_of_tile(const ViewSet& VS, uint32_t tile) {
    int lo = 0, hi = VS.n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (VS.v[mid].tile_base <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Tile t's list: from its first entry of the scanned counts to the next
// tile's first entry (the pair total after the last tile), clamped to the
// capacity; flags a pair total beyond it.
__global__ void __launch_bounds__(256) count_ranges_kernel(const __grid_constant__ ViewSet VS,
                                                           const uint32_t* __restrict__ H,
                                                           const uint32_t* __restrict__ view_count, uint32_t chunk,
                                                           uint32_t* counters, uint32_t capacity,
                                                           uint2* __restrict__ ranges) {
    __shared__ uint32_t s_off[FGS4D_MAX_VIEWS], s_ch[FGS4D_MAX_VIEWS];
    if (threadIdx.x == 0) {
        uint32_t off = 0;
        for (int i = 0; i < VS.n; i++) {
            const uint32_t ch = (view_count[i] + chunk - 1) / chunk;
            s_off[i] = off;
            s_ch[i] = ch;
            off += (uint32_t)(VS.v[i].tiles_x * VS.v[i].tiles_y) * ch;
        }
    }
    __syncthreads();
    const uint32_t n_pairs = counters[1], n_entries = counters[8];
    const uint32_t i0 = blockIdx.x * blockDim.x + threadIdx.x;
    if (i0 == 0 && n_pairs > capacity) atomicOr(&counters[2], FGS4D_STATUS_PAIR_OVERFLOW);
    for (uint32_t t = i0; t < VS.total_tiles; t += gridDim.x * blockDim.x) {
        const int v = find_view_of_tile(VS, t);
        const uint32_t tl = t - VS.v[v].tile_base;
        const uint32_t i_s = s_off[v] + tl * s_ch[v], i_e = i_s + s_ch[v];
        const uint32_t s = i_s < n_entries ? H[i_s] : n_pairs;
        const uint32_t e = i_e < n_entries ? H[i_e] : n_pairs;
        ranges[t] = make_uint2(min(s, capacity), min(e, capacity));
    }
}

struct LoadPlain {
    const uint32_t* a;
    __device__ uint32_t operator()(uint32_t i) const { return a[i]; }
};
struct StorePrefix {
    uint32_t* a;
    __device__ void operator()(uint32_t i, uint32_t prefix, uint32_t) const { a[i] = prefix; }
};

static int grid_cap(uint32_t want, int cap) { return (int)(want < (uint32_t)cap ? (want > 0 ? want : 1) : (uint32_t)cap); }

// Visible splats in Gaussian-major order (g, then view): i' = g V + v.
struct LoadVisibleGV {
    const uint32_t* tiles;
    uint32_t n, V;
    __device__ uint32_t operator()(uint32_t i) const { return tiles[(i % V) * n + i / V] > 0u ? 1u : 0u; }
};
struct StoreListGV {
    uint32_t* list;
    uint32_t n, V;
    __device__ void operator()(uint32_t i, uint32_t prefix, uint32_t x) const {
        if (x) list[prefix] = (i % V) * n + i / V;  // splat id v n + g
    }
};

cudaError_t compact_visible_gaussian_major(const uint32_t* tiles, uint32_t n, uint32_t V, uint32_t* list,
                                           uint32_t* count, uint32_t* scan_tmp, int sm_count, cudaStream_t st) {
    const uint32_t S = n * V;
    if (S == 0) return cudaMemsetAsync(count, 0, sizeof(uint32_t), st);
    const uint32_t want = (S + kTileItems - 1) / kTileItems;
    const int G = (int)max(1u, min(want, (uint32_t)min(kScanBlocksMax, 4 * sm_count)));
    return device_scan(LoadVisibleGV{tiles, n, V}, StoreListGV{list, n, V}, nullptr, S, scan_tmp, count, G, st);
}

int pair_sort_bits(uint32_t total_tiles) {
    int bits = 1;
    while (bits < 32 && (1ull << bits) < (unsigned long long)total_tiles) bits++;
    return bits;
}

// Steps 3-6 of the counting path, after the depth sort left the visible
// splat ids in (depth, index) order in sv[buf]: a stable pass by view, the
// (tile, chunk) counts, their scan (-> counters[1]), the scatter and the
// ranges.
static cudaError_t count_bin(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state, int sm_count,
                             cudaStream_t st, uint32_t* sk[2], uint32_t* sv[2], int buf, int Gs, int* out_buf) {
    const uint32_t S = (uint32_t)lay.n_splats;
    const uint32_t n_gauss = S / (uint32_t)VS.n;
    uint32_t* counters = reinterpret_cast<uint32_t*>(state + lay.counters);
    uint32_t* tiles = reinterpret_cast<uint32_t*>(state + lay.tiles_touched);
    uint32_t* hist = reinterpret_cast<uint32_t*>(state + lay.hist);
    uint32_t* digit_total = hist + kMaxDigits * kSortBlocksMax;
    uint32_t* scan_tmp = reinterpret_cast<uint32_t*>(state + lay.scan_tmp);
    uint32_t* H = reinterpret_cast<uint32_t*>(state + lay.chunk_hist);
    uint32_t* pv = reinterpret_cast<uint32_t*>(state + lay.pair_vals[0]);
    uint2* ranges = reinterpret_cast<uint2*>(state + lay.ranges);
    const void* rec = state + lay.records;
    const int stride_grid = 16 * sm_count;
    cudaError_t e;
    *out_buf = 0;
    // stable pass by view: the list becomes (view, depth, index) ordered and
    // the pass's digit totals are the visible splats per view
    const uint32_t* sorted = sv[buf];
    const uint32_t* view_count = &counters[0];  // one view: all visible splats
    if (VS.n > 1) {
        view_keys_kernel<<<grid_cap((S + 255) / 256, stride_grid), 256, 0, st>>>(sv[buf], counters, S, n_gauss,
                                                                                  sk[buf]);
        count_launches(1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        uint32_t* k2[2] = {sk[buf], sk[buf ^ 1]};
        uint32_t* v2[2] = {sv[buf], sv[buf ^ 1]};
        int vb = 0;
        e = radix_sort(k2, v2, &counters[0], S, pair_sort_bits((uint32_t)VS.n), hist, digit_total, Gs, st, &vb);
        if (e != cudaSuccess) return e;
        sorted = v2[vb];
        view_count = digit_total;
    }
    const uint32_t CH = lay.chunks_per_view, tmax = lay.view_tiles_max;
    const uint32_t warps = (uint32_t)VS.n * CH;
    const int blocks = (int)((warps + kCountWarps - 1) / kCountWarps);
    const size_t smem_hist = (size_t)kCountWarps * tmax * 4;
    const size_t smem_scatter = (size_t)kCountWarps * (2 * tmax + kCountBuf) * 4;
    if ((e = cudaFuncSetAttribute((const void*)count_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_hist)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute((const void*)count_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_scatter)) != cudaSuccess)
        return e;
    count_hist_kernel<<<blocks, kCountWarps * 32, smem_hist, st>>>(VS, sorted, view_count, rec,
                                                                   O.record_fp16, O.ln_alpha_min, O.bin, lay.chunk,
                                                                   CH, tmax, tiles, H, &counters[8]);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the entries in use (counters[8]) are at most total_tiles * chunks_per_view
    const uint32_t nH = VS.total_tiles * CH;
    const uint32_t want = (nH + kTileItems - 1) / kTileItems;
    const int Gh = (int)max(1u, min(want, (uint32_t)min(kScanBlocksMax, 4 * sm_count)));
    e = device_scan(LoadPlain{H}, StorePrefix{H}, &counters[8], nH, scan_tmp, &counters[1], Gh, st);
    if (e != cudaSuccess) return e;
    const uint32_t cap = (uint32_t)lay.capacity;
    count_scatter_kernel<<<blocks, kCountWarps * 32, smem_scatter, st>>>(
        VS, sorted, view_count, rec, O.record_fp16, O.ln_alpha_min, O.bin, lay.chunk, CH, tmax, tiles, H,
        cap, counters, pv);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    count_ranges_kernel<<<grid_cap((VS.total_tiles + 255) / 256, stride_grid), 256, 0, st>>>(
        VS, H, view_count, lay.chunk, counters, cap, ranges);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_bin_sort(const ViewSet& VS, const DevOpts& O, const StateLayout& lay, char* state, int sm_count,
                            cudaStream_t st, int* out_buf) {
    const uint32_t S = (uint32_t)lay.n_splats;
    uint32_t* counters = reinterpret_cast<uint32_t*>(state + lay.counters);
    uint32_t* tiles = reinterpret_cast<uint32_t*>(state + lay.tiles_touched);
    uint32_t* dkey = reinterpret_cast<uint32_t*>(state + lay.depth_key);
    uint32_t* sk[2] = {reinterpret_cast<uint32_t*>(state + lay.sort_keys[0]),
                       reinterpret_cast<uint32_t*>(state + lay.sort_keys[1])};
    uint32_t* sv[2] = {reinterpret_cast<uint32_t*>(state + lay.sort_vals[0]),
                       reinterpret_cast<uint32_t*>(state + lay.sort_vals[1])};
    uint32_t* offsets = reinterpret_cast<uint32_t*>(state + lay.offsets);
    uint32_t* scan_tmp = reinterpret_cast<uint32_t*>(state + lay.scan_tmp);
    uint32_t* hist = reinterpret_cast<uint32_t*>(state + lay.hist);
    uint32_t* digit_total = hist + kMaxDigits * kSortBlocksMax;
    uint2* ranges = reinterpret_cast<uint2*>(state + lay.ranges);
    uint32_t* pk[2] = {reinterpret_cast<uint32_t*>(state + lay.pair_keys[0]),
                       reinterpret_cast<uint32_t*>(state + lay.pair_keys[1])};
    uint32_t* pv[2] = {reinterpret_cast<uint32_t*>(state + lay.pair_vals[0]),
                       reinterpret_cast<uint32_t*>(state + lay.pair_vals[1])};
    const void* rec = state + lay.records;
    const uint32_t cap = (uint32_t)lay.capacity;
    cudaError_t e = cudaMemsetAsync(ranges, 0, sizeof(uint2) * (size_t)VS.total_tiles, st);
    if (e != cudaSuccess) return e;
    *out_buf = 0;
    if (S == 0) return cudaSuccess;
    auto grid_for = [&](uint32_t n) {
        const uint32_t want = (n + kTileItems - 1) / kTileItems;
        return (int)max(1u, min(want, (uint32_t)min(kSortBlocksMax, 4 * sm_count)));
    };
    // 1. compaction of visible splats -> counters[0]
    const int Gs = grid_for(S);
    e = device_scan(LoadVisible{tiles}, StoreCompact{tiles, dkey, sk[0], sv[0]}, nullptr, S, scan_tmp, &counters[0],
                    Gs, st);
    if (e != cudaSuccess) return e;
    // 2. depth sort (positive float bits sort as unsigned integers)
    int buf = 0;
    e = radix_sort(sk, sv, &counters[0], S, 32, hist, digit_total, Gs, st, &buf);
    if (e != cudaSuccess) return e;
    const uint32_t* sorted = sv[buf];
    const int stride_grid = 16 * sm_count;
    if (lay.count_sort) return count_bin(VS, O, lay, state, sm_count, st, sk, sv, buf, Gs, out_buf);
    // 3. exact tile counts (support ellipse), then pair offsets in depth order -> counters[1]
    ellipse_count_kernel<<<grid_cap((S + 255) / 256, stride_grid), 256, 0, st>>>(
        VS, (uint32_t)(S / (uint32_t)VS.n), sorted, rec, O.record_fp16, O.ln_alpha_min, S, counters, O.bin, tiles);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = device_scan(LoadTilesSorted{tiles, sorted}, StoreOffset{offsets}, &counters[0], S, scan_tmp, &counters[1], Gs,
                    st);
    if (e != cudaSuccess) return e;
    // 4. emission
    emit_pairs_kernel<<<grid_cap((S + 255) / 256, stride_grid), 256, 0, st>>>(
        VS, (uint32_t)(S / (uint32_t)VS.n), sorted, offsets, tiles, rec, O.record_fp16, O.ln_alpha_min, S, counters,
        cap, O.bin, pk[0], pv[0]);
    count_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (cap == 0) return cudaSuccess;
    // 5. stable sort of pairs by tile id
    const int bits = pair_sort_bits(VS.total_tiles + 1);  // + the dump tile id
    const int Gp = grid_for(cap);
    e = radix_sort(pk, pv, &counters[1], cap, bits, hist, digit_total, Gp, st, out_buf);
    if (e != cudaSuccess) return e;
    // 6. ranges
    tile_ranges_kernel<<<grid_cap((cap / 4 + 255) / 256, stride_grid), 256, 0, st>>>(pk[*out_buf], counters, cap,
                                                                                         VS.total_tiles,
                                                                                         ranges);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace fgs4d
