// Fused AdamW-GS step: visibility decision, shared-memory compaction of the
// visible rows of a tile, Sparse Adam + DAR on the visible rows, RSR on the
// StSS-sampled rows — one pass over HBM per step.
//
// One CTA handles one tile of kTile consecutive rows with 256 threads:
//   A. each thread decides visibility (camera frustum test of the mean,
//      caller mask, or all-visible) and StSS membership for kTile/256 rows,
//      issuing the load of a visible row's step counter right away; warp
//      ballots + a per-(chunk, warp) count table place every visible row in a
//      shared-memory list (ascending by row) next to the two bias-correction
//      factors of its new step count.
//   B. a flat loop over work items of each visible row:
//        48/kW SH items, kW SH columns each (their attributes, gradients and
//           moments are contiguous, so a warp reads whole rows),
//        3 small items: rotation; xyz + scale0; scale1 + scale2 + opacity,
//      and the same items, state only, for the RSR of invisible
//      StSS-sampled rows.  Items are grouped by kind so warps stay convergent.
// Every row's attributes, moments and counter are read and written by exactly
// one item, once.  The storage format of the moments is a template parameter
// (State<kPrec>): all arithmetic is FP32.


#include "step_common.cuh"

namespace gs {
namespace {

// ---------------------------------------------------------------- phase A

// Shared-memory lists of one tile.
template <int kTile>
struct TileLists {
    int32_t list[kTile];      // visible rows, bit 31 = StSS-sampled
    int32_t rlist[kTile];     // invisible StSS-sampled rows
    float2 fac[kTile];        // bias factors of each visible row
    int32_t cnt[2][kTile / 32];
};

// What the step with the active count and/or position noise on its visible
// rows (the terms form, kX) keeps beside the lists: for each listed visible
// row, the values its noise is drawn from as they were before the step
// (quaternion; log-scales and opacity logit), read in phase A, and the
// tile's count of rows active after the step.  The xyz item draws the noise
// from the kept values, so the items that update the rotation, scale and
// opacity cannot change its inputs, and the draw runs on converged warps.
template <int kTile>
struct TileTerms {
    float4 q[kTile];
    float4 sko[kTile];        // kappa 0-2, tau
    unsigned active;
};

// Decide visibility and StSS membership for the tile's rows, prefetch the
// step counters of visible rows (at byte kTByte of their m row), and compact
// both row sets into `L`; in a sparse tile, ask L2 for each visible row's
// data.  Returns the visible count in nv and the invisible-sampled count in
// nr.  kX: the inputs of a visible row's noise (App. Eq. disentangled_mu)
// go to X beside its list entry, and invisible rows, whose opacity this step
// leaves unchanged, are counted into X->active when the step counts N_a.
template <int kTile, int kRowBytes, int kTByte, bool kX>
__device__ __forceinline__ void tile_decide(const StepArgs &a, const int vis_src, const int64_t r0, TileLists<kTile> &L,
                                            TileTerms<kTile> *X, int &nv, int &nr)
{
    constexpr int kRpt = kTile / kThreads;
    constexpr int kWarps = kThreads / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nrow = (int)min((int64_t)kTile, (int64_t)a.n_rows - r0);
    unsigned bal_v[kRpt], bal_r[kRpt], bal_s[kRpt];
    uint32_t t_old[kRpt];
    float4 xq[kX ? kRpt : 1], xs[kX ? kRpt : 1];
    unsigned my_active = 0;
    if constexpr (kX) {
        if (tid == 0) X->active = 0u;
    }
#pragma unroll
    for (int j = 0; j < kRpt; ++j) {
        const int lr = j * kThreads + tid;
        const int64_t row = r0 + lr;
        const bool in = lr < nrow;
        bool vis = false, smp = false;
        t_old[j] = 0;
        if (in) {
            if (vis_src == kVisCamera) {
                const float *p = a.a_xyz + row * 3;
                vis = frustum_visible(p[0], p[1], p[2], a.cam);
            } else if (vis_src == kVisMask) {
                vis = a.mask_in[row] != 0;
            } else {
                vis = true;
            }
            if (vis && !a.bias_mode) {
                const char *tp = static_cast<const char *>(a.m) + (size_t)row * kRowBytes + kTByte;
                if constexpr (kTByte % 4 == 0) t_old[j] = *reinterpret_cast<const uint32_t *>(tp);
                else t_old[j] = *reinterpret_cast<const uint16_t *>(tp);      // FP16-block rows: uint16 t
            }
            if (a.mask_out) a.mask_out[row] = vis ? 1 : 0;
            if (a.restate) smp = stss_sampled(a, (int32_t)row);
        }
        if constexpr (kX) {
            if (in && vis && a.noise) {
                xq[j] = ld4(a.a_rot + row * 4);
                const float *ps = a.a_scale + row * 3;
                xs[j] = make_float4(ps[0], ps[1], ps[2], a.a_op[row]);
            }
            if (in && !vis && a.n_active) my_active += a.a_op[row] > a.tau_act ? 1u : 0u;
        }
        bal_v[j] = __ballot_sync(0xffffffffu, vis);
        bal_s[j] = __ballot_sync(0xffffffffu, smp);
        bal_r[j] = bal_s[j] & ~bal_v[j];
        if (lane == 0) {
            L.cnt[0][j * kWarps + warp] = __popc(bal_v[j]);
            L.cnt[1][j * kWarps + warp] = __popc(bal_r[j]);
        }
    }
    __syncthreads();
    if constexpr (kX) {
        if (a.n_active) {
            my_active = __reduce_add_sync(0xffffffffu, my_active);
            if (lane == 0 && my_active) atomicAdd(&X->active, my_active);
        }
    }
    nv = 0;
    nr = 0;
#pragma unroll 4
    for (int q = 0; q < kRpt * kWarps; ++q) {
        nv += L.cnt[0][q];
        nr += L.cnt[1][q];
    }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kRpt; ++j) {
        const int me = j * kWarps + warp;
        int bv = 0, br = 0;
        for (int q = 0; q < me; ++q) {
            bv += L.cnt[0][q];
            br += L.cnt[1][q];
        }
        const int32_t row = (int32_t)(r0 + j * kThreads + tid);
        if (bal_v[j] & (1u << lane)) {
            const bool smp = (bal_s[j] >> lane) & 1u;
            const int pos = bv + __popc(bal_v[j] & lt);
            L.list[pos] = row | (smp ? (int32_t)0x80000000 : 0);
            if (sparse_tile<kTile>(nv)) prefetch_row_l2<kRowBytes>(a, row);
            const uint32_t tb = a.bias_mode ? a.k_bias : t_old[j] + 1u;
            L.fac[pos] = (tb < (uint32_t)a.fac_len) ? a.fac[tb] : make_float2(1.0f, 1.0f);
            if constexpr (kX) { if (a.noise) { X->q[pos] = xq[j]; X->sko[pos] = xs[j]; } }
        }
        if (bal_r[j] & (1u << lane)) L.rlist[br + __popc(bal_r[j] & lt)] = row;
    }
    if (tid == 0 && a.n_visible && nv) atomicAdd(a.n_visible, (unsigned long long)nv);
    __syncthreads();
}

// ---------------------------------------------------------------- the kernel

// Phase B of one tile: the items of its visible and invisible-sampled rows
// (nv, nr of them in L), grouped by kind: all SH items, then the small
// items, then RSR.  kX: the xyz items draw the rows' noise from the values
// kept in X and subtract it, the opacity items count the rows active after
// the step, and the tile's count is added to a.n_active.
template <int kTile, int kPrec, int kW, bool kX>
__device__ __forceinline__ void tile_items(const StepArgs &a, const TileLists<kTile> &L, TileTerms<kTile> *X,
                                           const int nv, const int nr)
{
    constexpr int kNsh = 48 / kW, kItems = kNsh + kSmallItems<kPrec>;
    const int e_sh = kNsh * nv, e_vis = kItems * nv, e_all = e_vis + kItems * nr;
    // One flat item space, walked as three loops (SH items, small items, RSR
    // items) with the same item-to-thread assignment as a single loop: the
    // kinds no longer share a loop body, so their register demands do not
    // add up (FP16 block then fits 5 CTAs per SM).
    unsigned my_active = 0;
    int w = threadIdx.x;
    for (; w < e_sh; w += kThreads) {
        const int j = w / kNsh, i = w - j * kNsh;
        const int32_t e = L.list[j];
        sh_item<kPrec, kW>(a, e & 0x7fffffff, i, e < 0, L.fac[j]);
    }
    for (; w < e_vis; w += kThreads) {
        const int q = w - e_sh;
        const int j = q % nv, c = 12 + q / nv;
        const int32_t e = L.list[j];
        if constexpr (kX) {
            float3 nz = make_float3(0.f, 0.f, 0.f);
            if (c == 13 && a.noise) {
                const float4 q = X->q[j], s4 = X->sko[j];
                nz = noise_term(a, e & 0x7fffffff, q, s4.x, s4.y, s4.z, s4.w);
            }
            my_active += small_item<kPrec, true>(a, e & 0x7fffffff, c, e < 0, L.fac[j], nz) ? 1u : 0u;
        } else {
            small_item<kPrec>(a, e & 0x7fffffff, c, e < 0, L.fac[j]);
        }
    }
    for (; w < e_all; w += kThreads) {
        const int q = w - e_vis;
        const int j = q / kItems, i = q - j * kItems;
        rsr_item<kPrec, kW>(a, L.rlist[j], i);
    }
    if constexpr (kX) {
        if (a.n_active) {
            my_active = __reduce_add_sync(0xffffffffu, my_active);
            if ((threadIdx.x & 31) == 0 && my_active) atomicAdd(&X->active, my_active);
            __syncthreads();
            if (threadIdx.x == 0 && X->active) atomicAdd(a.n_active, (unsigned long long)X->active);
        }
    }
}

// One tile: phase A, then its items.
template <int kTile, int kPrec, int kW, bool kX = false>
__device__ __forceinline__ void process_tile(const StepArgs &a, const int vis_src, const int64_t r0,
                                             TileLists<kTile> &L, TileTerms<kTile> *X = nullptr)
{
    static_assert(kTile % kThreads == 0, "tile must be a multiple of the block");
    static_assert(kW == 4 || kW == 8, "SH items cover 4 or 8 columns");
    using S = State<kPrec>;
    int nv, nr;
    tile_decide<kTile, S::kRowBytes, S::kTByte, kX>(a, vis_src, r0, L, X, nv, nr);
    tile_items<kTile, kPrec, kW, kX>(a, L, X, nv, nr);
}

template <int kTile, int kMinBlocks, int kPrec, int kW>
__global__ void __launch_bounds__(kThreads, kMinBlocks) step_tile(const StepArgs a, const int vis_src)
{
    __shared__ TileLists<kTile> L;
    pdl_enter();
    prefetch_tile_ahead<kTile>(a, vis_src);
    process_tile<kTile, kPrec, kW>(a, vis_src, (int64_t)blockIdx.x * kTile, L);
}

// The terms form: the same step with the active count N_a (Sec. 4) and/or
// position noise on the visible rows (App. Eq. disentangled_mu).  AIU and
// noise on every row take the extended kernel instead.
template <int kTile, int kMinBlocks, int kPrec, int kW>
__global__ void __launch_bounds__(kThreads, kMinBlocks) step_tile_terms(const StepArgs a, const int vis_src)
{
    __shared__ TileLists<kTile> L;
    __shared__ TileTerms<kTile> X;
    pdl_enter();
    prefetch_tile_ahead<kTile>(a, vis_src);
    prefetch_tile_ahead_x<kTile>(a);
    process_tile<kTile, kPrec, kW, true>(a, vis_src, (int64_t)blockIdx.x * kTile, L, &X);
}

// Many scenes in one persistent launch.  The scene table lives in device
// memory (p); CTAs take the next tile of the whole batch from the work
// counter (tile t belongs to the scene s with tile_start[s] <= t <
// tile_start[s+1]) until all tiles are done, keeping the current scene's
// arguments in shared memory.  The last CTA to finish returns both counters
// to zero, so every launch (and every replay of a captured graph) starts
// from a clean counter.
template <int kTile, int kMinBlocks, int kPrec, int kW>
__global__ void __launch_bounds__(kThreads, kMinBlocks) step_batch(const BatchParams *__restrict__ p,
                                                                    unsigned *__restrict__ work,
                                                                    unsigned *__restrict__ done)
{
    __shared__ TileLists<kTile> L;
    __shared__ StepArgs sa;
    __shared__ int s_tile;
    const int tid = threadIdx.x;
    const int total = p->total_tiles, n_scenes = p->n_scenes;
    int cur = -1;
    for (;;) {
        if (tid == 0) s_tile = (int)atomicAdd(work, 1u);
        __syncthreads();
        const int t = s_tile;
        if (t >= total) break;
        int lo = 0, hi = n_scenes - 1;         // last scene whose first tile is <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p->tile_start[mid] <= t) lo = mid; else hi = mid - 1;
        }
        if (lo != cur) {
            const uint32_t *src = reinterpret_cast<const uint32_t *>(&p->args[lo]);
            uint32_t *dst = reinterpret_cast<uint32_t *>(&sa);
            for (int q = tid; q < (int)(sizeof(StepArgs) / 4); q += kThreads) dst[q] = src[q];
            cur = lo;
            __syncthreads();
        }
        process_tile<kTile, kPrec, kW>(sa, kVisCamera, (int64_t)(t - p->tile_start[lo]) * kTile, L);
        __syncthreads();                       // the lists are reused by the next tile
    }
    if (tid == 0 && atomicAdd(done, 1u) == gridDim.x - 1) {
        *work = 0u;
        *done = 0u;
    }
}

// Many scenes in one launch with one CTA per tile of the whole batch: CTA t
// finds its scene (the last whose first tile is <= t), copies that scene's
// arguments into shared memory and runs the tile.  The hardware schedules
// the CTAs as it does a single scene's; the tuner weighs this against the
// persistent form.  work and done are unused (same signature).
template <int kTile, int kMinBlocks, int kPrec, int kW>
__global__ void __launch_bounds__(kThreads, kMinBlocks) step_batch_grid(const BatchParams *__restrict__ p,
                                                                         unsigned *, unsigned *)
{
    __shared__ TileLists<kTile> L;
    __shared__ StepArgs sa;
    const int t = (int)blockIdx.x;
    if (t >= p->total_tiles) return;
    int lo = 0, hi = p->n_scenes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p->tile_start[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&p->args[lo]);
    uint32_t *dst = reinterpret_cast<uint32_t *>(&sa);
    for (int q = threadIdx.x; q < (int)(sizeof(StepArgs) / 4); q += kThreads) dst[q] = src[q];
    __syncthreads();
    process_tile<kTile, kPrec, kW>(sa, kVisCamera, (int64_t)(t - p->tile_start[lo]) * kTile, L);
}

}  // namespace

constexpr int kStepTile = 256;
// CTAs of 256 threads resident per SM: 5 (51 registers; no spills except a
// few words for FP16 block), where the extra warps hide more DRAM latency
// than 4 CTAs of 64 registers do (measured: FP32 1-5 %, FP16 block up to
// 7.5 %, BF16 4.6 %, hybrid 2 % faster on the 3 M workload).
template <int kPrec>
constexpr int kStepMinBlocks = 5;
constexpr int kShWF32 = 4, kShWBf16 = 8;   // SH columns per item

namespace {

// Resident CTAs per SM of the terms form: 5 where it fits 48 registers
// without spills (FP32, BF16), 4 for the hybrid and FP16-block formats.
template <int kPrec>
constexpr int kTermsMinBlocks = (kPrec == GS_MOM_FP32 || kPrec == GS_MOM_BF16) ? 5 : 4;

template <int kPrec, int kW, bool kX>
cudaError_t launch_tiles(const StepArgs &a, int vis_src, cudaStream_t s)
{
    auto k = kX ? step_tile_terms<kStepTile, kTermsMinBlocks<kPrec>, kPrec, kW>
                : step_tile<kStepTile, kStepMinBlocks<kPrec>, kPrec, kW>;
    static int s_res[64] = {};
    StepArgs b = a;
    b.tile_ahead = resident_ctas(reinterpret_cast<const void *>(k), s_res);
    const unsigned n_tiles = (unsigned)((a.n_rows + kStepTile - 1) / kStepTile);
    return launch_pdl(k, n_tiles, kThreads, s, b, vis_src);
}

}  // namespace

cudaError_t launch_step(const StepArgs &a, int prec, int vis_src, cudaStream_t s)
{
    if (a.n_rows <= 0) return cudaSuccess;
    if (prec == GS_MOM_FP8E4M3)
        return (a.noise || a.aiu || a.n_active) ? cudaErrorNotSupported : launch_step_fp8(a, vis_src, s);
    if (a.aiu || a.noise == GS_NOISE_ALL) return launch_step_ext(a, prec, vis_src, s);
    const bool x = a.n_active || a.noise;      // the count and/or noise on visible rows: the terms form
    switch (prec) {
    case GS_MOM_FP32:
        return x ? launch_tiles<GS_MOM_FP32, kShWF32, true>(a, vis_src, s)
                 : launch_tiles<GS_MOM_FP32, kShWF32, false>(a, vis_src, s);
    case GS_MOM_BF16:
        return x ? launch_tiles<GS_MOM_BF16, kShWBf16, true>(a, vis_src, s)
                 : launch_tiles<GS_MOM_BF16, kShWBf16, false>(a, vis_src, s);
    case GS_MOM_BF16_HYBRID:
        return x ? launch_tiles<GS_MOM_BF16_HYBRID, kShWBf16, true>(a, vis_src, s)
                 : launch_tiles<GS_MOM_BF16_HYBRID, kShWBf16, false>(a, vis_src, s);
    case GS_MOM_FP16_BLOCK:
        return x ? launch_tiles<GS_MOM_FP16_BLOCK, 8, true>(a, vis_src, s)
                 : launch_tiles<GS_MOM_FP16_BLOCK, 8, false>(a, vis_src, s);
    default: return cudaErrorNotSupported;
    }
}

// ------------------------------------------------------------ batched launch
namespace {

template <int kTile, int kMinBlocks, int kPrec, int kW>
cudaError_t launch_batch_grid_t(const BatchParams *p, unsigned *work, unsigned *done, int total_tiles, cudaStream_t s,
                                int *grid_out, void **fn_out)
{
    auto k = step_batch_grid<kTile, kMinBlocks, kPrec, kW>;
    const int grid = std::max(1, total_tiles);
    if (grid_out) *grid_out = grid;
    if (fn_out) {                              // only report the kernel and its grid
        *fn_out = reinterpret_cast<void *>(k);
        return cudaSuccess;
    }
    k<<<grid, kThreads, 0, s>>>(p, work, done);
    return cudaGetLastError();
}

template <int kTile, int kMinBlocks, int kPrec, int kW>
cudaError_t launch_batch_t(const BatchParams *p, unsigned *work, unsigned *done, int, cudaStream_t s, int *grid_out,
                           void **fn_out)
{
    auto k = step_batch<kTile, kMinBlocks, kPrec, kW>;
    static int s_grid[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int &grid = s_grid[dev & 63];
    if (!grid) {
        int per_sm = 0, sms = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kThreads, 0)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        grid = std::max(1, per_sm) * sms;      // persistent: every CTA resident
    }
    if (grid_out) *grid_out = grid;
    if (fn_out) {                              // only report the kernel and its grid
        *fn_out = reinterpret_cast<void *>(k);
        return cudaSuccess;
    }
    k<<<grid, kThreads, 0, s>>>(p, work, done);
    return cudaGetLastError();
}

using BatchFn = cudaError_t (*)(const BatchParams *, unsigned *, unsigned *, int, cudaStream_t, int *, void **);

// min_blocks 0 marks the one-CTA-per-tile form (5 CTAs per SM), otherwise the
// persistent form with that many resident CTAs per SM.
struct BatchCandidate {
    int tile, width, min_blocks;
    BatchFn fn;
};

const BatchCandidate kCandF32[] = {
    {256, 4, 4, launch_batch_t<256, 4, GS_MOM_FP32, 4>}, {512, 4, 4, launch_batch_t<512, 4, GS_MOM_FP32, 4>},
    {256, 4, 3, launch_batch_t<256, 3, GS_MOM_FP32, 4>}, {256, 8, 4, launch_batch_t<256, 4, GS_MOM_FP32, 8>},
    {256, 4, 5, launch_batch_t<256, 5, GS_MOM_FP32, 4>}, {512, 4, 5, launch_batch_t<512, 5, GS_MOM_FP32, 4>},
    {256, 4, 0, launch_batch_grid_t<256, 5, GS_MOM_FP32, 4>},
};
const BatchCandidate kCandBf16[] = {
    {256, 8, 4, launch_batch_t<256, 4, GS_MOM_BF16, 8>}, {512, 8, 4, launch_batch_t<512, 4, GS_MOM_BF16, 8>},
    {256, 4, 4, launch_batch_t<256, 4, GS_MOM_BF16, 4>},
};
const BatchCandidate kCandHyb[] = {
    {256, 8, 4, launch_batch_t<256, 4, GS_MOM_BF16_HYBRID, 8>},
    {512, 8, 4, launch_batch_t<512, 4, GS_MOM_BF16_HYBRID, 8>},
    {256, 4, 4, launch_batch_t<256, 4, GS_MOM_BF16_HYBRID, 4>},
};

const BatchCandidate kCandF16B[] = {
    {256, 8, 4, launch_batch_t<256, 4, GS_MOM_FP16_BLOCK, 8>},
    {512, 8, 4, launch_batch_t<512, 4, GS_MOM_FP16_BLOCK, 8>},
    {256, 8, 5, launch_batch_t<256, 5, GS_MOM_FP16_BLOCK, 8>},
    {256, 8, 0, launch_batch_grid_t<256, 5, GS_MOM_FP16_BLOCK, 8>},
};

const BatchCandidate *candidates(int prec, int *n)
{
    switch (prec) {
    case GS_MOM_FP32: *n = 7; return kCandF32;
    case GS_MOM_BF16: *n = 3; return kCandBf16;
    case GS_MOM_BF16_HYBRID: *n = 3; return kCandHyb;
    case GS_MOM_FP16_BLOCK: *n = 4; return kCandF16B;
    default: *n = 0; return nullptr;
    }
}

}  // namespace

int batch_candidates(int prec) { int n = 0; candidates(prec, &n); return n; }

void batch_candidate_info(int prec, int c, int *tile, int *width, int *min_blocks)
{
    int n = 0;
    const BatchCandidate *cs = candidates(prec, &n);
    *tile = cs[c].tile;
    *width = cs[c].width;
    *min_blocks = cs[c].min_blocks;
}

cudaError_t launch_batch(const BatchParams *p, unsigned *work, unsigned *done, int total_tiles, int prec, int cand,
                         cudaStream_t s, int *grid, void **fn)
{
    int n = 0;
    const BatchCandidate *cs = candidates(prec, &n);
    if (cand < 0 || cand >= n) return cudaErrorInvalidValue;
    return cs[cand].fn(p, work, done, total_tiles, s, grid, fn);
}

}  // namespace gs
