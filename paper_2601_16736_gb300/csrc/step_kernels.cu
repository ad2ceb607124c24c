// Fused AdamW-GS step: visibility decision, shared-memory compaction of the
// visible rows of a tile, Sparse Adam + DAR on the visible rows, RSR on the
// StSS-sampled rows — one pass over HBM per step.
//
// Work decomposition (one CTA = one tile of kTile consecutive rows, 256
// threads):
//   A. each thread decides visibility (camera frustum test of the mean,
//      caller mask, or all-visible) and StSS membership for kTile/256 rows;
//      warp ballots + a per-(chunk, warp) count table give every visible row
//      its position in a shared-memory list, ascending by row.
//   B. one thread per visible row reads its step counter and stages the two
//      bias-correction factors in shared memory.
//   C. a flat loop over work items: 12 SH items per visible row (one float4
//      of 4 SH columns each — a warp covers 2.7 rows of contiguous 192-B SH
//      rows and 256-B state rows), 1 item per visible row for the 11 small
//      columns (xyz, scale, rotation, opacity: scalar / float4 loads of the
//      caller's SoA groups, 3 float4 of the state row, DAR terms, t += 1),
//      and 15 state-only items per invisible StSS-sampled row (RSR).
// Every row's attributes, moments and counter are read and written by exactly
// one thread per column group, once.

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ float4 ldg4_stream(const float *p)
{
    return __ldcs(reinterpret_cast<const float4 *>(p));
}
__device__ __forceinline__ void st4(float *p, float4 x) { *reinterpret_cast<float4 *>(p) = x; }

// ---------------------------------------------------------------- FP32 state
struct StateF32 {
    static __device__ __forceinline__ float *row(void *base, int32_t r)
    {
        return static_cast<float *>(base) + (size_t)r * kSlots;
    }
    static __device__ __forceinline__ uint32_t load_t(void *m, int32_t r)
    {
        return reinterpret_cast<const uint32_t *>(row(m, r))[kSlotT];
    }
};

template <int kTile>
__global__ void __launch_bounds__(kThreads) step_tile_f32(const StepArgs a, const int vis_src)
{
    static_assert(kTile % kThreads == 0, "tile must be a multiple of the block");
    constexpr int kRpt = kTile / kThreads;    // rows per thread in phase A
    constexpr int kWarps = kThreads / 32;

    __shared__ int32_t s_list[kTile];         // visible rows, bit 31 = StSS-sampled
    __shared__ int32_t s_rlist[kTile];        // invisible StSS-sampled rows
    __shared__ float2 s_fac[kTile];
    __shared__ int32_t s_cnt[2][kRpt * kWarps];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t r0 = (int64_t)blockIdx.x * kTile;

    // ---- A: decide and compact
    unsigned bal_v[kRpt], bal_r[kRpt], bal_s[kRpt];
#pragma unroll
    for (int j = 0; j < kRpt; ++j) {
        const int64_t row = r0 + j * kThreads + tid;
        const bool in = row < a.n_rows;
        bool vis = false, smp = false;
        if (in) {
            if (vis_src == kVisCamera) {
                const float *p = a.a_xyz + row * 3;
                vis = frustum_visible(p[0], p[1], p[2], a.cam);
            } else if (vis_src == kVisMask) {
                vis = a.mask_in[row] != 0;
            } else {
                vis = true;
            }
            if (a.mask_out) a.mask_out[row] = vis ? 1 : 0;
            if (a.restate) smp = stss_sampled(a, (int32_t)row);
        }
        bal_v[j] = __ballot_sync(0xffffffffu, vis);
        bal_s[j] = __ballot_sync(0xffffffffu, smp);
        bal_r[j] = bal_s[j] & ~bal_v[j];
        if (lane == 0) {
            s_cnt[0][j * kWarps + warp] = __popc(bal_v[j]);
            s_cnt[1][j * kWarps + warp] = __popc(bal_r[j]);
        }
    }
    __syncthreads();
    int nv = 0, nr = 0;
#pragma unroll 4
    for (int q = 0; q < kRpt * kWarps; ++q) {
        nv += s_cnt[0][q];
        nr += s_cnt[1][q];
    }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kRpt; ++j) {
        const int me = j * kWarps + warp;
        int bv = 0, br = 0;
        for (int q = 0; q < me; ++q) {
            bv += s_cnt[0][q];
            br += s_cnt[1][q];
        }
        const int32_t row = (int32_t)(r0 + j * kThreads + tid);
        if (bal_v[j] & (1u << lane)) {
            const bool smp = (bal_s[j] >> lane) & 1u;
            s_list[bv + __popc(bal_v[j] & lt)] = row | (smp ? (int32_t)0x80000000 : 0);
        }
        if (bal_r[j] & (1u << lane)) s_rlist[br + __popc(bal_r[j] & lt)] = row;
    }
    if (tid == 0 && a.n_visible && nv) atomicAdd(a.n_visible, (unsigned long long)nv);
    __syncthreads();

    // ---- B: per-row bias-correction factors
    for (int j = tid; j < nv; j += kThreads) {
        const int32_t row = s_list[j] & 0x7fffffff;
        const uint32_t tnew = StateF32::load_t(a.m, row) + 1u;
        const uint32_t tb = a.bias_mode ? a.k_bias : tnew;
        s_fac[j] = (tb < (uint32_t)a.fac_len) ? a.fac[tb] : make_float2(1.0f, 1.0f);
    }
    __syncthreads();

    // ---- C: flat work loop
    const int n_sh = 12 * nv, n_vis = 13 * nv, n_all = 13 * nv + 15 * nr;
    for (int w = tid; w < n_all; w += kThreads) {
        if (w < n_sh) {
            // 4 SH columns of one visible row
            const int j = w / 12, c = w - j * 12;
            const int32_t e = s_list[j];
            const int32_t row = e & 0x7fffffff;
            const float2 f = s_fac[j];
            const size_t off = (size_t)row * 48 + c * 4;
            float4 th = ld4(a.a_sh + off);
            const float4 g = ldg4_stream(a.g_sh + off);
            float *mr = StateF32::row(a.m, row) + kSlotSh + c * 4;
            float *vr = StateF32::row(a.v, row) + kSlotSh + c * 4;
            float4 m = ld4(mr), v = ld4(vr);
            const float lr_dc = a.lr[4], lr_rest = a.lr[5];
            th.x = step_element(th.x, g.x, m.x, v.x, f.x, f.y, a, c == 0 ? lr_dc : lr_rest, false, 0.f, 0.f, 0.f);
            th.y = step_element(th.y, g.y, m.y, v.y, f.x, f.y, a, c == 0 ? lr_dc : lr_rest, false, 0.f, 0.f, 0.f);
            th.z = step_element(th.z, g.z, m.z, v.z, f.x, f.y, a, c == 0 ? lr_dc : lr_rest, false, 0.f, 0.f, 0.f);
            th.w = step_element(th.w, g.w, m.w, v.w, f.x, f.y, a, lr_rest, false, 0.f, 0.f, 0.f);
            if (e < 0) {
                m.x *= a.alpha1; m.y *= a.alpha1; m.z *= a.alpha1; m.w *= a.alpha1;
                v.x *= a.alpha2; v.y *= a.alpha2; v.z *= a.alpha2; v.w *= a.alpha2;
            }
            st4(a.a_sh + off, th);
            st4(mr, m);
            st4(vr, v);
        } else if (w < n_vis) {
            // the 11 small columns of one visible row + its step counter
            const int j = w - n_sh;
            const int32_t e = s_list[j];
            const int32_t row = e & 0x7fffffff;
            const float2 f = s_fac[j];
            float *mr = StateF32::row(a.m, row);
            float *vr = StateF32::row(a.v, row);
            float4 m0 = ld4(mr + 48), m1 = ld4(mr + 52), m2 = ld4(mr + 56);
            float4 v0 = ld4(vr + 48), v1 = ld4(vr + 52), v2 = ld4(vr + 56);
            float4 rot = ld4(a.a_rot + (size_t)row * 4);
            const float4 grot = ldg4_stream(a.g_rot + (size_t)row * 4);
            float *px = a.a_xyz + (size_t)row * 3;
            float *ps = a.a_scale + (size_t)row * 3;
            const float *gx = a.g_xyz + (size_t)row * 3;
            const float *gs = a.g_scale + (size_t)row * 3;
            float x0 = px[0], x1 = px[1], x2 = px[2];
            float s0 = ps[0], s1 = ps[1], s2 = ps[2];
            float op = a.a_op[row];
            const float gx0 = __ldcs(gx), gx1 = __ldcs(gx + 1), gx2 = __ldcs(gx + 2);
            const float gs0 = __ldcs(gs), gs1 = __ldcs(gs + 1), gs2 = __ldcs(gs + 2);
            const float gop = __ldcs(a.g_op + row);

            const bool ds = a.dar_s != 0, dop = a.dar_o != 0;
            const float lr_x = a.lr[0], lr_s = a.lr[1], lr_r = a.lr[2], lr_o = a.lr[3];
            rot.x = step_element(rot.x, grot.x, m0.x, v0.x, f.x, f.y, a, lr_r, false, 0.f, 0.f, 0.f);
            rot.y = step_element(rot.y, grot.y, m0.y, v0.y, f.x, f.y, a, lr_r, false, 0.f, 0.f, 0.f);
            rot.z = step_element(rot.z, grot.z, m0.z, v0.z, f.x, f.y, a, lr_r, false, 0.f, 0.f, 0.f);
            rot.w = step_element(rot.w, grot.w, m0.w, v0.w, f.x, f.y, a, lr_r, false, 0.f, 0.f, 0.f);
            x0 = step_element(x0, gx0, m1.x, v1.x, f.x, f.y, a, lr_x, false, 0.f, 0.f, 0.f);
            x1 = step_element(x1, gx1, m1.y, v1.y, f.x, f.y, a, lr_x, false, 0.f, 0.f, 0.f);
            x2 = step_element(x2, gx2, m1.z, v1.z, f.x, f.y, a, lr_x, false, 0.f, 0.f, 0.f);
            // scale: dR/dkappa = exp(kappa) at the old value (App. Eq. scale)
            s0 = step_element(s0, gs0, m1.w, v1.w, f.x, f.y, a, lr_s, ds, ds ? expf(s0) : 0.f, a.lam_s, a.clip_s);
            s1 = step_element(s1, gs1, m2.x, v2.x, f.x, f.y, a, lr_s, ds, ds ? expf(s1) : 0.f, a.lam_s, a.clip_s);
            s2 = step_element(s2, gs2, m2.y, v2.y, f.x, f.y, a, lr_s, ds, ds ? expf(s2) : 0.f, a.lam_s, a.clip_s);
            // opacity: dR/dtau = sig'(tau) at the old value (App. Eq. opacity)
            op = step_element(op, gop, m2.z, v2.z, f.x, f.y, a, lr_o, dop, dop ? dsigmoid(op) : 0.f, a.lam_o, a.clip_o);
            m2.w = __uint_as_float(__float_as_uint(m2.w) + 1u);    // t += 1
            if (e < 0) {
                m0.x *= a.alpha1; m0.y *= a.alpha1; m0.z *= a.alpha1; m0.w *= a.alpha1;
                m1.x *= a.alpha1; m1.y *= a.alpha1; m1.z *= a.alpha1; m1.w *= a.alpha1;
                m2.x *= a.alpha1; m2.y *= a.alpha1; m2.z *= a.alpha1;
                v0.x *= a.alpha2; v0.y *= a.alpha2; v0.z *= a.alpha2; v0.w *= a.alpha2;
                v1.x *= a.alpha2; v1.y *= a.alpha2; v1.z *= a.alpha2; v1.w *= a.alpha2;
                v2.x *= a.alpha2; v2.y *= a.alpha2; v2.z *= a.alpha2;
            }
            st4(a.a_rot + (size_t)row * 4, rot);
            px[0] = x0; px[1] = x1; px[2] = x2;
            ps[0] = s0; ps[1] = s1; ps[2] = s2;
            a.a_op[row] = op;
            st4(mr + 48, m0); st4(mr + 52, m1); st4(mr + 56, m2);
            st4(vr + 48, v0); st4(vr + 52, v1); st4(vr + 56, v2);
        } else {
            // RSR on one float4 of an invisible sampled row (slot 59 of m is t)
            const int q = w - n_vis;
            const int j = q / 15, c = q - j * 15;
            const int32_t row = s_rlist[j];
            float *mr = StateF32::row(a.m, row) + c * 4;
            float *vr = StateF32::row(a.v, row) + c * 4;
            float4 m = ld4(mr), v = ld4(vr);
            m.x *= a.alpha1; m.y *= a.alpha1; m.z *= a.alpha1;
            v.x *= a.alpha2; v.y *= a.alpha2; v.z *= a.alpha2;
            if (c != 14) { m.w *= a.alpha1; v.w *= a.alpha2; }
            st4(mr, m);
            st4(vr, v);
        }
    }
}

}  // namespace

constexpr int kStepTile = 512;

cudaError_t launch_step(const StepArgs &a, int prec, int vis_src, cudaStream_t s)
{
    if (a.n_rows <= 0) return cudaSuccess;
    const unsigned grid = (unsigned)((a.n_rows + kStepTile - 1) / kStepTile);
    switch (prec) {
    case GS_MOM_FP32:
        step_tile_f32<kStepTile><<<grid, kThreads, 0, s>>>(a, vis_src);
        break;
    default:
        return cudaErrorNotSupported;
    }
    return cudaGetLastError();
}

}  // namespace gs
