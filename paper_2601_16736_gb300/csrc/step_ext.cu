// The step with its optional terms: position noise (App. Eq.
// disentangled_mu), the Artificial Implicit Update of sampled invisible
// primitives (Sec. 3.2), and the active count N_a (Sec. 4, opacity > 1/255).
// Launched when a step asks for AIU or for noise on every row, the terms
// that touch invisible rows; the count and noise on visible rows alone take
// the terms form of the plain step kernel, and the plain step is untouched
// by any of them.
//
// Per tile of 256 rows (one CTA of 256 threads; 5 CTAs per SM for FP32 and
// BF16 moments, 4 for the others):
//   A. visibility, StSS, AIU and noise decisions per row.  A row that takes
//      the noise has it computed here, from its values before this step, and
//      kept in shared memory; a noise-only invisible row is finished here.
//      Rows no item touches are counted for N_a here.  Two lists: visible
//      rows, and invisible rows with RSR and/or AIU.
//   B. the plain step's items: SH items and 3 small items per listed row.
//      The xyz item subtracts the kept noise; the opacity item counts N_a.

#include "step_common.cuh"

namespace gs {
namespace {

constexpr uint8_t kFRsr = 1, kFAiu = 2, kFNoise = 4;

// The AIU step of one value from unchanged moments: theta - lr m^/(sqrt(v^) + eps).
__device__ __forceinline__ float aiu_element(float th, float m, float v, float2 f, float eps, float lr)
{
    return fmaf(-lr, (m * f.x) / fmaf(sqrtf(v), f.y, eps), th);
}

// SH item i of an invisible row with RSR and/or AIU: the AIU step of its
// attributes from the current moments, then the RSR scaling of the moments.
template <int kPrec, int kW>
__device__ __forceinline__ void inv_sh_item(const StepArgs &a, const int32_t row, const int i, const uint8_t fl,
                                            const float2 f)
{
    using S = State<kPrec>;
    float m[kW], v[kW];
    uint32_t t = 0;
    S::template load_sh<kW>(a, row, i, m, v, t);
    if (fl & kFAiu) {
        const size_t off = (size_t)row * 48 + kW * i;
#pragma unroll
        for (int q = 0; q < kW / 4; ++q) {
            float4 x = ld4(a.a_sh + off + 4 * q);
            const int e0 = 4 * q;
            const float l0 = ((i == 0 && e0 + 0 < 3) ? a.lr[4] : a.lr[5]) * a.aiu_scale;
            const float l1 = ((i == 0 && e0 + 1 < 3) ? a.lr[4] : a.lr[5]) * a.aiu_scale;
            const float l2 = ((i == 0 && e0 + 2 < 3) ? a.lr[4] : a.lr[5]) * a.aiu_scale;
            const float l3 = a.lr[5] * a.aiu_scale;
            x.x = aiu_element(x.x, m[e0], v[e0], f, a.eps, l0);
            x.y = aiu_element(x.y, m[e0 + 1], v[e0 + 1], f, a.eps, l1);
            x.z = aiu_element(x.z, m[e0 + 2], v[e0 + 2], f, a.eps, l2);
            x.w = aiu_element(x.w, m[e0 + 3], v[e0 + 3], f, a.eps, l3);
            st4(a.a_sh + off + 4 * q, x);
        }
    }
    if (fl & kFRsr) {
#pragma unroll
        for (int e = 0; e < kW; ++e) {
            m[e] *= a.alpha1;
            v[e] *= a.alpha2;
        }
        S::template store_sh<kW>(a, row, i, m, v, t);
    }
}

// FP16-block rows: small item c = 12 (rotation) or 13 (xyz, scale, opacity
// and t) of a listed row, with the optional terms as small_item_x.  Item 13
// returns whether the row is active after the step.
__device__ __forceinline__ bool small_item_x_f16b(const StepArgs &a, const int32_t row, const int c, const bool vis,
                                                  const uint8_t fl, const float2 f, const float3 nz)
{
    using S = State<GS_MOM_FP16_BLOCK>;
    const bool aiu = !vis && (fl & kFAiu);
    char *mr = S::row(a.m, row), *vr = S::row(a.v, row);
    const size_t r = (size_t)row;
    if (c == 12) {
        const uint2 um = *reinterpret_cast<const uint2 *>(mr + kF16BRot), uv = *reinterpret_cast<const uint2 *>(vr + kF16BRot);
        const uint32_t wm[2] = {um.x, um.y}, wv[2] = {uv.x, uv.y};
        float m[4], v[4];
        decode_w<4>(wm, dec_scale((uint8_t)mr[kF16BExp + 6]), m);
        decode_w<4>(wv, dec_scale((uint8_t)vr[kF16BExp + 6]), v);
        if (vis || aiu) {
            float *pt = a.a_rot + r * 4;
            float4 th = ld4(pt);
            const float l = a.lr[2];
            if (vis) {
                const float4 g = ldg4_stream(a.g_rot + r * 4);
                th.x = step_element(th.x, g.x, m[0], v[0], f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
                th.y = step_element(th.y, g.y, m[1], v[1], f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
                th.z = step_element(th.z, g.z, m[2], v[2], f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
                th.w = step_element(th.w, g.w, m[3], v[3], f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
            } else {
                const float la = l * a.aiu_scale;
                th.x = aiu_element(th.x, m[0], v[0], f, a.eps, la);
                th.y = aiu_element(th.y, m[1], v[1], f, a.eps, la);
                th.z = aiu_element(th.z, m[2], v[2], f, a.eps, la);
                th.w = aiu_element(th.w, m[3], v[3], f, a.eps, la);
            }
            st4(pt, th);
        }
        if (vis || (fl & kFRsr)) {             // an AIU step keeps the moments
            if (fl & kFRsr) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    m[q] *= a.alpha1;
                    v[q] *= a.alpha2;
                }
            }
            uint32_t hm[2], hv[2];
            const uint32_t em = encode_rn_w<4>(m, hm), ev = encode_sr_w<4>(v, hv, a, row, 6);
            __stcs(reinterpret_cast<uint2 *>(mr + kF16BRot), make_uint2(hm[0], hm[1]));
            __stcs(reinterpret_cast<uint2 *>(vr + kF16BRot), make_uint2(hv[0], hv[1]));
            mr[kF16BExp + 6] = (char)em;
            vr[kF16BExp + 6] = (char)ev;
        }
        return false;
    }
    const uint4 um = *reinterpret_cast<const uint4 *>(mr + kF16BXso), uv = *reinterpret_cast<const uint4 *>(vr + kF16BXso);
    const uint32_t wm[4] = {um.x, um.y, um.z, um.w & 0xffffu}, wv[4] = {uv.x, uv.y, uv.z, uv.w};
    float m[7], v[7];
    decode_w<7>(wm, dec_scale((uint8_t)mr[kF16BExp + 7]), m);
    decode_w<7>(wv, dec_scale((uint8_t)vr[kF16BExp + 7]), v);
    uint32_t t = um.w >> 16;
    float *px = a.a_xyz + r * 3, *ps = a.a_scale + r * 3, *po = a.a_op + r;
    float x0 = px[0], x1 = px[1], x2 = px[2], s0 = ps[0], s1 = ps[1], s2 = ps[2], op = *po;
    if (vis) {
        const float *gx = a.g_xyz + r * 3, *gs = a.g_scale + r * 3;
        const float g0 = __ldcs(gx), g1 = __ldcs(gx + 1), g2 = __ldcs(gx + 2);
        const float gs0 = __ldcs(gs), gs1 = __ldcs(gs + 1), gs2 = __ldcs(gs + 2), go = __ldcs(a.g_op + r);
        const bool ds = a.dar_s != 0, dop = a.dar_o != 0;
        // regulariser derivatives at the old values (App. Eqs. scale, opacity)
        const float r0s = ds ? expf(s0) : 0.f, r1s = ds ? expf(s1) : 0.f, r2s = ds ? expf(s2) : 0.f;
        const float rop = dop ? dsigmoid(op) : 0.f;
        x0 = step_element(x0, g0, m[0], v[0], f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
        x1 = step_element(x1, g1, m[1], v[1], f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
        x2 = step_element(x2, g2, m[2], v[2], f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
        s0 = step_element(s0, gs0, m[3], v[3], f.x, f.y, a, a.lr[1], ds, r0s, a.lam_s, a.clip_s);
        s1 = step_element(s1, gs1, m[4], v[4], f.x, f.y, a, a.lr[1], ds, r1s, a.lam_s, a.clip_s);
        s2 = step_element(s2, gs2, m[5], v[5], f.x, f.y, a, a.lr[1], ds, r2s, a.lam_s, a.clip_s);
        op = step_element(op, go, m[6], v[6], f.x, f.y, a, a.lr[3], dop, rop, a.lam_o, a.clip_o);
        t = min(t + 1u, 65535u);                // the row's own step count (Sec. 3.2)
    } else if (aiu) {
        const float lx = a.lr[0] * a.aiu_scale, ls = a.lr[1] * a.aiu_scale;
        x0 = aiu_element(x0, m[0], v[0], f, a.eps, lx);
        x1 = aiu_element(x1, m[1], v[1], f, a.eps, lx);
        x2 = aiu_element(x2, m[2], v[2], f, a.eps, lx);
        s0 = aiu_element(s0, m[3], v[3], f, a.eps, ls);
        s1 = aiu_element(s1, m[4], v[4], f, a.eps, ls);
        s2 = aiu_element(s2, m[5], v[5], f, a.eps, ls);
        op = aiu_element(op, m[6], v[6], f, a.eps, a.lr[3] * a.aiu_scale);
    }
    if (vis || (fl & kFRsr)) {
        if (fl & kFRsr) {
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                m[q] *= a.alpha1;
                v[q] *= a.alpha2;
            }
        }
        uint32_t hm[4], hv[4];
        const uint32_t em = encode_rn_w<7>(m, hm), ev = encode_sr_w<7>(v, hv, a, row, 0);
        __stcs(reinterpret_cast<uint4 *>(mr + kF16BXso), make_uint4(hm[0], hm[1], hm[2], hm[3] | t << 16));
        __stcs(reinterpret_cast<uint4 *>(vr + kF16BXso), make_uint4(hv[0], hv[1], hv[2], hv[3]));
        mr[kF16BExp + 7] = (char)em;
        vr[kF16BExp + 7] = (char)ev;
    }
    if (vis || aiu) {
        __stcs(ps, s0); __stcs(ps + 1, s1); __stcs(ps + 2, s2);
        __stcs(po, op);
    }
    if (vis || aiu || (fl & kFNoise)) {
        __stcs(px, x0 - nz.x); __stcs(px + 1, x1 - nz.y); __stcs(px + 2, x2 - nz.z);
    }
    return op > a.tau_act;
}

// Small item c of a listed row, as small_item of the plain step, with the
// optional terms.  vis: Sparse Adam + DAR, t += 1 (where chunk 14 keeps t);
// otherwise kFAiu: the AIU step from the current moments.  kFRsr scales the
// moments afterwards; chunk 13 subtracts the row's noise `nz` from xyz.
// Chunk 14 returns whether the row is active after the step.
template <int kPrec>
__device__ __forceinline__ bool small_item_x(const StepArgs &a, const int32_t row, const int c, const bool vis,
                                             const uint8_t fl, const float2 f, const float3 nz)
{
    if constexpr (kPrec == GS_MOM_FP16_BLOCK) {
        return small_item_x_f16b(a, row, c, vis, fl, f, nz);
    } else {
    using S = State<kPrec>;
    const bool aiu = !vis && (fl & kFAiu);
    Chunk k = S::load_small(a, row, c);
    float4 &m = k.m, &v = k.v;
    const size_t r = (size_t)row;
    bool active = false;
    if (c == 12) {
        float *pt = a.a_rot + r * 4;
        if (vis || aiu) {
            float4 th = ld4(pt);
            const float l = a.lr[2];
            if (vis) {
                const float4 g = ldg4_stream(a.g_rot + r * 4);
                th.x = step_element(th.x, g.x, m.x, v.x, f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
                th.y = step_element(th.y, g.y, m.y, v.y, f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
                th.z = step_element(th.z, g.z, m.z, v.z, f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
                th.w = step_element(th.w, g.w, m.w, v.w, f.x, f.y, a, l, false, 0.f, 0.f, 0.f);
            } else {
                const float la = l * a.aiu_scale;
                th.x = aiu_element(th.x, m.x, v.x, f, a.eps, la);
                th.y = aiu_element(th.y, m.y, v.y, f, a.eps, la);
                th.z = aiu_element(th.z, m.z, v.z, f, a.eps, la);
                th.w = aiu_element(th.w, m.w, v.w, f, a.eps, la);
            }
            st4(pt, th);
        }
    } else if (c == 13) {
        float *px = a.a_xyz + r * 3;
        float *ps = a.a_scale + r * 3;
        float x0 = px[0], x1 = px[1], x2 = px[2], s0 = ps[0];
        if (vis) {
            const float *gx = a.g_xyz + r * 3;
            const float g0 = __ldcs(gx), g1 = __ldcs(gx + 1), g2 = __ldcs(gx + 2), gs0 = __ldcs(a.g_scale + r * 3);
            const bool ds = a.dar_s != 0;
            const float r0s = ds ? expf(s0) : 0.f;
            x0 = step_element(x0, g0, m.x, v.x, f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
            x1 = step_element(x1, g1, m.y, v.y, f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
            x2 = step_element(x2, g2, m.z, v.z, f.x, f.y, a, a.lr[0], false, 0.f, 0.f, 0.f);
            s0 = step_element(s0, gs0, m.w, v.w, f.x, f.y, a, a.lr[1], ds, r0s, a.lam_s, a.clip_s);
        } else if (aiu) {
            const float lx = a.lr[0] * a.aiu_scale;
            x0 = aiu_element(x0, m.x, v.x, f, a.eps, lx);
            x1 = aiu_element(x1, m.y, v.y, f, a.eps, lx);
            x2 = aiu_element(x2, m.z, v.z, f, a.eps, lx);
            s0 = aiu_element(s0, m.w, v.w, f, a.eps, a.lr[1] * a.aiu_scale);
        }
        if (vis || aiu || (fl & kFNoise)) {
            __stcs(px, x0 - nz.x); __stcs(px + 1, x1 - nz.y); __stcs(px + 2, x2 - nz.z);
        }
        if (vis || aiu) __stcs(ps, s0);
    } else {
        float *ps = a.a_scale + r * 3;
        float *po = a.a_op + r;
        float s1 = ps[1], s2 = ps[2], op = *po;
        if (vis) {
            const float *gsp = a.g_scale + r * 3;
            const float gs1 = __ldcs(gsp + 1), gs2 = __ldcs(gsp + 2), go = __ldcs(a.g_op + r);
            const bool ds = a.dar_s != 0, dop = a.dar_o != 0;
            const float r1s = ds ? expf(s1) : 0.f, r2s = ds ? expf(s2) : 0.f;
            const float rop = dop ? dsigmoid(op) : 0.f;
            s1 = step_element(s1, gs1, m.x, v.x, f.x, f.y, a, a.lr[1], ds, r1s, a.lam_s, a.clip_s);
            s2 = step_element(s2, gs2, m.y, v.y, f.x, f.y, a, a.lr[1], ds, r2s, a.lam_s, a.clip_s);
            op = step_element(op, go, m.z, v.z, f.x, f.y, a, a.lr[3], dop, rop, a.lam_o, a.clip_o);
            if (!S::kTInSh) k.t += 1u;         // the row's own step count (Sec. 3.2)
        } else if (aiu) {
            const float ls = a.lr[1] * a.aiu_scale;
            s1 = aiu_element(s1, m.x, v.x, f, a.eps, ls);
            s2 = aiu_element(s2, m.y, v.y, f, a.eps, ls);
            op = aiu_element(op, m.z, v.z, f, a.eps, a.lr[3] * a.aiu_scale);
        }
        if (vis || aiu) {
            __stcs(ps + 1, s1); __stcs(ps + 2, s2);
            __stcs(po, op);
        }
        active = op > a.tau_act;
    }
    if (fl & kFRsr) {      // RSR post-scale (Eq. meth::restate); chunk 14 holds 3 moments
        m.x *= a.alpha1; m.y *= a.alpha1; m.z *= a.alpha1;
        v.x *= a.alpha2; v.y *= a.alpha2; v.z *= a.alpha2;
        if (c != 14) { m.w *= a.alpha1; v.w *= a.alpha2; }
    }
    if (vis || (fl & kFRsr)) S::store_small(a, row, c, k);    // an AIU step keeps the moments
    return active;
    }
}

// Shared-memory lists of one tile of the extended step.
template <int kTile>
struct TileListsX {
    int32_t list[kTile];      // visible rows
    int32_t ilist[kTile];     // invisible rows with RSR and/or AIU
    float2 fac[kTile];        // bias factors of the visible rows (count t + 1)
    float2 ifac[kTile];       // bias factors of the AIU rows (count t)
    float3 nz[kTile];         // noise of the visible rows (zero without)
    float3 inz[kTile];        // noise of the listed invisible rows
    uint8_t vflag[kTile];
    uint8_t iflag[kTile];
    int32_t cnt[2][kTile / 32];
    unsigned active;
};

__device__ __forceinline__ float2 factors(const StepArgs &a, uint32_t k)
{
    return k < (uint32_t)a.fac_len ? a.fac[k] : make_float2(1.0f, 1.0f);
}

// Phase A of the extended step; returns the two list lengths.
template <int kTile, int kRowBytes, int kTByte>
__device__ __forceinline__ void tile_decide_x(const StepArgs &a, const int vis_src, const int64_t r0,
                                              TileListsX<kTile> &L, int &nv, int &ni)
{
    constexpr int kRpt = kTile / kThreads;
    constexpr int kWarps = kThreads / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nrow = (int)min((int64_t)kTile, (int64_t)a.n_rows - r0);
    unsigned bal_v[kRpt], bal_i[kRpt];
    uint8_t flag[kRpt];
    uint32_t t_old[kRpt];
    float3 nz[kRpt];
    unsigned my_active = 0;
#pragma unroll
    for (int j = 0; j < kRpt; ++j) {
        const int lr = j * kThreads + tid;
        const int64_t row = r0 + lr;
        const bool in = lr < nrow;
        bool vis = false, in_i = false;
        uint8_t fl = 0;
        t_old[j] = 0;
        nz[j] = make_float3(0.f, 0.f, 0.f);
        if (in) {
            const float *p = a.a_xyz + row * 3;
            if (vis_src == kVisCamera) vis = frustum_visible(p[0], p[1], p[2], a.cam);
            else if (vis_src == kVisMask) vis = a.mask_in[row] != 0;
            else vis = true;
            if (a.mask_out) a.mask_out[row] = vis ? 1 : 0;
            if (a.restate && stss_sampled(a, (int32_t)row)) fl |= kFRsr;
            if (a.noise == GS_NOISE_ALL || (a.noise == GS_NOISE_VISIBLE && vis)) fl |= kFNoise;
            const bool aiu_draw = a.aiu && !vis && aiu_sampled(a, (int32_t)row);
            if ((vis || aiu_draw) && !a.bias_mode) {
                const char *tp = static_cast<const char *>(a.m) + (size_t)row * kRowBytes + kTByte;
                if constexpr (kTByte % 4 == 0) t_old[j] = *reinterpret_cast<const uint32_t *>(tp);
                else t_old[j] = *reinterpret_cast<const uint16_t *>(tp);      // FP16-block rows: uint16 t
            }
            // a primitive never seen has no moments: its AIU step is zero
            if (aiu_draw && (a.bias_mode || t_old[j] > 0u)) fl |= kFAiu;
            in_i = !vis && (fl & (kFRsr | kFAiu));
            float tau = 0.f;
            if ((fl & kFNoise) || (a.n_active && !vis && !in_i)) tau = a.a_op[row];
            if (fl & kFNoise) {
                const float4 q = ld4(a.a_rot + row * 4);
                const float *ps = a.a_scale + row * 3;
                nz[j] = noise_term(a, (int32_t)row, q, ps[0], ps[1], ps[2], tau);
                if (!vis && !in_i) {           // noise-only row: finished here
                    float *px = a.a_xyz + row * 3;
                    const float x0 = px[0], x1 = px[1], x2 = px[2];
                    __stcs(px, x0 - nz[j].x); __stcs(px + 1, x1 - nz[j].y); __stcs(px + 2, x2 - nz[j].z);
                }
            }
            if (a.n_active && !vis && !in_i) my_active += tau > a.tau_act ? 1u : 0u;
        }
        flag[j] = fl;
        bal_v[j] = __ballot_sync(0xffffffffu, vis);
        bal_i[j] = __ballot_sync(0xffffffffu, in_i);
        if (lane == 0) {
            L.cnt[0][j * kWarps + warp] = __popc(bal_v[j]);
            L.cnt[1][j * kWarps + warp] = __popc(bal_i[j]);
        }
    }
    if (tid == 0) L.active = 0u;
    __syncthreads();
    if (a.n_active) {
        my_active = __reduce_add_sync(0xffffffffu, my_active);
        if (lane == 0 && my_active) atomicAdd(&L.active, my_active);
    }
    nv = ni = 0;
    for (int q = 0; q < kRpt * kWarps; ++q) {
        nv += L.cnt[0][q];
        ni += L.cnt[1][q];
    }
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kRpt; ++j) {
        const int me = j * kWarps + warp;
        int bv = 0, bi = 0;
        for (int q = 0; q < me; ++q) {
            bv += L.cnt[0][q];
            bi += L.cnt[1][q];
        }
        const int32_t row = (int32_t)(r0 + j * kThreads + tid);
        const unsigned me_bit = 1u << lane;
        if (bal_v[j] & me_bit) {
            const int pos = bv + __popc(bal_v[j] & lt);
            L.list[pos] = row;
            if (sparse_tile<kTile>(nv)) prefetch_row_l2<kRowBytes>(a, row);
            L.vflag[pos] = flag[j];
            L.fac[pos] = factors(a, a.bias_mode ? a.k_bias : t_old[j] + 1u);
            L.nz[pos] = nz[j];
        }
        if (bal_i[j] & me_bit) {
            const int pos = bi + __popc(bal_i[j] & lt);
            L.ilist[pos] = row;
            L.iflag[pos] = flag[j];
            L.ifac[pos] = (flag[j] & kFAiu) ? factors(a, a.bias_mode ? a.k_bias : t_old[j])
                                            : make_float2(1.0f, 1.0f);
            L.inz[pos] = nz[j];
        }
    }
    if (tid == 0 && a.n_visible && nv) atomicAdd(a.n_visible, (unsigned long long)nv);
    __syncthreads();
}

template <int kTile, int kMinBlocks, int kPrec, int kW>
__global__ void __launch_bounds__(kThreads, kMinBlocks) step_tile_x(const StepArgs a, const int vis_src)
{
    static_assert(kTile % kThreads == 0, "tile must be a multiple of the block");
    using S = State<kPrec>;
    constexpr int kNsh = 48 / kW;
    __shared__ TileListsX<kTile> L;
    pdl_enter();
    prefetch_tile_ahead<kTile>(a, vis_src);
    prefetch_tile_ahead_x<kTile>(a);
    const int64_t r0 = (int64_t)blockIdx.x * kTile;
    int nv, ni;
    tile_decide_x<kTile, S::kRowBytes, S::kTByte>(a, vis_src, r0, L, nv, ni);

    unsigned my_active = 0;
    constexpr int kSmall = kSmallItems<kPrec>, kOpItem = 11 + kSmall;     // the item holding the opacity
    const int e_sh = kNsh * nv, e_vis = e_sh + kSmall * nv, e_ish = e_vis + kNsh * ni, e_all = e_ish + kSmall * ni;
    // One flat item space walked as four loops, one per item kind, with the
    // item-to-thread assignment a single loop would give: the kinds do not
    // share a loop body, so their register demands do not add up.
    int w = threadIdx.x;
    for (; w < e_sh; w += kThreads) {
        const int j = w / kNsh, i = w - j * kNsh;
        sh_item<kPrec, kW>(a, L.list[j], i, (L.vflag[j] & kFRsr) != 0, L.fac[j]);
    }
    for (; w < e_vis; w += kThreads) {
        const int q = w - e_sh;
        const int j = q % nv, c = 12 + q / nv;
        const bool act = small_item_x<kPrec>(a, L.list[j], c, true, L.vflag[j], L.fac[j], L.nz[j]);
        my_active += (c == kOpItem && act) ? 1u : 0u;
    }
    for (; w < e_ish; w += kThreads) {
        const int q = w - e_vis;
        const int j = q / kNsh, i = q - j * kNsh;
        inv_sh_item<kPrec, kW>(a, L.ilist[j], i, L.iflag[j], L.ifac[j]);
    }
    for (; w < e_all; w += kThreads) {
        const int q = w - e_ish;
        const int j = q % ni, c = 12 + q / ni;
        const bool act = small_item_x<kPrec>(a, L.ilist[j], c, false, L.iflag[j], L.ifac[j], L.inz[j]);
        my_active += (c == kOpItem && act) ? 1u : 0u;
    }
    if (a.n_active) {
        my_active = __reduce_add_sync(0xffffffffu, my_active);
        if ((threadIdx.x & 31) == 0 && my_active) atomicAdd(&L.active, my_active);
        __syncthreads();
        if (threadIdx.x == 0 && L.active) atomicAdd(a.n_active, (unsigned long long)L.active);
    }
}

}  // namespace

constexpr int kExtTile = 256;
// Resident CTAs per SM: 5 for FP32 and BF16 moments (48 registers, no
// spills; BF16 4 % faster than at 4), 4 for the hybrid and FP16-block
// formats (at 5 they spill and gain nothing).
template <int kPrec>
constexpr int kExtMinBlocks = (kPrec == GS_MOM_FP32 || kPrec == GS_MOM_BF16) ? 5 : 4;

namespace {

template <int kPrec, int kW>
cudaError_t launch_ext_t(const StepArgs &a, int vis_src, cudaStream_t s)
{
    auto k = step_tile_x<kExtTile, kExtMinBlocks<kPrec>, kPrec, kW>;
    static int s_res[64] = {};
    StepArgs b = a;
    b.tile_ahead = resident_ctas(reinterpret_cast<const void *>(k), s_res);
    const unsigned grid = (unsigned)((a.n_rows + kExtTile - 1) / kExtTile);
    return launch_pdl(k, grid, kThreads, s, b, vis_src);
}

}  // namespace

cudaError_t launch_step_ext(const StepArgs &a, int prec, int vis_src, cudaStream_t s)
{
    if (a.n_rows <= 0) return cudaSuccess;
    switch (prec) {
    case GS_MOM_FP32: return launch_ext_t<GS_MOM_FP32, 4>(a, vis_src, s);
    case GS_MOM_BF16: return launch_ext_t<GS_MOM_BF16, 8>(a, vis_src, s);
    case GS_MOM_BF16_HYBRID: return launch_ext_t<GS_MOM_BF16_HYBRID, 8>(a, vis_src, s);
    case GS_MOM_FP16_BLOCK: return launch_ext_t<GS_MOM_FP16_BLOCK, 8>(a, vis_src, s);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace gs
