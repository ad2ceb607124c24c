"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (FP32 kernels vs FP64 oracle): per attribute group
max|d| / max|ref| <= 1e-5 after one step and <= 1e-4 after 1000 steps;
after one step also elementwise |d| <= 1e-5 (|ref| + 1e-3).  Visibility
masks, compacted lists, counts, step counters and re-indexed state are
compared bit-exactly.
"""
import numpy as np
import pytest

from harness import check_mask, check_trajectory_masks, GpuScene, OracleRun, assert_close, group_errors
from paper_2601_16736_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

LR = synth.lr_for_step(1, 10)


@pytest.fixture(scope="module")
def G():
    from paper_2601_16736_gb300 import build
    build.build()
    from paper_2601_16736_gb300 import gsopt
    return gsopt


# ------------------------------------------------------------- visibility

@pytest.mark.parametrize("scene", ["uniform", "blobs"])
def test_visibility_matches_fp64_definition(G, orc, scene):
    """Mask, count and list against the oracle's FP64 frustum decision: equal
    everywhere except means within 1e-6 of a plane, which are counted and
    reported with the disagreements among them."""
    n = 250_001
    groups = synth.scene_uniform(n, 91) if scene == "uniform" else synth.scene_blobs(n, 92, 12.5)
    xyz = torch.from_numpy(groups["xyz"]).cuda()
    run = GpuScene(groups)
    mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
    rows = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    near = differ = 0
    for cam in synth.ring_cameras(6, (-30.0, 0.0, 30.0)):
        G.gs_visibility(run.h, xyz, G.make_camera(cam), mask, rows, cnt)
        torch.cuda.synchronize()
        got = mask.cpu().numpy()
        c = check_mask(orc, got, groups["xyz"], cam)
        near += c["near_plane"]
        differ += c["differ"]
        assert int(cnt.item()) == int(got.sum())
        lst = rows.cpu().numpy()[:int(cnt.item())]
        assert np.array_equal(np.sort(lst), np.nonzero(got)[0])
    print(f"means within 1e-6 of a frustum plane: {near}; decisions differing from FP64: {differ}")
    assert differ == 0
    run.close()


def _near_plane_means(cam, n, seed):
    """Means placed at relative distances 1e-8 .. 1e-4 from the side planes
    of `cam` (margins of about 1e-8 .. 1e-3): most fall inside the FP32
    evaluation's rounding band, where the kernels decide in FP64."""
    rng = np.random.default_rng(seed)
    R = cam[:9].reshape(3, 3).astype(np.float64)
    t = cam[9:12].astype(np.float64)
    tx, ty = float(cam[12]), float(cam[13])
    pz = rng.uniform(0.5, 40.0, n)
    side = rng.integers(0, 4, n)
    d = rng.normal(0, 1, n) * 10.0 ** rng.uniform(-8, -4, n)
    sgn = np.where(side % 2 == 0, 1.0, -1.0)
    px = np.where(side < 2, sgn * pz * tx * (1 + d), rng.uniform(-1, 1, n) * pz * tx)
    py = np.where(side >= 2, sgn * pz * ty * (1 + d), rng.uniform(-1, 1, n) * pz * ty)
    return np.linalg.solve(R, (np.stack([px, py, pz], 1) - t).T).T.astype(np.float32)


def _skewed_camera():
    """A camera whose R is not a rotation (scaled and sheared rows, a large
    translation): the kernels' rounding band must hold for any 3x3 R."""
    cam = synth.ring_cameras(4, (20.0,))[1].copy()
    R = cam[:9].reshape(3, 3).astype(np.float64)
    S = np.array([[2.5, 0.3, 0.0], [0.0, 0.7, -0.2], [0.1, 0.0, 1.6]])
    cam[:9] = (S @ R).reshape(-1).astype(np.float32)
    cam[9:12] = np.array([3.0, -7.5, 42.0], np.float32)
    cam[12], cam[13] = np.float32(0.9), np.float32(0.4)
    return cam


def test_visibility_exact_near_planes(G, orc):
    """Means inside the FP32 rounding band of the side planes: the GPU's
    decision (FP32, re-taken in FP64 inside twice the FP32 error bound)
    equals the FP64 definition away from 1e-6 of a plane, and in fact
    everywhere but within 1e-9 of one.  A plain FP32 evaluation differs from
    FP64 on thousands of these rows, many of them farther than 1e-6 from the
    plane."""
    n = 200_003
    tot = {"near_plane": 0, "differ": 0, "differ_beyond_1e-9": 0, "fp32_differ_beyond_1e-6": 0}
    for i, cam in enumerate(synth.ring_cameras(4, (-30.0, 0.0, 30.0)) + [_skewed_camera()]):
        xyz_np = _near_plane_means(cam, n, 1200 + i)
        run = GpuScene({"xyz": xyz_np, "scale": np.zeros((n, 3), np.float32), "rot": np.zeros((n, 4), np.float32),
                        "opacity": np.zeros((n, 1), np.float32), "sh": np.zeros((n, 48), np.float32)})
        mask = torch.zeros(n, dtype=torch.uint8, device="cuda")
        G.gs_visibility(run.h, run.attrs["xyz"], G.make_camera(cam), mask)
        got = mask.cpu().numpy()
        c = check_mask(orc, got, xyz_np, cam)
        margin, ref = orc.frustum_margin_f64(xyz_np, cam)
        tot["near_plane"] += c["near_plane"]
        tot["differ"] += c["differ"]
        tot["differ_beyond_1e-9"] += int(((got != ref) & (np.abs(margin) > 1e-9)).sum())
        f32 = orc.visibility_f32(xyz_np, cam)
        tot["fp32_differ_beyond_1e-6"] += int(((f32 != ref) & (np.abs(margin) > 1e-6)).sum())
        # the fused step takes the same decision
        run.step_camera(cam, G.make_params(LR, 1))
        torch.cuda.synchronize()
        assert np.array_equal(run.mask[:n].cpu().numpy(), got)
        run.close()
    print("near-plane means:", tot)
    assert tot["differ_beyond_1e-9"] == 0
    assert tot["fp32_differ_beyond_1e-6"] > 0, "the probe does not reach the FP32 rounding band"


def _runs_ascending(lst, tile):
    """Each tile of `tile` rows forms one contiguous, ascending run of the list."""
    ids = lst // tile
    starts = np.flatnonzero(np.r_[True, ids[1:] != ids[:-1]])
    assert len(np.unique(ids)) == len(starts), "a tile's rows are split across the list"
    same = ids[1:] == ids[:-1]
    assert np.all(lst[1:][same] > lst[:-1][same]), "rows within a tile not ascending"


@pytest.mark.parametrize("offset", [0, 1])
def test_visibility_layouts_and_list_order(G, orc, offset):
    """Aligned means (four rows per thread) and means starting 12 B past a
    16-B boundary (one row per thread) give the same mask, count and list
    set; each CTA's share of the list is one ascending run."""
    n = 100_003
    groups = synth.scene_blobs(n + offset, 93, 12.5)
    xyz_all = torch.from_numpy(groups["xyz"]).cuda()
    xyz = xyz_all[offset:]
    assert (xyz.data_ptr() % 16 == 0) == (offset == 0)
    run = GpuScene({k: v[offset:] for k, v in groups.items()})
    mask_all = torch.zeros(n + offset, dtype=torch.uint8, device="cuda")
    mask = mask_all[offset:]
    rows = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    for cam in synth.ring_cameras(4):
        G.gs_visibility(run.h, xyz, G.make_camera(cam), mask, rows, cnt)
        torch.cuda.synchronize()
        ref = mask.cpu().numpy()
        check_mask(orc, ref, groups["xyz"][offset:], cam)
        c = int(cnt.item())
        assert c == int(ref.sum())
        lst = rows.cpu().numpy()[:c]
        assert np.array_equal(np.sort(lst), np.nonzero(ref)[0])
        _runs_ascending(lst, 2048 if offset == 0 else 256)
        # mask alone, no list or count
        mask.zero_()
        G.gs_visibility(run.h, xyz, G.make_camera(cam), mask, None, None)
        torch.cuda.synchronize()
        assert np.array_equal(mask.cpu().numpy(), ref)
    if offset:
        assert int(mask_all[0].item()) == 0, "write before the mask's first row"
    run.close()


# ---------------------------------------------------------- one-step parity

@pytest.mark.parametrize("scene,restate", [("uniform", False), ("blobs", True)])
def test_one_step_parity(G, orc, scene, restate):
    n = 100_003
    groups = synth.scene_uniform(n, 101) if scene == "uniform" else synth.scene_blobs(n, 102, 12.5)
    grads = synth.grads_rows(n, 103)
    cam = synth.ring_cameras(8)[3]
    run = GpuScene(groups)
    run.set_grads(grads)
    p = G.make_params(LR, 100, restate=restate, restate_ratio=0.3, seed=7)
    run.step_camera(cam, p)
    got = run.rows()
    m, v, t = run.state()

    ref = OracleRun(orc, synth.to_rows(groups))
    vis = ref.visible(cam)
    assert np.array_equal(run.mask.cpu().numpy(), vis)
    assert int(run.nvis.item()) == int(vis.sum())
    ref.st.t[:] = 0
    ref.step(grads, vis, LR, True, True, 100, restate=restate, ratio=0.3, seed=7)
    assert_close(got, ref.st.theta, 1e-5, 1e-5, what="theta")
    assert_close(m, ref.st.m, 1e-5, what="m")
    assert_close(v, ref.st.v, 1e-5, what="v")
    assert np.array_equal(t, ref.st.t)
    inv = vis == 0
    assert np.array_equal(got[inv], synth.to_rows(groups)[inv])   # invisible rows untouched
    run.close()


@pytest.mark.parametrize("n", [1, 31, 33, 255, 257, 511, 512, 513, 1025, 1537])
@pytest.mark.parametrize("pattern", ["all", "none", "one", "random"])
def test_edge_sizes_and_masks(G, orc, n, pattern):
    groups = synth.scene_uniform(n, 200 + n)
    grads = synth.grads_rows(n, 300 + n)
    grads[n // 2] = 0.0                                 # a visible row with zero gradient: v stays 0
    rng = np.random.default_rng(n)
    if pattern == "all":
        mask_np = None
    elif pattern == "none":
        mask_np = np.zeros(n, np.uint8)
    elif pattern == "one":
        mask_np = np.zeros(n, np.uint8)
        mask_np[n - 1] = 1
    else:
        mask_np = (rng.random(n) < 0.5).astype(np.uint8)
    run = GpuScene(groups)
    run.set_grads(grads)
    ref = OracleRun(orc, synth.to_rows(groups))
    mask_t = None if mask_np is None else torch.from_numpy(mask_np).cuda()
    for k in (1, 2, 100):
        p = G.make_params(LR, k, restate=(k == 100), restate_ratio=1.0 if n % 2 else 0.5, seed=11)
        run.step_mask(mask_t, p)
        ref.step(grads, mask_np, LR, True, True, k, restate=(k == 100), ratio=1.0 if n % 2 else 0.5, seed=11)
    got = run.rows()
    m, v, t = run.state()
    assert_close(got, ref.st.theta, 1e-5, 1e-5, what="theta")
    assert_close(m, ref.st.m, 1e-5, what="m")
    assert_close(v, ref.st.v, 1e-5, what="v")
    assert np.array_equal(t, ref.st.t)
    if pattern == "none":
        assert got.tobytes() == synth.to_rows(groups).tobytes()
    run.close()


def test_global_bias_mode(G, orc):
    n = 5000
    groups = synth.scene_blobs(n, 401, 12.5)
    run = GpuScene(groups, bias_mode=1)
    ref = OracleRun(orc, synth.to_rows(groups), bias_mode=1)
    rng = np.random.default_rng(402)
    for k in range(1, 31):
        grads = synth.grads_rows(n, 403, k)
        mask_np = (rng.random(n) < 0.3).astype(np.uint8)
        run.set_grads(grads)
        run.step_mask(torch.from_numpy(mask_np).cuda(), G.make_params(LR, k))
        ref.step(grads, mask_np, LR, True, True, k)
    assert_close(run.rows(), ref.st.theta, 1e-5, what="theta")


@pytest.mark.parametrize("reg_mode", [1, 2, 3])
def test_regulariser_variants(G, orc, reg_mode):
    n = 4000
    groups = synth.scene_uniform(n, 500 + reg_mode)
    kw = dict(reg_mode=reg_mode)
    if reg_mode == 3:
        kw["lambda_o"] = 50.0                    # so the clip is active
    run = GpuScene(groups, **kw)
    ref = OracleRun(orc, synth.to_rows(groups), **kw)
    rng = np.random.default_rng(600)
    for k in range(1, 11):
        grads = synth.grads_rows(n, 601, k)
        mask_np = (rng.random(n) < 0.5).astype(np.uint8)
        nv = int(mask_np.sum())
        run.set_grads(grads)
        run.step_mask(torch.from_numpy(mask_np).cuda(), G.make_params(LR, k, n_visible=nv))
        ref.step(grads, mask_np, LR, True, True, k, n_visible=nv)
    assert_close(run.rows(), ref.st.theta, 1e-5, what=f"reg_mode {reg_mode}")


# ------------------------------------------------------------ multi-step

def _run_sequence(G, orc, wl, n_steps, sample=None):
    """Run n_steps of the workload's schedule on the GPU (all rows) and on the
    oracle (all rows, or the `sample` of row ids); returns the comparison."""
    groups = wl.scene_groups()
    cams = wl.cameras()
    order = synth.view_order(len(cams), n_steps, wl.seed)
    n = wl.n
    nbuf = wl.grad_buffers
    grads_host = [synth.grads_rows(n, wl.seed, b) for b in range(nbuf)]
    run = GpuScene(groups)
    gdev = []
    for gh in grads_host:
        gdev.append({k: torch.from_numpy(v).cuda() for k, v in synth.from_rows(gh).items()})
    ids = np.arange(n) if sample is None else np.asarray(sample)
    ref = OracleRun(orc, synth.to_rows(groups)[ids], row_ids=ids)
    diverged = np.zeros(ids.size, bool)
    n_ambiguous = 0
    ids_dev = torch.from_numpy(ids).cuda()
    for k in range(1, n_steps + 1):
        cam = cams[order[k - 1]]
        b = (k - 1) % nbuf
        lr = synth.lr_for_step(k, n_steps)
        rs = k % wl.restate_every == 0
        p = G.make_params(lr, k, dar_opacity=wl.dar, dar_scale=wl.dar, restate=rs,
                          restate_ratio=wl.restate_ratio, seed=wl.seed)
        gxyz = run.attrs["xyz"][ids_dev].cpu().numpy()          # the means this step decides on
        G.gs_step_camera(run.h, G.make_attrs(run.attrs), G.make_attrs(gdev[b]), G.make_camera(cam), p,
                         mask_out=run.mask)
        gmask = run.mask[ids_dev].cpu().numpy()
        omask = ref.visible(cam)
        differ = gmask != omask
        if differ.any():
            n_ambiguous += check_trajectory_masks(orc, gmask, omask, ref.st.theta[:, 0:3], gxyz, cam)
            diverged |= differ
        ref.step(grads_host[b][ids], omask, lr, wl.dar, wl.dar, k,
                 restate=rs, ratio=wl.restate_ratio, seed=wl.seed)
    got = run.rows()[ids]
    _, _, t = run.state()
    keep = ~diverged
    run.close()
    return got, ref, t[ids], keep, n_ambiguous


def test_multi_step_parity_small(G, orc):
    wl = synth.Workload("small", 20_011, 300, 777, "blobs", extent=12.5,
                        elevations=(-30.0, 0.0, 30.0), n_azimuth=20, grad_buffers=5)
    got, ref, t, keep, amb = _run_sequence(G, orc, wl, 300)
    assert keep.mean() > 0.999
    assert_close(got, ref.st.theta, 1e-4, rows=keep, what="300 steps")
    assert np.array_equal(t[keep], ref.st.t[keep])
    print("ambiguous decisions:", amb, group_errors(got, ref.st.theta, rows=keep))


@pytest.mark.parametrize("method", ["sparse_adam", "adamw_gs"])
def test_c1_full_workload(G, orc, method):
    """The 100 k-primitive, 50-step workload, every row against the oracle:
    plain Sparse Adam (no DAR, no RSR) and AdamW-GS (DAR every step, RSR
    every 25 steps so that two re-state events fall inside the run)."""
    import dataclasses
    wl = synth.WORKLOADS["c1_100k"]
    if method == "sparse_adam":
        wl = dataclasses.replace(wl, dar=False, restate_every=10 ** 9)
    else:
        wl = dataclasses.replace(wl, restate_every=25, restate_ratio=0.3)
    got, ref, t, keep, amb = _run_sequence(G, orc, wl, wl.steps)
    assert keep.mean() > 0.999
    errs = assert_close(got, ref.st.theta, 1e-4, rows=keep, what=f"{method}, {wl.steps} steps")
    assert np.array_equal(t[keep], ref.st.t[keep])
    assert (t > 0).mean() > 0.5                  # most rows were visible at some step
    print(method, "ambiguous decisions:", amb, errs)


def test_full_size_1000_steps_sampled(G, orc):
    """The 1 M-primitive, 1000-step workload in the launch configuration the
    bench times, checked on 3000 sampled primitives the oracle follows."""
    wl = synth.WORKLOADS["c2_1m"]
    sample = np.sort(np.random.default_rng(5).choice(wl.n, 3000, replace=False))
    got, ref, t, keep, amb = _run_sequence(G, orc, wl, wl.steps, sample=sample)
    assert keep.mean() > 0.998
    errs = assert_close(got, ref.st.theta, 1e-4, rows=keep, what="1000 steps")
    assert np.array_equal(t[keep], ref.st.t[keep])
    print("ambiguous decisions:", amb, errs)


# --------------------------------------------------------- state handling

def _random_state(n, seed):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=(n, 59)).astype(np.float32), rng.random((n, 59)).astype(np.float32),
            rng.integers(0, 1000, n).astype(np.uint32))


def test_export_import_roundtrip(G):
    n = 3001
    run = GpuScene(synth.scene_uniform(n, 700))
    m, v, t = _random_state(n, 701)
    G.gs_opt_import_state(run.h, torch.from_numpy(m).cuda(), torch.from_numpy(v).cuda(),
                          torch.from_numpy(t.view(np.int32)).cuda())
    m2, v2, t2 = run.state()
    assert m2.tobytes() == m.tobytes() and v2.tobytes() == v.tobytes() and t2.tobytes() == t.tobytes()
    run.close()


@pytest.mark.parametrize("n_new_kind", ["same", "grow", "shrink"])
def test_reindex_matches_oracle(G, orc, n_new_kind):
    n = 50_000
    run = GpuScene(synth.scene_uniform(n, 710))
    m, v, t = _random_state(n, 711)
    G.gs_opt_import_state(run.h, torch.from_numpy(m).cuda(), torch.from_numpy(v).cuda(),
                          torch.from_numpy(t.view(np.int32)).cuda())
    if n_new_kind == "same":
        src, reset, _ = synth.reindex_event(n, 712, 0)
    else:
        n_new = n + 7777 if n_new_kind == "grow" else n - 7777
        rng = np.random.default_rng(713)
        src = rng.integers(-1, n, n_new).astype(np.int32)
        reset = (rng.random(n_new) < 0.05).astype(np.uint8)
    G.gs_reindex_state(run.h, torch.from_numpy(src).cuda(), torch.from_numpy(reset).cuda(), src.size)
    run.n = src.size
    assert G.gs_opt_rows(run.h) == src.size
    m2, v2, t2 = run.state()
    st = orc.State(np.zeros((n, 59)), m.astype(np.float64), v.astype(np.float64), t)
    out = orc.reindex(st, src, reset)
    assert np.array_equal(m2.astype(np.float64), out.m) and np.array_equal(v2.astype(np.float64), out.v)
    assert np.array_equal(t2, out.t)
    assert G.gs_opt_sync_errors(run.h) == G.GS_OK
    run.close()


def test_reindex_out_of_range_is_reported_not_read(G):
    n = 1000
    run = GpuScene(synth.scene_uniform(n, 720))
    src = np.arange(n, dtype=np.int32)
    src[17] = n + 5
    G.gs_reindex_state(run.h, torch.from_numpy(src).cuda(), None, n)
    assert G.gs_opt_sync_errors(run.h) == G.GS_ERR_INVALID_ARG
    assert G.gs_opt_sync_errors(run.h) == G.GS_OK
    _, _, t = run.state()
    assert t[17] == 0
    run.close()


@pytest.mark.parametrize("n", [1, 17, 7001])
def test_gather_attrs(G, n):
    groups = synth.scene_uniform(n, 730 + n)
    run = GpuScene(groups)
    src, reset, attr_src = synth.reindex_event(n, 731, 0)
    attr_src = attr_src.copy()
    if attr_src.size > 2:
        attr_src[1] = -1                     # a negative entry leaves the output row untouched
    sentinel = -7.5
    out = {k: torch.full((attr_src.size, v.shape[1]), sentinel, dtype=torch.float32, device="cuda")
           for k, v in groups.items()}
    G.gs_gather_attrs(run.h, G.make_attrs(run.attrs), n, G.make_attrs(out), torch.from_numpy(attr_src).cuda(),
                      attr_src.size)
    torch.cuda.synchronize()
    assert G.gs_opt_sync_errors(run.h) == G.GS_OK
    for k, v in groups.items():
        got = out[k].cpu().numpy()
        ok = attr_src >= 0
        assert np.array_equal(got[ok], v[attr_src[ok]])
        assert np.all(got[~ok] == sentinel)
    # an out-of-range source is skipped and reported by the next sync
    bad = np.zeros(5, np.int32)
    bad[3] = n + 4
    out2 = {k: torch.full((5, v.shape[1]), sentinel, dtype=torch.float32, device="cuda") for k, v in groups.items()}
    G.gs_gather_attrs(run.h, G.make_attrs(run.attrs), n, G.make_attrs(out2), torch.from_numpy(bad).cuda(), 5)
    torch.cuda.synchronize()
    assert G.gs_opt_sync_errors(run.h) == G.GS_ERR_INVALID_ARG
    for k, v in groups.items():
        got = out2[k].cpu().numpy()
        assert np.all(got[3] == sentinel)
        assert np.array_equal(got[[0, 1, 2, 4]], v[[0, 0, 0, 0]])
    run.close()


def test_bias_table_matches_oracle(G, orc):
    run = GpuScene(synth.scene_uniform(10, 740))
    L = G.gs_bias_table_len(run.h)
    # first k at which both FP32 factors are exactly 1: 1/sqrt(1 - 0.999^k)
    # rounds to 1.0f once 0.999^k <= 2^-23, i.e. from k ~ 15936 on
    k = np.arange(1, 40000, dtype=np.float64)
    f1 = (1.0 / (1.0 - 0.9 ** k)).astype(np.float32)
    f2 = (1.0 / np.sqrt(1.0 - 0.999 ** k)).astype(np.float32)
    first = int(k[np.nonzero((f1 == 1.0) & (f2 == 1.0))[0][0]])
    assert abs(L - (first + 1)) <= 1
    b1 = torch.zeros(L, dtype=torch.float64, device="cuda")
    b2 = torch.zeros_like(b1)
    G.gs_bias_table(run.h, b1, b2, L)
    torch.cuda.synchronize()
    np.testing.assert_allclose(b1.cpu().numpy()[1:], orc.bias_denominators(0.9, L)[1:], rtol=1e-13)
    np.testing.assert_allclose(b2.cpu().numpy()[1:], orc.bias_denominators(0.999, L)[1:], rtol=1e-12)
    run.close()


@pytest.mark.parametrize("prec", ["FP32", "FP16_BLOCK", "FP8E4M3"])
@pytest.mark.parametrize("pinned", [True, False])
def test_step_host_equals_device_path(G, pinned, prec):
    """Pinned host gradients are read in place by the kernel, pageable ones
    are staged on the device first: both give the device path's result,
    attributes and moments, over two steps."""
    n = 20_000
    groups = synth.scene_blobs(n, 750, 12.5)
    cams = synth.ring_cameras(5)
    kw = dict(prec=getattr(G, "GS_MOM_" + prec))
    a, b = GpuScene(groups, **kw), GpuScene(groups, **kw)
    for k in (1, 2):
        grads = synth.grads_rows(n, 751, k)
        a.set_grads(grads)
        p = G.make_params(LR, k)
        a.step_camera(cams[k], p)
        gh = {g: torch.from_numpy(np.ascontiguousarray(v)) for g, v in synth.from_rows(grads).items()}
        if pinned:
            gh = {g: v.pin_memory() for g, v in gh.items()}
        nv = G.gs_step_host(b.h, G.make_attrs(b.attrs), G.make_attrs(gh), G.make_camera(cams[k]), p)
        assert nv == int(a.nvis.item())
    assert a.rows().tobytes() == b.rows().tobytes()
    for x, y in zip(a.state(), b.state()):
        assert x.tobytes() == y.tobytes()
    a.close()
    b.close()


# ---------------------------------------------------------- argument checks

def test_invalid_arguments_are_rejected(G):
    n = 1000
    groups = synth.scene_uniform(n, 760)
    run = GpuScene(groups)
    A, Gr = G.make_attrs(run.attrs), G.make_attrs(run.grads)
    cam = G.make_camera(synth.ring_cameras(4)[0])
    ok = G.make_params(LR, 1)
    with pytest.raises(G.GsError):                             # iteration 0
        G.gs_step_camera(run.h, A, Gr, cam, G.make_params(LR, 0))
    with pytest.raises(G.GsError):                             # ratio out of range
        G.gs_step_camera(run.h, A, Gr, cam, G.make_params(LR, 1, restate=True, restate_ratio=1.5))
    host = {k: torch.from_numpy(v) for k, v in groups.items()}
    with pytest.raises(G.GsError):                             # host memory as device attrs
        G.gs_step_camera(run.h, G.make_attrs(host), Gr, cam, ok)
    mis = dict(run.attrs)
    buf = torch.zeros(n * 48 + 1, dtype=torch.float32, device="cuda")
    mis["sh"] = buf[1:].view(n, 48)                              # 4-byte misaligned
    with pytest.raises(G.GsError):
        G.gs_step_camera(run.h, G.make_attrs(mis), Gr, cam, ok)
    bad_cam = synth.ring_cameras(4)[0].copy()
    bad_cam[3] = np.nan
    with pytest.raises(G.GsError):
        G.gs_step_camera(run.h, A, Gr, G.make_camera(bad_cam), ok)
    G.gs_step_camera(run.h, A, Gr, cam, ok)                      # the valid call still works
    torch.cuda.synchronize()
    run.close()
