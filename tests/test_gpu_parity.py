"""GPU path (through the C ABI) against the FP64 CPU oracle.

Images: max-abs <= 2e-4 per channel on every pixel the oracle does not flag
(a flagged pixel has a discrete decision within rounding distance of its
threshold, where FP32 may legitimately decide the other way; flagged pixels
must stay rare).  Gradients: element by element, |g_gpu - g_oracle| <=
1e-3 |g_oracle| + eps_k, where eps_k = 1e-3 times the 99th percentile of
|g_oracle| over the entries of parameter group k (the FP32 rounding of a sum
of per-pixel terms scales with the group's large entries, not with the
entry's own, possibly cancelled, value); dL/dimage is zero on flagged pixels
so that both sides differentiate the same piecewise-smooth function.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2310_10642_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

IMG_TOL = 2e-4
GRAD_TOL = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_10642_gb300 import native
    native.build()
    native.lib()


def gpu_forward(G, views, opts=None, shs_dtype=None, capacity=None):
    from paper_2310_10642_gb300 import render as R
    p = R.params_to_device(G, shs_dtype=shs_dtype or torch.float32)
    fr = R.Frame(G["logit"].shape[0], views, opts, pair_capacity=capacity)
    fr.forward(p)
    torch.cuda.synchronize()
    imgs = [x.double().cpu().numpy() for x in fr.split(fr.image)]
    Ts = [x.double().cpu().numpy() for x in fr.split(fr.final_T, 1)]
    return fr, p, imgs, Ts


def assert_image_parity(img, Tg, ref, tol=IMG_TOL, max_flag_frac=0.05):
    """Every pixel within tol of the oracle, plus the oracle's ambiguity bound
    where a discrete decision lies within rounding distance of its threshold
    (a depth near-tie, an alpha at alpha_min, a stop at T_min, a borderline
    cull): there single precision may validly take the other branch, and the
    bound says how far that can move the pixel and T.  Most pixels must carry
    no such slack, so that the check is not vacuous."""
    slack = ref["amb_image"] > tol
    assert slack.mean() <= max_flag_frac, f"too many ambiguous pixels: {slack.mean():.4f}"
    err = np.abs(img - ref["image"])
    excess = err - (tol + 1.001 * ref["amb_image"])[None]
    assert excess.max() <= 0.0, f"image beyond tolerance + ambiguity bound by {excess.max():.3e}"
    excessT = np.abs(Tg - ref["T"]) - (tol + 1.001 * ref["amb_T"])
    assert excessT.max() <= 0.0, f"T beyond tolerance + ambiguity bound by {excessT.max():.3e}"
    e = err.max(axis=0)
    return dict(max_abs=float(e.max()), max_abs_unambiguous=float(e[~slack].max()) if (~slack).any() else 0.0,
                ambiguous_frac=float(slack.mean()))


# ---------------------------------------------------------------------------- forward
TILES = pytest.mark.parametrize("tile", [16, 32])
# (compositing tile, binning tile): every binning factor the library accepts
TILE_BINS = pytest.mark.parametrize("tile,bin", [(16, 16), (16, 32), (16, 64), (32, 32), (32, 64)])


@TILE_BINS
def test_forward_config0_full_frame(tile, bin):
    c = I.config(0)
    G, views = c["gaussians"], c["views"]
    fr, _, imgs, Ts = gpu_forward(G, views, dict(tile_size=tile, bin_size=bin))
    ref = O.render(G, views[0])
    assert fr.last_counters.n_visible == ref["n_visible"]
    assert_image_parity(imgs[0], Ts[0], ref)
    assert ref["image"].max() > 0.1  # not a blank scene


def ragged_scene(n=3000, seed=11, L=3, K=2):
    G = I.gaussians(n, seed, L, K)
    views = [I.view((0.3, 0.2, 4.0), 77, 53, 0.31, bg=(0.1, 0.3, 0.2)),
             I.view((-2.0, 1.0, 3.3), 40, 96, 0.55),
             I.view((1.5, -0.5, -3.6), 130, 31, 0.8, bg=(1.0, 1.0, 1.0))]
    return G, views


@TILE_BINS
def test_forward_ragged_multiview(tile, bin):
    G, views = ragged_scene()
    _, _, imgs, Ts = gpu_forward(G, views, dict(tile_size=tile, bin_size=bin))
    for v, img, T in zip(views, imgs, Ts):
        ref = O.render(G, v)
        st = assert_image_parity(img, T, ref)
        print(f"[parity] fp32 tile {tile} bin {bin} {v['width']}x{v['height']}: {st}")


def test_forward_bf16_coefficients_are_exact_inputs():
    """BF16 4DSH storage: the oracle on the same (rounded) coefficients matches to FP32 tolerance."""
    G, views = ragged_scene(n=1500, seed=12)
    shs16 = torch.as_tensor(G["shs"]).to(torch.bfloat16)
    G16 = dict(G, shs=shs16.float().numpy())
    _, _, imgs, Ts = gpu_forward(dict(G, shs=shs16), views, shs_dtype=torch.bfloat16)
    for v, img, T in zip(views, imgs, Ts):
        assert_image_parity(img, T, O.render(G16, v))


def read_state(fr):
    """Records, tile counts, ranges and the sorted lists, via fgs4d_state_layout."""
    info = fr.layout()
    st = fr.state
    S = int(info.n_splats)
    rb = int(info.record_bytes)
    rec = st[info.records: info.records + S * rb].view(torch.float32).view(S, rb // 4).cpu().numpy()
    tiles = st[info.tiles_touched: info.tiles_touched + 4 * S].view(torch.int32).cpu().numpy()
    nt = int(info.total_tiles)
    ranges = st[info.ranges: info.ranges + 8 * nt].view(torch.int32).view(nt, 2).cpu().numpy()
    npairs = int(fr.last_counters.n_pairs)
    vals = st[info.pair_vals: info.pair_vals + 4 * npairs].view(torch.int32).cpu().numpy()
    return rec, tiles, ranges, vals


def test_slice_project_records_match_oracle():
    G, views = ragged_scene(n=2500, seed=13)
    fr, _, _, _ = gpu_forward(G, views)
    rec, tiles, _, _ = read_state(fr)
    n = G["logit"].shape[0]
    for vi, v in enumerate(views):
        ref = O.project_all(G, v)
        vis_g = tiles[vi * n:(vi + 1) * n] > 0
        vis_o = ref["visible"] == 1
        border = ref["borderline"] == 1
        # GPU-visible but oracle-culled only for borderline decisions
        assert np.all(border[vis_g & ~vis_o])
        # oracle-visible but GPU-culled: borderline, or the support box (the bounding box
        # of alpha_eff G >= alpha_min) misses the image
        k2 = 2.0 * np.log(np.maximum(ref["alpha_eff"] * 255.0, 1.0))
        hx = np.sqrt(k2 * ref["cov2d"][:, 0]) if n else np.zeros(0)
        hy = np.sqrt(k2 * ref["cov2d"][:, 2]) if n else np.zeros(0)
        miss = ((ref["u"] + hx < -0.4) | (ref["u"] - hx > v["width"] - 0.6) |
                (ref["v"] + hy < -0.4) | (ref["v"] - hy > v["height"] - 0.6))
        # or its support ellipse reaches no pixel centre (binning keeps no tile for it)
        for g in np.nonzero(vis_o & ~vis_g & ~border & ~miss)[0]:
            x0, x1 = max(math.ceil(ref["u"][g] - hx[g]), 0), min(math.floor(ref["u"][g] + hx[g]), v["width"] - 1)
            y0, y1 = max(math.ceil(ref["v"][g] - hy[g]), 0), min(math.floor(ref["v"][g] + hy[g]), v["height"] - 1)
            xs, ys = np.meshgrid(np.arange(x0, x1 + 1) - ref["u"][g], np.arange(y0, y1 + 1) - ref["v"][g])
            a, b, c = ref["conic"][g]
            alpha = ref["alpha_eff"][g] * np.exp(-0.5 * (a * xs * xs + c * ys * ys) - b * xs * ys)
            assert alpha.size == 0 or alpha.max() < 1.0 / 255.0 * 1.001, g
        both = vis_g & vis_o
        assert both.sum() > 50
        r = rec[vi * n:(vi + 1) * n][both]
        def close(a, b, rtol, atol, what):
            err = np.abs(a - b) / (np.abs(b) * rtol + atol)
            assert err.max() <= 1.0, f"{what}: worst {err.max():.3g}"
        close(r[:, 0], ref["u"][both], 1e-5, 1e-3, "u")
        close(r[:, 1], ref["v"][both], 1e-5, 1e-3, "v")
        conic = ref["conic"][both]
        scale = np.abs(conic).max(axis=1)
        for k, col in enumerate((2, 3, 4)):
            close(r[:, col], conic[:, k], 1e-4, 1e-4 * scale, f"conic{k}")
        close(r[:, 5], ref["alpha_eff"][both], 1e-5, 1e-7, "alpha_eff")
        col = ref["color"][both]
        for ch, c in enumerate((6, 7, 8)):
            close(r[:, c], col[:, ch], 1e-5, 1e-5, f"color{ch}")
        close(r[:, 9], ref["depth"][both], 1e-6, 1e-6, "depth")


def large_splat_scene():
    """Splats from a few pixels to most of a 320x240 view: at 16-pixel bins
    some 32 consecutive splats own more pairs than the scatter's staging
    buffer holds."""
    G = I.gaussians(400, 31, 3, 2, log_s_xyz=(-2.0, 1.0))
    views = [I.view((0.2, 0.1, 4.0), 320, 240, 0.4), I.view((-1.5, 0.5, 3.5), 200, 150, 0.6)]
    return G, views


def check_tile_lists(G, views, fr, tile):
    """Every splat is listed in the binning tiles (tile x tile pixels) its
    support ellipse reaches (R7 with slack): within its support box, once
    per tile, as many tiles as the binning counted, and in every tile holding
    a pixel where the record's own alpha (in FP64) clears alpha_min; each
    tile's list is in (depth, index) order.  Returns (listed pairs, box
    tiles)."""
    rec, tiles, ranges, vals = read_state(fr)
    n = G["logit"].shape[0]
    amin = 1.0 / 255.0
    listed = {}
    for t in range(ranges.shape[0]):
        s, e = ranges[t]
        got = list(vals[s:e]) if e > s else []
        assert got == sorted(got, key=lambda sid: (rec[sid, 9], sid)), f"tile {t} out of depth order"
        for sid in got:
            listed.setdefault(int(sid), []).append(t)
    tile_base = 0
    box_total = listed_total = 0
    for vi, v in enumerate(views):
        tx_n = (v["width"] + tile - 1) // tile
        for g in np.nonzero(tiles[vi * n:(vi + 1) * n])[0]:
            sid = vi * n + g
            u, vv, a, b, c, ae, hx, hy = (float(rec[sid, k]) for k in (0, 1, 2, 3, 4, 5, 10, 11))
            px0, px1 = max(math.ceil(u - hx), 0), min(math.floor(u + hx), v["width"] - 1)
            py0, py1 = max(math.ceil(vv - hy), 0), min(math.floor(vv + hy), v["height"] - 1)
            box = {tile_base + ty * tx_n + tx for ty in range(py0 // tile, py1 // tile + 1)
                   for tx in range(px0 // tile, px1 // tile + 1)}
            got = listed.get(sid, [])
            assert len(got) == len(set(got)) == tiles[sid] and set(got) <= box, sid
            xs, ys = np.meshgrid(np.arange(px0, px1 + 1), np.arange(py0, py1 + 1))
            dx, dy = xs - u, ys - vv
            alpha = ae * np.exp(-0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy)
            need = {tile_base + (y // tile) * tx_n + (x // tile)
                    for x, y in zip(xs[alpha >= amin * 1.001], ys[alpha >= amin * 1.001])}
            assert need <= set(got), sid
            box_total += len(box)
            listed_total += len(got)
        tile_base += tx_n * ((v["height"] + tile - 1) // tile)
    assert tile_base == ranges.shape[0]
    assert sum(len(x) for x in listed.values()) == int(fr.last_counters.n_pairs)
    return listed_total, box_total


def huge_splat_scene():
    """A 720x560 view (1575 binning tiles of 16 pixels) with a few splats
    whose support ellipse reaches more than 1024 of them."""
    G = I.gaussians(150, 33, 3, 2, log_s_xyz=(-2.0, 0.8))
    return G, [I.view((0.0, 0.2, 3.0), 720, 560, 0.5)]


@TILE_BINS
@pytest.mark.parametrize("scene", ["ragged", "large", "huge"])
def test_tile_lists_are_depth_ordered_and_complete(tile, bin, scene):
    """The lists of check_tile_lists, per binning tile (bin x bin pixels)
    whatever the compositing tile.  The scenes take every way through the
    pair scatter (a warp stages the pairs of 32 consecutive splats in a
    1024-entry buffer): rounds whose pairs fit the buffer (ragged), rounds
    that go through it in runs of lanes (large splats at 16-pixel bins), and
    single splats with more pairs than it holds, walked alone (huge, at
    16-pixel bins)."""
    G, views = {"ragged": lambda: ragged_scene(n=2500, seed=14), "large": large_splat_scene,
                "huge": huge_splat_scene}[scene]()
    fr, _, _, _ = gpu_forward(G, views, dict(tile_size=tile, bin_size=bin))
    # rounds of the scatter: 32 consecutive splats of a view's (depth, index) ordered run (the
    # few visible splats whose ellipse reaches no tile hold no pairs and are left out here)
    rec, tiles, _, _ = read_state(fr)
    n = G["logit"].shape[0]
    rounds = []
    for vi in range(len(views)):
        vis = [vi * n + g for g in np.nonzero(tiles[vi * n:(vi + 1) * n])[0]]
        run = [int(tiles[sid]) for sid in sorted(vis, key=lambda sid: (rec[sid, 9], sid))]
        rounds += [sum(run[k:k + 32]) for k in range(0, len(run), 32)]
    if scene == "ragged":
        assert min(rounds) <= 1024  # a round whose pairs fit the warp's staging buffer
    if scene == "large" and bin == 16:
        assert max(rounds) > 1024  # and one whose pairs do not
    if scene == "huge" and bin == 16:
        assert tiles.max() > 1024  # a splat with more pairs than the buffer
    listed_total, box_total = check_tile_lists(G, views, fr, bin)
    print(f"[bin] bin {bin}: {listed_total} pairs vs {box_total} box tiles ({listed_total / box_total:.3f})")
    assert listed_total < box_total  # the ellipse drops tiles the box would keep


@pytest.mark.parametrize("n", [768, 769])
@pytest.mark.parametrize("tile,bin", [(16, 16), (32, 64)])
def test_binning_chunks_at_view_edges(n, tile, bin):
    """The counting path cuts each view's depth-ordered run of visible splats
    into chunks of 256.  Here every Gaussian is visible in the first and the
    last view (n = 768: three full chunks; 769: a fourth chunk of one
    splat) and none in the middle view, which looks away (no chunk at all:
    its tiles' lists are empty).  Lists as check_tile_lists, images and T
    against the oracle."""
    G = I.gaussians(n, 47, 2, 1, log_s_xyz=(-3.5, 0.4))
    t = 0.4
    G["mu"][3] = t  # centred in time: p(t) = 1, no splat fails the temporal filter
    views = [I.view((0.3, 0.2, 4.0), 160, 120, t, fov_x_deg=60.0),
             I.view((0.0, 0.0, 4.0), 96, 64, t, target=(0.0, 0.0, 8.0), bg=(0.3, 0.5, 0.7)),
             I.view((-3.5, 0.5, 1.5), 130, 100, t, fov_x_deg=60.0, bg=(1.0, 1.0, 1.0))]
    fr, _, imgs, Ts = gpu_forward(G, views, dict(tile_size=tile, bin_size=bin))
    per_view = [O.render(G, v) for v in views]
    assert [r["n_visible"] for r in per_view] == [n, 0, n]
    assert fr.last_counters.n_visible == 2 * n
    check_tile_lists(G, views, fr, bin)
    for img, T, ref in zip(imgs, Ts, per_view):
        assert_image_parity(img, T, ref)
    assert np.allclose(imgs[1], np.array([0.3, 0.5, 0.7])[:, None, None]) and np.all(Ts[1] == 1.0)


def test_views_over_4096_tiles_take_the_radix_path():
    """A view with more than 4096 binning tiles (1600 x 1400 pixels at
    16-pixel bins: 100 x 88) is binned by a radix sort of the pairs on their
    tile id instead of the counting sort (the state then holds keys and
    values, double-buffered: 16 bytes per pair instead of 4).  Its lists pass
    the same checks, and its image and T equal, bit for bit, those of
    32-pixel bins, which take the counting path."""
    from paper_2310_10642_gb300 import native as N
    G = I.gaussians(6000, 43, 3, 2, log_s_xyz=(-2.5, 0.8))
    views = [I.view((0.2, 0.3, 3.6), 1600, 1400, 0.45), I.view((-1.0, 0.4, 3.0), 90, 70, 0.2)]
    out = {}
    for b in (16, 32):
        opts = dict(tile_size=16, bin_size=b)
        fr, _, imgs, Ts = gpu_forward(G, views, opts)
        per_pair = (N.fgs4d_state_size(6000, fr.c_views, 2, 1000, fr.c_opts) -
                    N.fgs4d_state_size(6000, fr.c_views, 2, 0, fr.c_opts)) / 1000
        assert per_pair >= (16 if b == 16 else 4) and per_pair < (17 if b == 16 else 5), per_pair
        assert fr.counters().status == 0 and fr.last_counters.n_pairs > 10000
        check_tile_lists(G, views, fr, b)
        out[b] = (imgs, Ts)
    for k in range(2):
        np.testing.assert_array_equal(out[16][0][k], out[32][0][k])
        np.testing.assert_array_equal(out[16][1][k], out[32][1][k])
    assert out[16][0][0].max() > 0.1  # not a blank frame


@TILE_BINS
def test_batched_equals_one_by_one(tile, bin):
    G, views = ragged_scene(n=2000, seed=15)
    _, _, imgs, Ts = gpu_forward(G, views, dict(tile_size=tile, bin_size=bin))
    for v, img, T in zip(views, imgs, Ts):
        _, _, im1, T1 = gpu_forward(G, [v], dict(tile_size=tile, bin_size=bin))
        np.testing.assert_array_equal(img, im1[0])
        np.testing.assert_array_equal(T, T1[0])


@pytest.mark.parametrize("mixed", [False, True])
def test_cuda_graph_batch_of_uneven_views(mixed):
    """The batched workload's shape at reduced size (4 timestamps x 20 arc
    cameras at one size plus 20 views at half size, 100 views): one whole
    forward+backward step captured as a CUDA graph.  Replays after the
    parameters are overwritten in place equal eager launches on the new
    parameters (images and T bit for bit, gradients up to the order of FP32
    atomic sums), and the batch equals its views rendered one by one."""
    from paper_2310_10642_gb300 import render as R
    c = I.config(2, n=20000, scale=0.15)
    G, views = c["gaussians"], c["views"]
    assert len(views) == 100 and len({(v["width"], v["height"]) for v in views}) == 2
    opts = dict(c["options"], tile_size=32, record_fp16=int(mixed))
    sd = torch.bfloat16 if mixed else torch.float32
    p = R.params_to_device(G, shs_dtype=sd)
    fr = R.Frame(G["logit"].shape[0], views, opts)
    fr.forward(p)
    fr._alloc(int(fr.last_counters.n_pairs * 1.5) + 4096)
    dL = torch.randn(3 * fr.total_pixels, device="cuda", generator=torch.Generator(device="cuda").manual_seed(5))
    grads = {k: torch.empty(p[k].shape, device="cuda") for k in R.PARAM_KEYS}

    def step():
        fr.slice_project(p)
        fr.bin_sort()
        fr.render()
        fr.backward(p, dL, grads)

    step()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    G2 = I.gaussians(G["logit"].shape[0], 777, G["sh_degree"], G["n_freq"])
    G2["period"] = G["period"]
    p2 = R.params_to_device(G2, shs_dtype=sd)
    for k in R.PARAM_KEYS:
        p[k].copy_(p2[k])
    g.replay()
    torch.cuda.synchronize()
    assert fr.counters().status == 0
    img_g, T_g = fr.image.clone(), fr.final_T.clone()
    grad_g = {k: v.clone() for k, v in grads.items()}
    step()
    torch.cuda.synchronize()
    assert torch.equal(img_g, fr.image) and torch.equal(T_g, fr.final_T)
    for k in R.PARAM_KEYS:
        rel = float((grad_g[k] - grads[k]).norm() / grads[k].norm())
        assert rel < 1e-5, (k, rel)
    imgs, Ts = fr.split(img_g), fr.split(T_g, 1)
    for i in (0, 37, 79, 80, 99):
        f1 = R.Frame(G["logit"].shape[0], [views[i]], opts)
        f1.forward(p)
        assert torch.equal(f1.image.view_as(imgs[i]), imgs[i]) and torch.equal(f1.final_T.view_as(Ts[i]), Ts[i])


@pytest.mark.parametrize("groups,mixed", [(2, True), (3, False)])
def test_split_frame_equals_one_batch(groups, mixed):
    """SplitFrame: the views as contiguous groups on their own streams, the
    projection adjoints chained into one set of gradients (the first group
    overwrites, the others accumulate).  Images, T and n_last equal those of
    one Frame over all views bit for bit; gradients equal its gradients up to
    the order of FP32 sums; an eager step and a replay of the captured step
    agree likewise."""
    from paper_2310_10642_gb300 import render as R
    c = I.config(2, n=20000, scale=0.1)
    G, views = c["gaussians"], c["views"][:12]
    opts = dict(c["options"], tile_size=32, bin_size=64, record_fp16=int(mixed))
    p = R.params_to_device(G, shs_dtype=torch.bfloat16 if mixed else torch.float32)
    n = G["logit"].shape[0]
    fr = R.Frame(n, views, opts)
    fr.forward(p)
    dL = torch.randn(3 * fr.total_pixels, device="cuda", generator=torch.Generator(device="cuda").manual_seed(9))
    ref = {k: v.clone() for k, v in fr.backward(p, dL).items()}
    sf = R.SplitFrame(n, views, opts, groups=groups)
    assert sf.groups == groups and sf.total_pixels == fr.total_pixels
    sf.forward(p, check=True)
    grads = {k: torch.full(p[k].shape, float("nan"), device="cuda") for k in R.PARAM_KEYS}
    sf.step(p, dL, grads)
    torch.cuda.synchronize()
    assert torch.equal(sf.image, fr.image) and torch.equal(sf.final_T, fr.final_T)
    assert torch.equal(sf.n_last, fr.n_last)

    def close(got, want, what):  # FP32 sums in another order: 1e-4, a tenth of the oracle bar
        for k in R.PARAM_KEYS:
            assert_elementwise(got[k].double().cpu().numpy(), want[k].double().cpu().numpy(), 1e-4,
                               f"{what} {k}", floor=1e-4 * grad_floor(want[k].double().cpu().numpy(), 1.0))
    close(grads, ref, f"split x{groups}")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        sf.step(p, dL, grads)
    for k in grads:
        grads[k].fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(sf.image, fr.image)
    close(grads, ref, f"split x{groups} graph")
    assert all(c_.status == 0 for c_ in sf.counters())


@pytest.mark.parametrize("tile,mixed", [(16, False), (32, False), (32, True)])
def test_render_stats_count_the_walk(tile, mixed):
    """fgs4d_render_stats: same image as fgs4d_render; its blended-pair count
    equals the oracle's contributor count summed over the pixels (up to one
    per flagged pixel, whose decisions may validly differ); its walk count is
    the sum of n_last; every blended pair lies inside its splat's box."""
    G, views = ragged_scene(n=2500, seed=17)
    opts = dict(tile_size=tile, record_fp16=int(mixed))
    fr, p, imgs, _ = gpu_forward(G, views, opts, shs_dtype=torch.bfloat16 if mixed else None)
    img0, T0, last0 = fr.image.clone(), fr.final_T.clone(), fr.n_last.clone()
    st = fr.render_stats()
    torch.cuda.synchronize()
    assert torch.equal(img0, fr.image) and torch.equal(T0, fr.final_T) and torch.equal(last0, fr.n_last)
    assert st["walked"] == int(fr.n_last.sum())
    assert st["evaluated"] >= st["in_box"] >= st["blended"] > 0
    Gr = dict(G, shs=torch.as_tensor(G["shs"]).to(torch.bfloat16).float().numpy()) if mixed else G
    refs = [O.render(Gr, v) for v in views]
    want = sum(int(r["n_contrib"].sum()) for r in refs)
    slack = sum(int((r["flags"] != 0).sum()) for r in refs)
    if mixed:  # 16-bit conics move alpha by more than the FP32-sized flag margins
        slack += int(2e-3 * want)
    assert abs(st["blended"] - want) <= slack, (st["blended"], want, slack)


@TILES
def test_batch_depth_does_not_change_results(tile):
    """batch_depth only changes how many records a tile stages per batch:
    images, T and n_last are bit-identical; gradients differ only by the
    order of FP32 sums."""
    from paper_2310_10642_gb300 import render as R
    G, views = ragged_scene(n=2500, seed=19)
    p = R.params_to_device(G)
    dL = torch.randn(sum(3 * v["width"] * v["height"] for v in views), device="cuda",
                     generator=torch.Generator(device="cuda").manual_seed(3))
    out = {}
    for B in (32, 64, 128, 256):
        fr = R.Frame(G["logit"].shape[0], views, dict(tile_size=tile, batch_depth=B))
        fr.forward(p)
        g = fr.backward(p, dL)
        torch.cuda.synchronize()
        out[B] = (fr.image.clone(), fr.final_T.clone(), fr.n_last.clone(), {k: v.clone() for k, v in g.items()})
    ref = out[256]
    for B in (32, 64, 128):
        img, T, nl, g = out[B]
        assert torch.equal(img, ref[0]) and torch.equal(T, ref[1]) and torch.equal(nl, ref[2])
        for k in R.PARAM_KEYS:
            rel = float((g[k] - ref[3][k]).norm() / ref[3][k].norm())
            assert rel < 1e-5, (B, k, rel)


@TILES
def test_bin_size_does_not_change_results(tile):
    """bin_size only changes which list a compositing tile walks (its binning
    tile's, holding the splats of every compositing tile inside it): images
    and T are bit-identical, since a pixel composites the same splats in the
    same order; n_last counts positions in the larger list, so it can only
    grow; gradients differ only by the order of FP32 sums."""
    from paper_2310_10642_gb300 import render as R
    G, views = ragged_scene(n=2500, seed=21)
    p = R.params_to_device(G)
    dL = torch.randn(sum(3 * v["width"] * v["height"] for v in views), device="cuda",
                     generator=torch.Generator(device="cuda").manual_seed(4))
    out = {}
    bins = [b for b in (16, 32, 64) if b >= tile]
    for b in bins:
        fr = R.Frame(G["logit"].shape[0], views, dict(tile_size=tile, bin_size=b))
        fr.forward(p)
        g = fr.backward(p, dL)
        torch.cuda.synchronize()
        assert fr.counters().status == 0
        out[b] = (fr.image.clone(), fr.final_T.clone(), fr.n_last.clone(), {k: v.clone() for k, v in g.items()},
                  int(fr.last_counters.n_pairs))
    ref = out[tile]
    for b in bins[1:]:
        img, T, nl, g, npairs = out[b]
        assert torch.equal(img, ref[0]) and torch.equal(T, ref[1])
        assert bool((nl >= ref[2]).all())
        assert npairs < ref[4]  # coarser bins: fewer (splat, tile) pairs
        for k in R.PARAM_KEYS:
            rel = float((g[k] - ref[3][k]).norm() / ref[3][k].norm())
            assert rel < 1e-5, (b, k, rel)


def test_autotune_groups_returns_a_timed_count():
    from paper_2310_10642_gb300 import autotune as A
    from paper_2310_10642_gb300 import render as R
    G, views = ragged_scene(n=2000, seed=24)
    p = R.params_to_device(G)
    g, table = A.tune_groups(p, views, dict(tile_size=32), groups=(1, 2), reps=2, warmup=1)
    assert g in (1, 2) and [t["groups"] for t in table] == [1, 2] and all(t["ms"] > 0 for t in table)
    assert min(t["ms"] for t in table) == [t["ms"] for t in table if t["groups"] == g][0]


def test_autotune_returns_a_timed_candidate():
    from paper_2310_10642_gb300 import autotune as A
    from paper_2310_10642_gb300 import render as R
    G, views = ragged_scene(n=2000, seed=23)
    p = R.params_to_device(G)
    cands = A.candidates((16, 32), (64, 256), (1, 2))
    opts, table = A.tune(p, views, dict(record_fp16=0), cands=cands, reps=2, warmup=1, cache=None)
    pick = {k: opts[k] for k in A.KNOBS}
    assert pick in cands
    assert len(table) == 8 and all(t["ms"] > 0 for t in table)
    assert min(t["ms"] for t in table) == [t["ms"] for t in table if all(t[k] == pick[k] for k in A.KNOBS)][0]


def test_fp64_fallback_for_ill_conditioned_slices():
    """Gaussians stretched along a space-time diagonal: Sigma_{xyz|t} is a tiny
    difference of large numbers (Eq. 9); the GPU recomputes it in FP64."""
    n = 400
    r = np.random.default_rng(3)
    th = r.uniform(0.6, 1.0, size=n)  # rotation in the x-t plane
    q = np.stack([np.cos(th / 2), np.zeros(n), np.zeros(n), np.sin(th / 2)]).astype(np.float32)
    G = I.gaussians(n, 99, 1, 1)
    G["ql"], G["qr"] = q.copy(), q.copy()
    G["log_s"][0] = -1.0  # long axis (mixes x and t)
    G["log_s"][3] = -7.5  # very thin across it
    G["mu"][3] = 0.5
    views = [I.view((0.0, 0.0, 4.0), 96, 96, 0.5)]
    fr, _, imgs, Ts = gpu_forward(G, views)
    ref = O.render(G, views[0])
    assert_image_parity(imgs[0], Ts[0], ref)


# ---------------------------------------------------------------------------- edge cases
def test_edge_cases_empty_culled_tiny():
    from paper_2310_10642_gb300 import native as N
    # no Gaussians at all
    G = I.gaussians(0, 1, 1, 1)
    v = I.view((0, 0, 4), 33, 17, 0.5, bg=(0.2, 0.4, 0.6))
    fr, _, imgs, Ts = gpu_forward(G, [v])
    assert np.allclose(imgs[0], np.array([0.2, 0.4, 0.6])[:, None, None]) and np.all(Ts[0] == 1.0)
    # every Gaussian culled by the temporal filter
    G = I.gaussians(500, 2, 1, 1)
    G["mu"][3] += 50.0
    fr, _, imgs, _ = gpu_forward(G, [v])
    assert fr.last_counters.n_visible == 0 and np.allclose(imgs[0], np.array([0.2, 0.4, 0.6])[:, None, None])
    # 1x1 image, one-tile images, one-row images, for both tile sizes
    G = I.gaussians(800, 3, 2, 1)
    for tile in (16, 32):
        for w, h in ((1, 1), (16, 16), (32, 32), (17, 1), (33, 2)):
            vv = I.view((0.1, 0.2, 4.0), w, h, 0.5)
            _, _, imgs, Ts = gpu_forward(G, [vv], dict(tile_size=tile))
            assert_image_parity(imgs[0], Ts[0], O.render(G, vv), max_flag_frac=1.0)


def test_pair_capacity_overflow_is_reported_not_faulted():
    from paper_2310_10642_gb300 import native as N
    from paper_2310_10642_gb300 import render as R
    c = I.config(0)
    p = R.params_to_device(c["gaussians"])
    fr = R.Frame(2000, c["views"], pair_capacity=16)
    fr.forward(p, check=False)
    cnt = fr.counters()
    assert cnt.status & N.STATUS_PAIR_OVERFLOW and cnt.n_pairs > 16
    fr.forward(p, check=True)  # grows and re-runs
    assert not (fr.last_counters.status & N.STATUS_PAIR_OVERFLOW)


def test_nonfinite_and_zero_quaternion_are_flagged():
    from paper_2310_10642_gb300 import native as N
    G = I.gaussians(300, 4, 1, 1)
    G["mu"][0, 5] = np.nan
    G["ql"][:, 7] = 0.0
    v = I.view((0, 0, 4), 64, 64, 0.5)
    fr, _, imgs, _ = gpu_forward(G, [v])
    assert fr.last_counters.status & N.STATUS_NONFINITE
    assert np.all(np.isfinite(imgs[0]))


# ---------------------------------------------------------------------------- backward
def grads_gpu(fr, p, dL_list):
    dL = torch.cat([torch.as_tensor(d, dtype=torch.float32).reshape(-1) for d in dL_list]).cuda()
    g = fr.backward(p, dL)
    torch.cuda.synchronize()
    return {k: v.double().cpu().numpy() for k, v in g.items()}


GROUPS = ("mu", "log_s", "ql", "qr", "logit", "shs")


def grad_floor(ref, tol=GRAD_TOL):
    """eps_k of one parameter group: tol x the 99th percentile of |reference|
    over its non-zero entries."""
    mag = np.abs(np.asarray(ref, dtype=np.float64)).ravel()
    mag = mag[mag > 0]
    return tol * float(np.percentile(mag, 99)) if mag.size else 0.0


def assert_elementwise(a, b, tol, name, floor=None, allow_frac=0.0):
    """|a - b| <= tol |b| + eps element by element (eps = grad_floor(b, tol)
    unless given); returns the worst entry's ratio to its bound and the
    worst relative error among the entries above eps.  allow_frac > 0 lets
    that fraction of the entries exceed the bound (each is printed), with
    the whole group within tol in norm."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (name, a.shape, b.shape)
    assert np.all(np.isfinite(a)), f"{name}: non-finite GPU gradient"
    eps = grad_floor(b, tol) if floor is None else floor
    assert eps > 0, f"{name}: reference gradient is zero"
    err = np.abs(a - b)
    ratio = err / (tol * np.abs(b) + eps)
    i = np.unravel_index(int(np.argmax(ratio)), ratio.shape)
    big = np.abs(b) > eps
    rel_big = float((err[big] / np.abs(b[big])).max()) if big.any() else 0.0
    print(f"[parity] gradient {name}: worst entry {tuple(int(x) for x in i)} gpu {a[i]:.6e} oracle {b[i]:.6e} "
          f"(|err| / bound {ratio[i]:.3f}, eps {eps:.3e}); worst rel. error above eps {rel_big:.3e} "
          f"over {int(big.sum())} of {b.size} entries")
    if allow_frac > 0.0:
        over = np.argwhere(ratio > 1.0)
        for j in over[:20]:
            j = tuple(j)
            print(f"[parity]   {name}: entry {j} gpu {a[j]:.6e} oracle {b[j]:.6e} at {ratio[j]:.3f} x the bound")
        assert len(over) <= allow_frac * b.size, f"{name}: {len(over)} of {b.size} entries beyond the bound"
        rel = float(np.linalg.norm(a - b) / np.linalg.norm(b))
        assert rel <= tol, f"{name}: relative error {rel:.3e} in norm"
        return float(ratio[i]), rel_big
    assert ratio[i] <= 1.0, (f"{name}: entry {tuple(int(x) for x in i)} gpu {a[i]:.9e} oracle {b[i]:.9e} "
                             f"beyond {tol:g} relative + {eps:.3e}")
    return float(ratio[i]), rel_big


def assert_grad_parity(gg, go, tol=GRAD_TOL, keys=GROUPS, what=""):
    """Element-wise parity of every parameter group (see module docstring)."""
    return {k: assert_elementwise(gg[k], go[k], tol, f"{what}{k}") for k in keys}


def masked_dL(views, refs, seed):
    r = np.random.default_rng(seed)
    out = []
    for v, ref in zip(views, refs):
        d = r.normal(size=(3, v["height"], v["width"]))
        d[:, ref["flags"] != 0] = 0.0
        out.append(d)
    return out


@TILES
def test_backward_matches_oracle(tile):
    G, views = ragged_scene(n=1500, seed=21)
    fr, p, _, _ = gpu_forward(G, views, dict(tile_size=tile))
    refs = [O.render(G, v) for v in views]
    dL = masked_dL(views, refs, 5)
    gg = grads_gpu(fr, p, dL)
    go = O.backward_views(G, views, dL)
    assert_grad_parity(gg, go)


@pytest.mark.parametrize("tile,mixed", [(16, False), (32, False), (32, True)])
def test_backward_in_two_steps(tile, mixed):
    """fgs4d_render_backward_2d + fgs4d_project_backward equal
    fgs4d_render_backward, and the per-splat 2D gradients of the first step
    match the oracle's adjoint of Eq. 6 alone."""
    G, views = ragged_scene(n=1500, seed=27)
    sd = torch.bfloat16 if mixed else torch.float32
    fr, p, _, _ = gpu_forward(G, views, dict(tile_size=tile, record_fp16=int(mixed)), shs_dtype=sd)
    Gr = dict(G, shs=torch.as_tensor(G["shs"]).to(torch.bfloat16).float().numpy()) if mixed else G
    refs = [O.render(Gr, v) for v in views]
    dL = masked_dL(views, refs, 8)
    dLt = torch.cat([torch.as_tensor(d, dtype=torch.float32).reshape(-1) for d in dL]).cuda()
    g1 = {k: v.clone() for k, v in fr.backward(p, dLt).items()}
    fr.backward_2d(dLt)
    g2d = fr.grad2d().double().cpu().numpy()  # before the second step, which reuses the section
    g2 = fr.project_backward(p)
    torch.cuda.synchronize()
    for k in g1:
        rel = float((g1[k] - g2[k]).norm() / g1[k].norm())
        assert rel < 1e-5, (k, rel)
    tol = MIXED_GRAD_TOL if mixed else GRAD_TOL
    # Mixed: the 16-bit Cholesky conic moves alpha by up to |power| 2^-14 relative near alpha_min
    # (about 3e-4, beyond the oracle's FP32-sized flag margin), so a few alpha_min decisions may
    # differ at unflagged pixels; in a per-splat sum that cancels they can take an intermediate 2D
    # gradient past the element-wise bound.  At most 0.1% of these entries may, the column in norm
    # stays within 1e-2; the parameter gradients of the mixed path are checked entry by entry.
    allow = 1e-3 if mixed else 0.0
    for vi, v in enumerate(views):
        want = O.backward(Gr, v, dL[vi])["grad2d"]
        got = g2d[vi]
        for c, name in enumerate(("u", "v", "a", "b", "c", "alpha_eff", "R", "G", "B")):
            assert_elementwise(got[:, c], want[:, c], tol, f"view {vi} dL/d{name}", allow_frac=allow)


@TILES
def test_backward_config0(tile):
    c = I.config(0)
    G, views = c["gaussians"], c["views"]
    fr, p, _, _ = gpu_forward(G, views, dict(tile_size=tile))
    refs = [O.render(G, v) for v in views]
    dL = masked_dL(views, refs, 6)
    assert_grad_parity(grads_gpu(fr, p, dL), O.backward_views(G, views, dL))


def test_backward_central_differences():
    """GPU gradient vs FP64 central differences of the oracle's forward on 64
    random parameters with a non-negligible gradient, whose stencil changes no
    discrete decision (the oracle's per-pixel contributor sequences, an
    order-sensitive hash, are the same at x - h, x and x + h), element by
    element at 1e-3 relative plus the group's floor eps_k."""
    G, views = ragged_scene(n=600, seed=31, L=2, K=1)
    G["log_s"][:3] += 0.7
    views = views[:2]
    fr, p, _, _ = gpu_forward(G, views)
    refs = [O.render(G, v) for v in views]
    dL = masked_dL(views, refs, 7)
    gg = grads_gpu(fr, p, dL)
    go = O.backward_views(G, views, dL)
    floors = {k: grad_floor(go[k]) for k in GROUPS}
    G64 = {k: (np.asarray(v, dtype=np.float64) if isinstance(v, np.ndarray) else v) for k, v in G.items()}

    def loss(Gx):  # sum over views and pixels of dL * image, in FP64
        return sum(float(np.sum(d * O.render(Gx, v)["image"])) for v, d in zip(views, dL))

    rng = np.random.default_rng(8)
    checked, tried, worst = 0, 0, 0.0
    while checked < 64 and tried < 2000:
        tried += 1
        key = GROUPS[tried % len(GROUPS)]
        arr = G64[key]
        idx = tuple(int(rng.integers(0, s)) for s in arr.shape)
        if abs(gg[key][idx]) < 10 * floors[key]:
            continue  # a gradient this small only tests the floor
        x0 = float(arr[idx])
        h = 1e-6 * max(1.0, abs(x0))
        Gp = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in G64.items()}
        Gm = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in G64.items()}
        Gp[key][idx] = x0 + h
        Gm[key][idx] = x0 - h
        same = all(np.array_equal(O.render(Gx, v)["seq_hash"], ref["seq_hash"])
                   for Gx in (Gp, Gm) for v, ref in zip(views, refs))
        if not same:
            continue
        fd = (loss(Gp) - loss(Gm)) / (2.0 * h)
        an = float(gg[key][idx])
        r = abs(fd - an) / (GRAD_TOL * abs(fd) + floors[key])
        worst = max(worst, r)
        assert r <= 1.0, (key, idx, an, fd, floors[key])
        checked += 1
    print(f"[parity] central differences (FP64 oracle): {checked} parameters, worst |err| / bound {worst:.3f}")
    assert checked >= 48


def test_autograd_function_l1_loss():
    """Render4DGS through torch.autograd on an L1 loss whose per-pixel terms
    are masked where the oracle flags a decision within rounding distance of
    its threshold (both sides then differentiate the same function); the
    gradients of all raw parameters match the oracle's element by element.
    The forward does not synchronise: with the device kept busy, the call
    returns before the GPU has rendered."""
    from paper_2310_10642_gb300 import render as R
    G, views = ragged_scene(n=1200, seed=41, L=1, K=1)
    p = R.params_to_device(G)
    refs = [O.render(G, v) for v in views]
    masks = [torch.as_tensor(r["flags"] == 0, dtype=torch.float32).cuda() for r in refs]
    for r in refs:
        assert (r["flags"] != 0).mean() < 0.02
    targets = [torch.as_tensor(t).cuda() for t in I.random_target(views, 77)]

    def run():
        leaves = {k: p[k].clone().requires_grad_(True) for k in R.PARAM_KEYS}
        params = dict(leaves, sh_degree=p["sh_degree"], n_freq=p["n_freq"], period=p["period"])
        imgs, fr = R.render(params, views, frame=frame)
        return leaves, imgs, fr

    frame = R.Frame(G["logit"].shape[0], views)
    run()  # the first call sizes the pair capacity (one synchronisation)
    torch.cuda.synchronize()
    torch.cuda._sleep(200_000_000)  # keeps the stream busy for ~0.1 s
    leaves, imgs, fr = run()
    assert not torch.cuda.current_stream().query(), "the differentiable forward synchronised"
    loss = sum(((im - t).abs() * m).mean() for im, t, m in zip(imgs, targets, masks))
    loss.backward()
    assert fr.status().status == 0
    dL = [np.sign(im.detach().cpu().numpy() - t.cpu().numpy()) * m.cpu().numpy() / im.numel()
          for im, t, m in zip(imgs, targets, masks)]
    go = O.backward_views(G, views, dL)
    gg = {k: leaves[k].grad.double().cpu().numpy() for k in R.PARAM_KEYS}
    assert_grad_parity(gg, go, what="autograd ")


# ---------------------------------------------------------------------------- mixed precision
MIXED_IMG_TOL = 2e-3
MIXED_GRAD_TOL = 1e-2


@TILES
def test_mixed_precision_against_fp64_oracle(tile):
    """BF16 4DSH coefficients + 16-bit block-exponent Cholesky conics in the
    splat records, FP32 compositing.  Against the oracle fed the same
    BF16-rounded coefficients the images stay within 1e-3 (the conics' share);
    against the original FP32 inputs within 3e-3 on this scene, where the BF16
    rounding of the coefficients alone moves the oracle's own image by up to
    1.4e-3.  (The 2e-3 bar on the benchmarked workload is
    test_full_size_workload_crops.)  The path evaluates the renderer at the
    BF16-rounded coefficients, so its gradient is compared with the oracle's
    gradient there: at the FP32 coefficients the colour clamp max(c + 1/2, 0)
    switches for colours within BF16 rounding of zero."""
    G, views = ragged_scene(n=2500, seed=51)
    opts = dict(tile_size=tile, record_fp16=1)
    fr, p, imgs, Ts = gpu_forward(G, views, opts, shs_dtype=torch.bfloat16)
    G16 = dict(G, shs=torch.as_tensor(G["shs"]).to(torch.bfloat16).float().numpy())
    for img, T, v in zip(imgs, Ts, views):
        st = assert_image_parity(img, T, O.render(G16, v), tol=1e-3)
        print(f"[parity] mixed tile {tile} vs oracle(BF16 coefficients): {st}")
    refs = [O.render(G, v) for v in views]
    for img, T, ref in zip(imgs, Ts, refs):
        st = assert_image_parity(img, T, ref, tol=3e-3)
        print(f"[parity] mixed tile {tile} vs oracle(FP32 coefficients): {st}")
    refs16 = [O.render(G16, v) for v in views]
    dL = masked_dL(views, refs16, 9)
    gg = grads_gpu(fr, p, dL)
    go = O.backward_views(G16, views, dL)
    assert_grad_parity(gg, go, MIXED_GRAD_TOL, what=f"mixed tile {tile} ")


# ---------------------------------------------------------------------------- full size
@pytest.mark.parametrize("mixed", [False, True])
def test_full_size_workload_crops(mixed):
    """The benchmarked workload itself (1M clustered Gaussians, 20 views at
    1352x1014, 32x32 tiles, one launch per stage): 64x64 centre crops of three
    views against the oracle, and the gradient of a loss on the crops."""
    c = I.config(3)
    G, views = c["gaussians"], c["views"]
    opts = dict(c["options"], tile_size=32, record_fp16=int(mixed))
    fr, p, imgs, Ts = gpu_forward(G, views, opts, shs_dtype=torch.bfloat16 if mixed else torch.float32)
    tol = MIXED_IMG_TOL if mixed else IMG_TOL
    crop = 64
    picks = [0, 9, 19]
    dL = [np.zeros((3, v["height"], v["width"])) for v in views]
    rng = np.random.default_rng(13)
    for vi in picks:
        v = views[vi]
        x0, y0 = v["width"] // 2 - crop // 2, v["height"] // 2 - crop // 2
        ref = O.render(G, v, window=(x0, y0, crop, crop), prefilter=True)
        sub = imgs[vi][:, y0:y0 + crop, x0:x0 + crop]
        subT = Ts[vi][y0:y0 + crop, x0:x0 + crop]
        # dense clustered scene: thousands of splats per pixel, so more decisions sit near thresholds
        # (measured on GB300: 5.7-6.7% of the crops' pixels carry slack beyond 2e-4, 0.1-0.6% beyond 2e-3)
        st = assert_image_parity(sub, subT, ref, tol=tol, max_flag_frac=0.08)
        print(f"[parity] full-size {'mixed' if mixed else 'fp32'} view {vi} 64x64 crop: {st}")
        w = rng.normal(size=(3, crop, crop))
        w[:, ref["flags"] != 0] = 0.0
        dL[vi][:, y0:y0 + crop, x0:x0 + crop] = w
    gg = grads_gpu(fr, p, dL)
    # the mixed path differentiates the renderer at the BF16-rounded coefficients
    Gref = dict(G, shs=torch.as_tensor(G["shs"]).to(torch.bfloat16).float().numpy()) if mixed else G
    go = None
    for vi in picks[:2]:
        v = views[vi]
        x0, y0 = v["width"] // 2 - crop // 2, v["height"] // 2 - crop // 2
        gv = O.backward(Gref, v, dL[vi][:, y0:y0 + crop, x0:x0 + crop], window=(x0, y0, crop, crop), prefilter=True)
        gv.pop("grad2d")
        go = gv if go is None else {k: go[k] + gv[k] for k in go}
    # the GPU gradient above also holds the third view's crop: recompute without it
    dL[picks[2]][:] = 0.0
    gg = grads_gpu(fr, p, dL)
    gtol = MIXED_GRAD_TOL if mixed else GRAD_TOL
    assert_grad_parity(gg, go, gtol, what=f"full-size {'mixed' if mixed else 'fp32'} ")


# ---------------------------------------------------------------------------- densification (Sec. 3.4)
def test_densification_statistics_match_oracle():
    """mean2d_abs = sum over views of |dL/dmu_2d|, mu_t_abs = sum over views of
    |dL/dmu_t|, each view's gradient taken on its own (the oracle's per-view
    adjoint)."""
    G, views = ragged_scene(n=1500, seed=31)
    fr, p, _, _ = gpu_forward(G, views)
    refs = [O.render(G, v) for v in views]
    dL = masked_dL(views, refs, 12)
    dLt = torch.cat([torch.as_tensor(d, dtype=torch.float32).reshape(-1) for d in dL]).cuda()
    g = fr.backward(p, dLt, mean2d=True)
    torch.cuda.synchronize()
    m2d_want = np.zeros(G["logit"].shape[0])
    mt_want = np.zeros(G["logit"].shape[0])
    for v, d in zip(views, dL):
        o = O.backward(G, v, d)
        m2d_want += np.hypot(o["grad2d"][:, 0], o["grad2d"][:, 1])
        mt_want += np.abs(o["mu"][3])
    for key, want in (("mean2d_abs", m2d_want), ("mu_t_abs", mt_want)):
        assert_elementwise(g[key].double().cpu().numpy(), want, GRAD_TOL, key)


def test_split_sampler_draws_from_the_4d_density():
    from paper_2310_10642_gb300 import native as N
    from paper_2310_10642_gb300 import render as R
    G = I.gaussians(500, 33, 1, 1)
    p = R.params_to_device(G)
    r = np.random.default_rng(4)
    m = 777
    idx = r.integers(0, 500, size=m).astype(np.int64)
    idx[5] = idx[6]  # repeated Gaussians are independent samples
    idx[-1] = 10_000  # out of range: NaN, no access
    z = r.normal(size=(4, m)).astype(np.float32)
    idx_d, z_d = torch.as_tensor(idx).cuda(), torch.as_tensor(z).cuda()
    out = torch.empty(4, m, device="cuda")
    N.fgs4d_sample_split(R.gaussians_struct(p), idx_d.data_ptr(), z_d.data_ptr(), m, out.data_ptr(),
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = out.double().cpu().numpy()
    for j in range(m - 1):
        gi = idx[j]
        Rm = O.rotation4(G["ql"][:, gi], G["qr"][:, gi])
        want = G["mu"][:, gi] + Rm @ (np.exp(G["log_s"][:, gi].astype(np.float64)) * z[:, j])
        assert np.abs(got[:, j] - want).max() < 2e-5 * (1 + np.abs(want).max()), j
    assert np.all(np.isnan(got[:, -1]))


# ---------------------------------------------------------------------------- No-4DRot variant
def _conj(q):
    return q * np.array([1.0, -1.0, -1.0, -1.0])


def _hamilton(p, q):
    a1, b1, c1, d1 = p
    a2, b2, c2, d2 = q
    return np.array([a1 * a2 - b1 * b2 - c1 * c2 - d1 * d2, a1 * b2 + b1 * a2 + c1 * d2 - d1 * c2,
                     a1 * c2 - b1 * d2 + c1 * a2 + d1 * b2, a1 * d2 + b1 * c2 - c1 * b2 + d1 * a2])


def _r3(q):
    w, x, y, z = q / np.linalg.norm(q)
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def _quat_of(R):
    """Unit quaternion (w, x, y, z) whose usual rotation matrix is R."""
    tr = np.trace(R)
    if tr > 0:
        s = 2 * np.sqrt(tr + 1)
        q = [s / 4, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    elif R[0, 0] > R[1, 1] and R[0, 0] > R[2, 2]:
        s = 2 * np.sqrt(1 + R[0, 0] - R[1, 1] - R[2, 2])
        q = [(R[2, 1] - R[1, 2]) / s, s / 4, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s]
    elif R[1, 1] > R[2, 2]:
        s = 2 * np.sqrt(1 + R[1, 1] - R[0, 0] - R[2, 2])
        q = [(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, s / 4, (R[1, 2] + R[2, 1]) / s]
    else:
        s = 2 * np.sqrt(1 + R[2, 2] - R[0, 0] - R[1, 1])
        q = [(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, s / 4]
    return np.array(q)


def _pair_for(M):
    """(q_l, q_r) with q_l x q_r = M x for quaternions x (Eq. 8's reading)."""
    e0 = M[:, 0]
    Ra = np.stack([_hamilton(M[:, k], _conj(e0))[1:] for k in (1, 2, 3)], axis=1)
    a = _quat_of(Ra)
    return a, _hamilton(_conj(a), e0)


def test_no_4drot_variant_against_oracle():
    """FGS4D_ROT_SPATIAL: q_left rotates x, y, z; the oracle renders the same
    Gaussians through Eq. 8 with the quaternion pair that gives
    blockdiag(R3(q), 1).  Images and the gradients of every parameter but
    q_left match the oracle; dL/dq_left matches FP64 central differences of
    the oracle through that pair; dL/dq_right is zero; the splats do not move
    with t."""
    from paper_2310_10642_gb300 import native as N
    from paper_2310_10642_gb300 import render as R
    G, views = ragged_scene(n=500, seed=43)
    n = G["logit"].shape[0]
    q3 = G["ql"].astype(np.float64)

    def oracle_params(q):
        pairs = []
        for g in range(n):
            M = np.eye(4)
            M[:3, :3] = _r3(q[:, g])
            a, b = _pair_for(M)
            if g < 5:  # the pair reproduces the block-diagonal rotation under the oracle's Eq. 8
                assert np.abs(O.rotation4(a, b) - M).max() < 1e-12
            pairs.append((a, b))
        return dict(G, ql=np.stack([a for a, _ in pairs], 1), qr=np.stack([b for _, b in pairs], 1))

    Go = oracle_params(q3)
    Gs = dict(G, rotation=N.ROT_SPATIAL, qr=np.full_like(G["qr"], np.nan))  # q_right must not be read
    fr, p, imgs, Ts = gpu_forward(Gs, views, dict(tile_size=32))
    refs = [O.render(Go, v) for v in views]
    for img, T, ref in zip(imgs, Ts, refs):
        assert_image_parity(img, T, ref)
    dL = masked_dL(views, refs, 14)
    gg = grads_gpu(fr, p, dL)
    go = O.backward_views(Go, views, dL)
    assert_grad_parity(gg, go, keys=("mu", "log_s", "logit", "shs"), what="No-4DRot ")
    assert np.all(gg["qr"] == 0.0)
    # dL/dq_left by central differences of the oracle (loss = sum dL * image)
    def loss(q):
        Gq = oracle_params(q)
        return sum(float(np.sum(d * O.render(Gq, v)["image"])) for v, d in zip(views, dL))
    top = np.argsort(-np.abs(gg["ql"]).sum(0))[:8]
    eps = grad_floor(gg["ql"])
    for g in top:
        for i in range(4):
            h = 1e-6
            qp, qm = q3.copy(), q3.copy()
            qp[i, g] += h
            qm[i, g] -= h
            fd = (loss(qp) - loss(qm)) / (2 * h)
            assert abs(fd - gg["ql"][i, g]) <= GRAD_TOL * abs(fd) + eps, (g, i, fd, gg["ql"][i, g], eps)
    # no motion: the projected means do not depend on t
    v0, v1 = dict(views[0], t=0.2), dict(views[0], t=0.7)
    f0 = R.Frame(n, [v0, v1], dict(tile_size=32))
    f0.slice_project(p)
    info = f0.layout()
    rec = f0.state[info.records: info.records + 2 * n * info.record_bytes].view(torch.float32).view(2, n, -1)
    tt = f0.state[info.tiles_touched: info.tiles_touched + 8 * n].view(torch.int32).view(2, n)
    both = (tt[0] > 0) & (tt[1] > 0)
    assert int(both.sum()) > 10
    assert torch.equal(rec[0, both, :5], rec[1, both, :5])  # u, v and the conic


def _block_diagonal_pairs(q3):
    """Per Gaussian the quaternion pair (q_l, q_r) whose Eq. 8 rotation is
    blockdiag(R3(q), 1): the oracle's form of a spatial-only rotation."""
    pairs = [_pair_for(np.block([[_r3(q3[:, g]), np.zeros((3, 1))], [np.zeros((1, 3)), np.ones((1, 1))]]))
             for g in range(q3.shape[1])]
    return np.stack([a for a, _ in pairs], 1), np.stack([b for _, b in pairs], 1)


@pytest.mark.parametrize("n_freq,mixed", [(0, False), (1, False), (0, True)])
def test_static_3dgs_special_case_against_oracle(n_freq, mixed):
    """FGS4D_ROT_STATIC (3DGS as the special case of 4DGS, Sec. 3.1): the
    GPU reads neither q_right nor mu_t nor s_t (all NaN here).  The oracle
    renders the same Gaussians as 4D ones with the block-diagonal rotation
    pair and mu_t = the view's t, so that p(t) = 1 and dt = 0 exactly.
    Images and the gradients of mu_xyz, log s_xyz, the opacity and the
    coefficients match element by element; the gradients of q_right, mu_t and
    log s_t are zero; dL/dq_left matches FP64 central differences of the
    oracle through the pair.  Mixed precision (BF16 coefficients, 16-bit
    conics) against the oracle at the rounded coefficients, at the mixed
    tolerances.  The depth and flow maps: static splats do not move, so both
    flow planes are 0, and the depth plane is the oracle's compositing of the
    camera depths."""
    from paper_2310_10642_gb300 import native as N
    G, views = ragged_scene(n=800, seed=47, L=3, K=n_freq)
    if mixed:
        G = dict(G, shs=torch.as_tensor(G["shs"]).to(torch.bfloat16).float().numpy())
    n = G["logit"].shape[0]
    q3 = G["ql"].astype(np.float64)
    ql_o, qr_o = _block_diagonal_pairs(q3)
    Gs = dict(G, rotation=N.ROT_STATIC, qr=np.full_like(G["qr"], np.nan))
    Gs["mu"] = G["mu"].copy()
    Gs["mu"][3] = np.nan
    Gs["log_s"] = G["log_s"].copy()
    Gs["log_s"][3] = np.nan
    opts = dict(tile_size=32, record_fp16=int(mixed), aux_channels=1)
    fr, p, imgs, Ts = gpu_forward(Gs, views, opts, shs_dtype=torch.bfloat16 if mixed else None)
    assert fr.last_counters.status == 0
    img_tol, grad_tol = (1e-3, MIXED_GRAD_TOL) if mixed else (IMG_TOL, GRAD_TOL)

    def oracle_for(v, ql=ql_o, qr=qr_o):
        mu = G["mu"].astype(np.float64).copy()
        mu[3] = v["t"]
        return dict(G, mu=mu, ql=ql, qr=qr)

    refs = [O.render(oracle_for(v), v) for v in views]
    for img, T, ref in zip(imgs, Ts, refs):
        assert_image_parity(img, T, ref, tol=img_tol)
    aux = [a.double().cpu().numpy() for a in fr.split(fr.render_aux().clone())]
    for v, a, ref in zip(views, aux, refs):
        assert np.all(a[1:] == 0.0)  # no motion
        want = O.render_values(oracle_for(v), v, O.aux_values(oracle_for(v), v, 0.0))
        ok = ref["flags"] == 0
        depth_range = max(float(np.abs(want[0]).max()), 1e-9)
        err = float(np.abs(a[0] - want[0])[ok].max()) / depth_range
        assert err <= (3e-3 if mixed else 2e-4), err
    dL = masked_dL(views, refs, 15)
    gg = grads_gpu(fr, p, dL)
    go = None
    for v, d in zip(views, dL):
        o = O.backward(oracle_for(v), v, d)
        o.pop("grad2d")
        go = o if go is None else {k: go[k] + o[k] for k in go}
    for k in ("mu", "log_s"):
        assert_elementwise(gg[k][:3], go[k][:3], grad_tol, f"static {k}[xyz]")
        assert np.all(gg[k][3] == 0.0), k  # no time axis
    assert_grad_parity(gg, go, grad_tol, keys=("logit", "shs"), what="static ")
    assert np.all(gg["qr"] == 0.0)
    if mixed:
        return  # dL/dq_left by differences: covered at FP32

    def loss(q):
        a, b = _block_diagonal_pairs(q)
        return sum(float(np.sum(d * O.render(oracle_for(v, a, b), v)["image"])) for v, d in zip(views, dL))
    eps = grad_floor(gg["ql"])
    for g in np.argsort(-np.abs(gg["ql"]).sum(0))[:4]:
        for i in range(4):
            h = 1e-6
            qp, qm = q3.copy(), q3.copy()
            qp[i, g] += h
            qm[i, g] -= h
            fd = (loss(qp) - loss(qm)) / (2 * h)
            assert abs(fd - gg["ql"][i, g]) <= GRAD_TOL * abs(fd) + eps, (g, i, fd, gg["ql"][i, g], eps)


# ---------------------------------------------------------------------------- depth and flow maps
@pytest.mark.parametrize("tile,mixed", [(16, False), (32, False), (32, True)])
def test_depth_and_flow_maps_match_oracle(tile, mixed):
    """fgs4d_render_aux: accumulated camera depth and the flow of the projected
    conditional means over flow_dt, composited with the image's weights,
    against the oracle's compositing of the same per-splat values."""
    G, views = ragged_scene(n=2500, seed=53)
    dt = 0.02
    opts = dict(tile_size=tile, record_fp16=int(mixed), aux_channels=1, flow_dt=dt)
    fr, p, imgs, Ts = gpu_forward(G, views, opts, shs_dtype=torch.bfloat16 if mixed else None)
    img0 = fr.image.clone()
    aux = [a.double().cpu().numpy() for a in fr.split(fr.render_aux().clone())]
    torch.cuda.synchronize()
    assert torch.equal(img0, fr.image)  # the aux walk leaves the image alone
    Gr = dict(G, shs=torch.as_tensor(G["shs"]).to(torch.bfloat16).float().numpy()) if mixed else G
    tol = 3e-3 if mixed else 2e-4
    for v, a in zip(views, aux):
        ref = O.render(Gr, v)
        vals = O.aux_values(Gr, v, dt)
        want = O.render_values(Gr, v, vals)
        ok = ref["flags"] == 0
        assert ok.mean() > 0.9
        scale = np.abs(vals[np.abs(vals).sum(1) > 0]).max(axis=0)
        for ch, name in enumerate(("depth", "flow u", "flow v")):
            err = np.abs(a[ch] - want[ch])[ok].max() / scale[ch]
            print(f"[parity] aux {name} tile {tile} mixed {mixed}: max error / value range {err:.3e}")
            assert err <= tol, (name, err)
        assert np.abs(want[1:]).max() > 1e-3  # the scene does move


# ---------------------------------------------------------------------------- maximum sizes, other workloads
def test_maximum_sizes():
    """The largest batch (FGS4D_MAX_VIEWS views of uneven sizes in one launch)
    and the widest and tallest images the ABI accepts (16384 pixels)."""
    from paper_2310_10642_gb300 import native as N
    G = I.gaussians(3000, 81, 2, 1)
    r = np.random.default_rng(8)
    views = [I.view(tuple(r.normal(size=3) * 0.3 + np.array([0.0, 0.0, 3.6])), int(r.integers(8, 40)),
                    int(r.integers(8, 40)), float(r.uniform())) for _ in range(N.MAX_VIEWS)]
    for tile in (16, 32):
        _, _, imgs, Ts = gpu_forward(G, views, dict(tile_size=tile))
        for i in (0, 63, N.MAX_VIEWS - 1):
            assert_image_parity(imgs[i], Ts[i], O.render(G, views[i]), max_flag_frac=1.0)
    # 50 degrees along the long side, so each view sees the scene through a thin slot
    for w, h in ((16384, 3), (5, 16384)):
        fx = 0.5 * max(w, h) / math.tan(math.radians(25.0))
        v = I.view((0.0, 0.0, 3.0), w, h, 0.5, fov_x_deg=2.0 * math.degrees(math.atan(0.5 * w / fx)))
        _, _, imgs, Ts = gpu_forward(G, [v], dict(tile_size=32))
        assert_image_parity(imgs[0], Ts[0], O.render(G, v), max_flag_frac=1.0)


def test_config1_crops_and_gradients():
    """Differentiable render at the 100k-Gaussian workload (16 cameras on a
    sphere, 800x800, per-view t): 64x64 crops of two views against the oracle,
    and the gradient of a loss on those crops."""
    c = I.config(1)
    G, views = c["gaussians"], c["views"]
    fr, p, imgs, Ts = gpu_forward(G, views, dict(c["options"], tile_size=32))
    crop = 64
    dL = [np.zeros((3, v["height"], v["width"])) for v in views]
    rng = np.random.default_rng(21)
    picks = [3, 11]
    for vi in picks:
        v = views[vi]
        x0, y0 = v["width"] // 2 - crop // 2, v["height"] // 2 - crop // 2
        ref = O.render(G, v, window=(x0, y0, crop, crop), prefilter=True)
        st = assert_image_parity(imgs[vi][:, y0:y0 + crop, x0:x0 + crop], Ts[vi][y0:y0 + crop, x0:x0 + crop], ref)
        print(f"[parity] config 1 view {vi} crop: {st}")
        w = rng.normal(size=(3, crop, crop))
        w[:, ref["flags"] != 0] = 0.0
        dL[vi][:, y0:y0 + crop, x0:x0 + crop] = w
    gg = grads_gpu(fr, p, dL)
    go = None
    for vi in picks:
        v = views[vi]
        x0, y0 = v["width"] // 2 - crop // 2, v["height"] // 2 - crop // 2
        gv = O.backward(G, v, dL[vi][:, y0:y0 + crop, x0:x0 + crop], window=(x0, y0, crop, crop), prefilter=True)
        gv.pop("grad2d")
        go = gv if go is None else {k: go[k] + gv[k] for k in go}
    assert_grad_parity(gg, go)


@pytest.mark.parametrize("graphs,split", [(False, False), (True, False), (True, True)])
def test_host_pipeline_equals_plain_steps(graphs, split):
    """HostPipeline (copies of neighbouring steps overlapped with compute)
    returns, for each step's host inputs, what a plain forward + backward of
    those inputs returns, eagerly or replaying each slot's captured graph
    (five steps: both slots replay); also with the step as two view groups
    on two streams (SplitFrame), as the benchmark runs it."""
    from paper_2310_10642_gb300 import render as R
    from paper_2310_10642_gb300.pipeline import HostPipeline
    G, views = ragged_scene(n=1500, seed=61)
    p = R.params_to_device(G)
    fr = R.Frame(G["logit"].shape[0], views, dict(tile_size=32))
    fr.forward(p)
    npix = fr.total_pixels
    gen = torch.Generator().manual_seed(2)
    inputs, outputs, want = [], [], []
    for k in range(5):
        hp = {key: (p[key].cpu() + (0.01 * k if key == "mu" else 0.0)).pin_memory() for key in R.PARAM_KEYS}
        hd = torch.randn(3 * npix, generator=gen).pin_memory()
        inputs.append((hp, hd))
        outputs.append((torch.empty(3 * npix).pin_memory(),
                        {key: torch.empty(p[key].shape).pin_memory() for key in R.PARAM_KEYS}))
        dp = dict(p, **{key: hp[key].cuda() for key in R.PARAM_KEYS})
        fr.forward(dp, check=False)
        g = fr.backward(dp, hd.cuda())
        want.append((fr.image.cpu(), {key: v.cpu() for key, v in g.items()}))
    run_frame = fr
    if split:
        run_frame = R.SplitFrame(G["logit"].shape[0], views, dict(tile_size=32), groups=2)
        run_frame.forward(p, check=True)
        assert run_frame.groups == 2
    pipe = HostPipeline(run_frame, p, graphs=graphs)
    pipe.run(inputs, outputs)
    torch.cuda.synchronize()
    assert all((sl["graph"] is not None) == graphs for sl in pipe.slots)
    for (img, g), (wi, wg) in zip(outputs, want):
        assert torch.equal(img, wi)
        for key in R.PARAM_KEYS:
            assert float((g[key] - wg[key]).norm() / wg[key].norm()) < 1e-5, key
