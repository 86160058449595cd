"""The seeded input generators both sides are fed from: determinism, the
shapes and distributions of the recipe, and cameras that look at their
target (CPU only; the module holds none of the rendering arithmetic)."""
import numpy as np
import pytest

from paper_2310_10642_gb300 import inputs as I


def test_same_seed_same_inputs_and_seeds_differ_per_workload():
    a = I.config(1, n=500, n_views=3)
    b = I.config(1, n=500, n_views=3)
    for k in ("mu", "log_s", "ql", "qr", "logit", "shs"):
        assert np.array_equal(a["gaussians"][k], b["gaussians"][k])
    assert [v["t"] for v in a["views"]] == [v["t"] for v in b["views"]]
    c = I.config(2, n=500, n_views=3)
    assert not np.array_equal(a["gaussians"]["mu"], c["gaussians"]["mu"])


@pytest.mark.parametrize("k,L,K", [(0, 1, 1), (1, 3, 2), (3, 3, 2)])
def test_parameter_layout(k, L, K):
    G = I.config(k, n=1000, n_views=2)["gaussians"]
    n = 1000
    assert G["sh_degree"] == L and G["n_freq"] == K
    assert G["mu"].shape == (4, n) and G["log_s"].shape == (4, n)
    assert G["ql"].shape == (4, n) and G["qr"].shape == (4, n) and G["logit"].shape == (n,)
    assert G["shs"].shape == (3 * (L + 1) ** 2 * (K + 1), n)
    for key in ("mu", "log_s", "ql", "qr", "logit", "shs"):
        assert G[key].dtype == np.float32 and G[key].flags["C_CONTIGUOUS"]


def test_distributions_of_the_recipe():
    n = 200_000
    G = I.gaussians(n, 7, 3, 2)
    assert np.all(np.abs(G["mu"][:3]) <= 1.0) and np.all((G["mu"][3] >= 0.0) & (G["mu"][3] <= 1.0))
    assert abs(G["log_s"][:3].mean() + 3.0) < 0.01 and abs(G["log_s"][:3].std() - 0.5) < 0.01
    assert abs(G["log_s"][3].mean() + 2.0) < 0.01 and abs(G["log_s"][3].std() - 0.5) < 0.01
    assert abs(G["logit"].mean()) < 0.01 and abs(G["logit"].std() - 1.0) < 0.01
    assert abs(G["shs"].std() - 0.2) < 0.002
    # normal quaternions are uniform on S^3 after normalisation: each squared component averages 1/4
    q = G["ql"] / np.linalg.norm(G["ql"], axis=0)
    assert np.allclose((q * q).mean(axis=1), 0.25, atol=0.005)


def test_clustered_means_mix_blobs_and_uniform_points_70_30():
    n = 100_000
    G = I.gaussians(n, 11, 1, 1, clustered=True)
    xyz = G["mu"][:3].T.astype(np.float64)
    centres = I.rng(11).uniform(-1.0, 1.0, size=(64, 3))  # the generator's first draw

    def near(p, r=0.2):
        return float((np.min(np.linalg.norm(p[:, None, :] - centres[None], axis=2), axis=1) < r).mean())

    # the share within 0.2 of a centre, against the same share for pure blob points
    # (sigma 0.1) and pure uniform points drawn independently here
    s = np.random.default_rng(5)
    blob = centres[s.integers(0, 64, size=n)] + s.normal(0.0, 0.1, size=(n, 3))
    uni = s.uniform(-1.0, 1.0, size=(n, 3))
    want = 0.7 * near(blob) + 0.3 * near(uni)
    assert near(blob) - near(uni) > 0.3  # the share separates the two kinds
    assert abs(near(xyz) - want) < 0.01


def test_cameras_look_at_the_target():
    for eye in I.arc_eyes(5) + 0.0:
        v = I.view(eye, 1352, 1014, 0.5)
        M = np.asarray(v["viewmat"]).reshape(3, 4)
        W, tau = M[:, :3], M[:, 3]
        assert np.allclose(W @ W.T, np.eye(3), atol=1e-12) and np.linalg.det(W) > 0
        xc = W @ np.zeros(3) + tau  # the target projects to the principal point, in front
        assert xc[2] > 0
        assert abs(v["fx"] * xc[0] / xc[2]) < 1e-9 and abs(v["fy"] * xc[1] / xc[2]) < 1e-9
        assert v["cx"] == (1352 - 1) / 2 and v["cy"] == (1014 - 1) / 2
        # 50 degrees of horizontal field of view
        assert np.isclose(2 * np.degrees(np.arctan(0.5 * 1352 / v["fx"])), 50.0)
        # +y points down: a world point above the target lands above the image centre
        up = W @ np.array([0.0, 1.0, 0.0]) + tau
        assert up[1] / up[2] < 0


def test_workload_view_sets():
    c3 = I.config(3, n=100)
    assert len(c3["views"]) == 20 and {(v["width"], v["height"]) for v in c3["views"]} == {(1352, 1014)}
    frames = np.arange(300) / 299.0
    assert all(np.isclose(frames, v["t"]).any() for v in c3["views"])
    c4 = I.config(4, n=100)
    sizes = [(v["width"], v["height"]) for v in c4["views"]]
    assert sizes == [(1352, 1014)] * 4 + [(800, 800)] * 4
    c2 = I.config(2, n=100)
    assert len(c2["views"]) == 100


def test_split_views_balances_contiguous_groups():
    """The view groups of SplitFrame: contiguous, non-empty, balanced by pixel
    count, and never more groups than views."""
    from paper_2310_10642_gb300 import render as R
    same = [I.view((0, 0, 4), 100, 80, 0.5)] * 20
    assert R.split_views(same, 2) == [10]
    assert R.split_views(same, 4) == [5, 10, 15]
    assert R.split_views(same[:1], 2) == [] and R.split_views(same[:3], 5) == [1, 2]
    uneven = [I.view((0, 0, 4), 100, 100, 0.5), I.view((0, 0, 4), 10, 10, 0.5), I.view((0, 0, 4), 100, 100, 0.5)]
    assert R.split_views(uneven, 2) == [2]
    c = I.config(2, n=10, scale=0.1)
    cuts = R.split_views(c["views"], 2)
    pix = [v["width"] * v["height"] for v in c["views"]]
    a = sum(pix[:cuts[0]])
    assert abs(a - (sum(pix) - a)) <= max(pix)
