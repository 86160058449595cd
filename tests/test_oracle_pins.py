"""Pins of the FP64 oracle against things other than itself.

Each test names the part of the paper it pins and what it is pinned by: a
printed value (the Eq. 8 sign pattern), a textbook identity computed another
way (Hamilton product, precision-matrix conditioning, scipy's spherical
harmonics), a closed form, an independent static-3DGS renderer for the
space-time-independent special case, or finite differences of the oracle's
own forward pass (for the hand-derived gradient).
"""
import math
import os

import numpy as np
import pytest

from paper_2310_10642_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def hamilton(p, q):
    """Textbook quaternion product p * q, scalar first."""
    a1, b1, c1, d1 = p
    a2, b2, c2, d2 = q
    return np.array([a1 * a2 - b1 * b2 - c1 * c2 - d1 * d2,
                     a1 * b2 + b1 * a2 + c1 * d2 - d1 * c2,
                     a1 * c2 - b1 * d2 + c1 * a2 + d1 * b2,
                     a1 * d2 + b1 * c2 - c1 * b2 + d1 * a2])


def unit(rng, k=4):
    q = rng.normal(size=k)
    return q / np.linalg.norm(q)


# ------------------------------------------------------------------ Eq. 8
def test_eq8_printed_sign_pattern(oracle):
    """The oracle's L(q_l), R(q_r) reproduce the matrices printed in Eq. 8."""
    lines = [l.split() for l in open(os.path.join(GOLDEN, "eq8_rotation_pattern.txt")) if l.strip() and not l.startswith("#")]
    pats = {lines[0][0]: lines[1:5], lines[5][0]: lines[6:10]}
    for name, fn, comps in (("L", oracle.quat_left, "abcd"), ("R", oracle.quat_right, "pqrs")):
        for k, comp in enumerate(comps):
            e = np.zeros(4)
            e[k] = 1.0
            M = fn(e)
            want = np.array([[(1.0 if cell[0] == "+" else -1.0) if cell[1] == comp else 0.0 for cell in row]
                             for row in pats[name]])
            np.testing.assert_array_equal(M, want)


def test_eq8_is_left_and_right_quaternion_multiplication(oracle):
    """R x = q_l * x * q_r (Hamilton product): pins every entry and sign of Eq. 8."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        ql, qr, x = unit(rng), unit(rng), rng.normal(size=4)
        np.testing.assert_allclose(oracle.quat_left(ql) @ x, hamilton(ql, x), atol=1e-14)
        np.testing.assert_allclose(oracle.quat_right(qr) @ x, hamilton(x, qr), atol=1e-14)
        R = oracle.rotation4(ql * 3.0, qr * 0.5)  # normalisation inside
        np.testing.assert_allclose(R @ x, hamilton(hamilton(ql, x), qr), atol=1e-13)


def test_eq8_rotation_invariants(oracle):
    """I1: R R^T = I, det R = +1, and the two isoclinic factors commute."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        ql, qr = unit(rng), unit(rng)
        R = oracle.rotation4(ql, qr)
        np.testing.assert_allclose(R @ R.T, np.eye(4), atol=1e-13)
        assert abs(np.linalg.det(R) - 1.0) < 1e-12
        L, Rr = oracle.quat_left(ql), oracle.quat_right(qr)
        np.testing.assert_allclose(L @ Rr, Rr @ L, atol=1e-13)


def test_eq7_covariance_spectrum(oracle):
    """I2: Sigma = R S S^T R^T is symmetric with eigenvalues s^2."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        ls = rng.normal(-2.0, 1.0, size=4)
        S = oracle.covariance4(ls, unit(rng), unit(rng))
        np.testing.assert_allclose(S, S.T, atol=1e-15)
        np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(S)), np.sort(np.exp(2 * ls)), rtol=1e-10)


# ------------------------------------------------------------------ Eq. 9, Eq. 10, App. B
def test_eq9_matches_precision_matrix_conditioning(oracle):
    """Conditional of a Gaussian computed through the precision matrix
    Lambda = Sigma^-1: Sigma_{x|t} = Lambda_xx^-1, mu_{x|t} = mu_x - Lambda_xx^-1 Lambda_xt (t - mu_t)."""
    rng = np.random.default_rng(4)
    for _ in range(30):
        ls = rng.normal(-2.0, 0.7, size=4)
        Sigma = oracle.covariance4(ls, unit(rng), unit(rng))
        mu = rng.normal(size=4)
        t = rng.normal()
        mu3, S3, p = oracle.condition(mu, Sigma, t)
        Lam = np.linalg.inv(Sigma)
        S3_ref = np.linalg.inv(Lam[:3, :3])
        mu3_ref = mu[:3] - S3_ref @ Lam[:3, 3] * (t - mu[3])
        np.testing.assert_allclose(S3, S3_ref, rtol=1e-8, atol=1e-14)
        np.testing.assert_allclose(mu3, mu3_ref, rtol=1e-8, atol=1e-12)
        # I4: PSD; I5: det Sigma = Sigma_44 det Sigma_{xyz|t} (App. B)
        assert np.linalg.eigvalsh(S3).min() > -1e-12 * np.abs(S3).max()
        np.testing.assert_allclose(np.linalg.det(Sigma), Sigma[3, 3] * np.linalg.det(S3), rtol=1e-9)
        # R1: unnormalised marginal, peak value 1
        assert abs(p - math.exp(-0.5 * (t - mu[3]) ** 2 / Sigma[3, 3])) < 1e-15


def test_appendix_b_factorisation(oracle):
    """The unnormalised 4D Gaussian equals p(t) times the unnormalised
    conditional 3D Gaussian at every point (App. B)."""
    rng = np.random.default_rng(5)
    for _ in range(10):
        Sigma = oracle.covariance4(rng.normal(-1.0, 0.5, size=4), unit(rng), unit(rng))
        mu = rng.normal(size=4)
        Lam = np.linalg.inv(Sigma)
        for _ in range(10):
            x = mu + rng.normal(scale=0.3, size=4)
            mu3, S3, p = oracle.condition(mu, Sigma, x[3])
            d3 = x[:3] - mu3
            joint = math.exp(-0.5 * (x - mu) @ Lam @ (x - mu))
            fact = p * math.exp(-0.5 * d3 @ np.linalg.solve(S3, d3))
            assert abs(joint - fact) < 1e-12 * max(1.0, joint)


def test_eq9_closed_form_xt_rotation(oracle):
    """C1: q_l = q_r = (cos th/2, 0, 0, sin th/2) rotates the x-t plane by th;
    Sigma_xx|t = sx^2 st^2 / D and d mu_x / dt = cos th sin th (sx^2 - st^2) / D,
    D = sin^2 th sx^2 + cos^2 th st^2."""
    for th in (0.1, 0.7, 1.3, 2.9):
        q = np.array([math.cos(th / 2), 0.0, 0.0, math.sin(th / 2)])
        sx, sy, sz, st = 0.3, 0.2, 0.1, 0.5
        Sigma = oracle.covariance4(np.log([sx, sy, sz, st]), q, q)
        D = math.sin(th) ** 2 * sx ** 2 + math.cos(th) ** 2 * st ** 2
        mu = np.array([0.1, 0.2, 0.3, 0.4])
        t = 0.9
        mu3, S3, p = oracle.condition(mu, Sigma, t)
        assert abs(S3[0, 0] - sx ** 2 * st ** 2 / D) < 1e-13
        assert abs(S3[1, 1] - sy ** 2) < 1e-13 and abs(S3[2, 2] - sz ** 2) < 1e-13
        vel = math.cos(th) * math.sin(th) * (sx ** 2 - st ** 2) / D
        assert abs(mu3[0] - (mu[0] + vel * (t - mu[3]))) < 1e-13
        assert abs(p - math.exp(-0.5 * (t - mu[3]) ** 2 / D)) < 1e-14


def test_block_diagonal_rotation_pair(oracle):
    """I3 premise: q_r = (a, b, c, -d) for q_l = (a, b, c, d) leaves the t axis fixed."""
    rng = np.random.default_rng(6)
    for _ in range(10):
        ql = unit(rng)
        qr = ql * np.array([1, 1, 1, -1])
        R = oracle.rotation4(ql, qr)
        np.testing.assert_allclose(R[3], [0, 0, 0, 1], atol=1e-14)
        np.testing.assert_allclose(R[:, 3], [0, 0, 0, 1], atol=1e-14)


# ------------------------------------------------------------------ Eq. 11
def _real_sh_scipy(L, d):
    from scipy.special import sph_harm_y
    x, y, z = d
    theta = math.acos(max(-1.0, min(1.0, z)))
    phi = math.atan2(y, x) % (2 * math.pi)
    out = np.zeros((L + 1) ** 2)
    for l in range(L + 1):
        for m in range(-l, l + 1):
            Yc = complex(sph_harm_y(l, abs(m), theta, phi))
            if m == 0:
                v = Yc.real
            elif m > 0:
                v = math.sqrt(2) * Yc.real
            else:
                v = math.sqrt(2) * Yc.imag
            out[l * l + l + m] = v
    return out


def test_sh_matches_scipy(oracle):
    """Real SH with Condon-Shortley phase: Y_l^m = sqrt2 Re / Im of scipy's complex Y_l^|m|."""
    rng = np.random.default_rng(7)
    for _ in range(40):
        d = unit(rng, 3)
        np.testing.assert_allclose(oracle.sh_basis(4, d), _real_sh_scipy(4, d), atol=1e-12)


def test_sh_orthonormal_by_quadrature(oracle):
    """<Y_i, Y_j> over S^2 = delta_ij (Gauss-Legendre in cos th x uniform phi)."""
    L = 3
    xs, ws = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros(((L + 1) ** 2, (L + 1) ** 2))
    for z, w in zip(xs, ws):
        for k in range(nphi):
            phi = 2 * math.pi * k / nphi
            r = math.sqrt(1 - z * z)
            Y = oracle.sh_basis(L, [r * math.cos(phi), r * math.sin(phi), z])
            G += w * (2 * math.pi / nphi) * np.outer(Y, Y)
    np.testing.assert_allclose(G, np.eye((L + 1) ** 2), atol=1e-12)


def test_sh_gradient_by_differences(oracle):
    """dY from the closed form agrees with central differences of Y."""
    rng = np.random.default_rng(8)
    for _ in range(10):
        d = rng.normal(size=3)
        Y, dY = oracle.sh_basis(3, d, with_grad=True)
        for i in range(3):
            h = np.zeros(3)
            h[i] = 1e-6
            fd = (oracle.sh_basis(3, d + h) - oracle.sh_basis(3, d - h)) / 2e-6
            np.testing.assert_allclose(dY[:, i], fd, atol=1e-7)


# ------------------------------------------------------------------ helpers for renders
def one_gaussian(mu, log_s, ql=(1, 0, 0, 0), qr=(1, 0, 0, 0), logit=0.0, shs=None, L=0, K=0, period=1.0):
    nrow = 3 * (L + 1) ** 2 * (K + 1)
    return dict(mu=np.array(mu, float).reshape(4, 1), log_s=np.array(log_s, float).reshape(4, 1),
                ql=np.array(ql, float).reshape(4, 1), qr=np.array(qr, float).reshape(4, 1),
                logit=np.array([logit], float),
                shs=(np.zeros((nrow, 1)) if shs is None else np.array(shs, float).reshape(nrow, 1)),
                sh_degree=L, n_freq=K, period=period)


def concat(gs):
    out = {k: np.concatenate([g[k] for g in gs], axis=-1) for k in ("mu", "log_s", "ql", "qr", "logit", "shs")}
    for k in ("sh_degree", "n_freq", "period"):
        out[k] = gs[0][k]
    return out


Y00 = 0.5 / math.sqrt(math.pi)


def test_single_isotropic_splat_closed_form(oracle):
    """C2: one isotropic Gaussian on the optical axis at depth z, no dilation:
    Sigma_2d = (f s / z)^2 I, pixel = c a p exp(-r^2 z^2 / (2 f^2 s^2)) + (1 - that) bg."""
    s, st, mu_t, t = 0.05, 0.3, 0.45, 0.5
    k0 = 0.7
    g = one_gaussian([0, 0, 0, mu_t], np.log([s, s, s, st]), logit=0.3, shs=[k0, -k0, 0.2])
    v = I.view((0.0, 0.0, 4.0), 33, 33, t, bg=(0.1, 0.2, 0.3))
    opts = dict(dilation=0.0, clamp_fov=0.0)
    r = oracle.render(g, v, opts)
    f, z = v["fx"], 4.0
    alpha = 1 / (1 + math.exp(-0.3)) * math.exp(-0.5 * (t - mu_t) ** 2 / st ** 2)
    ys, xs = np.mgrid[0:33, 0:33]
    r2 = (xs - 16.0) ** 2 + (ys - 16.0) ** 2
    a = np.minimum(0.99, alpha * np.exp(-0.5 * r2 * z * z / (f * f * s * s)))
    a = np.where(a < 1 / 255, 0.0, a)
    for ch, (kc, bg) in enumerate(zip([k0, -k0, 0.2], (0.1, 0.2, 0.3))):
        c = max(kc * Y00 + 0.5, 0.0)
        np.testing.assert_allclose(r["image"][ch], c * a + (1 - a) * bg, atol=1e-13)
    np.testing.assert_allclose(r["T"], 1 - a, atol=1e-13)


def test_layered_splats_transmittance_and_termination(oracle):
    """B2: three opaque splats stacked in depth: alpha clamps to 0.99 and the
    third would drop T below 1e-4, so it is not added (R4, R5)."""
    gs = [one_gaussian([0, 0, z0, 0.5], np.log([0.3, 0.3, 0.01, 1.0]), logit=8.0, shs=[c, c, c])
          for z0, c in ((0.0, 1.0), (0.5, -0.5), (1.0, 0.3))]
    g = concat(gs)
    v = I.view((0.0, 0.0, 4.0), 5, 5, 0.5, bg=(0.5, 0.5, 0.5))
    r = oracle.render(g, v, dict(dilation=0.0, clamp_fov=0.0))
    c0 = lambda k: max(k * Y00 + 0.5, 0.0)
    # front splat is the one nearest the camera (z0 = 1.0 -> depth 3)
    want = c0(0.3) * 0.99 + c0(-0.5) * 0.99 * 0.01 + 0.5 * 1e-4
    assert abs(r["image"][0, 2, 2] - want) < 1e-12
    assert abs(r["T"][2, 2] - 1e-4) < 1e-15 and r["n_contrib"][2, 2] == 2


def test_ambiguity_bound_covers_flipped_decisions(oracle):
    """The ambiguity bounds that the parity tests add to their tolerance,
    pinned by re-rendering with the decisions taken the other way: moving
    alpha_min (R4) or T_min (R5) by just under the flag margin flips exactly
    the decisions that lie inside it, and the image and T may then move by no
    more than the bounds (1% slack: a flip also rescales the T that later
    flips see by 1/(1 - alpha))."""
    am, tm = oracle.DEFAULT_OPTIONS["alpha_min"], oracle.DEFAULT_OPTIONS["T_min"]
    v = I.view((0.2, -0.1, 3.2), 96, 72, 0.45, bg=(0.3, 0.6, 0.9))
    moved = {"alpha_min": 0, "T_min": 0}
    for dense in (False, True):
        G = I.gaussians(4000, 61, 2, 1)
        if dense:  # larger, more opaque splats: most pixels stop early (R5)
            G["log_s"][:3] += 1.0
            G["logit"] += 3.0
        base = oracle.render(G, v)
        for fa, ft in ((1 + 0.9e-4, 1.0), (1 - 0.9e-4, 1.0), (1.0, 1 + 1.8e-3), (1.0, 1 - 1.8e-3)):
            r = oracle.render(G, v, dict(alpha_min=am * fa, T_min=tm * ft))
            d = np.abs(r["image"] - base["image"]).max(axis=0)
            dT = np.abs(r["T"] - base["T"])
            moved["alpha_min" if ft == 1.0 else "T_min"] += int((d > 1e-12).sum())
            assert np.all(d <= 1.01 * base["amb_image"] + 1e-12)
            assert np.all(dT <= 1.01 * base["amb_T"] + 1e-12)
        # most pixels carry no slack at all
        assert (base["amb_image"] > 0).mean() < 0.1
    # decisions of both kinds did flip: the check is not vacuous
    assert moved["alpha_min"] > 0 and moved["T_min"] > 0


def _point_at(v, px, py, d):
    """World point seen at pixel (px, py) at camera depth d, for a view whose
    camera sits at (0, 0, 4) and looks at the origin (+x right, +y down)."""
    return [(px - v["cx"]) * d / v["fx"], -(py - v["cy"]) * d / v["fy"], 4.0 - d]


def _flip_check(oracle, G, v, base, opts, moved_key, moved):
    r = oracle.render(G, v, opts)
    d = np.abs(r["image"] - base["image"]).max(axis=0)
    dT = np.abs(r["T"] - base["T"])
    moved[moved_key] += int((d > 1e-12).sum())
    assert np.all(d <= 1.01 * base["amb_image"] + 1e-12), (moved_key, float((d - base["amb_image"]).max()))
    assert np.all(dT <= 1.01 * base["amb_T"] + 1e-12), moved_key


def test_ambiguity_bound_covers_borderline_culls(oracle):
    """The bound's Gaussian-level terms, pinned by flipping the culls that lie
    inside their margins: Gaussians planted with p(t) (Sec. 4.2 filter), the
    camera depth (near plane) or alpha_eff (R7) within half a margin of the
    threshold, over a sparse random scene; moving p_min, near_z or alpha_min
    by 0.9 of its margin culls or keeps each of them the other way, and
    image and T may move by no more than the bounds."""
    o = oracle.DEFAULT_OPTIONS
    t = 0.5
    v = I.view((0.0, 0.0, 4.0), 80, 64, t, bg=(0.3, 0.6, 0.9))
    rng = np.random.default_rng(71)
    planted = []
    amin = o["alpha_min"]
    for k in range(72):
        kind = k % 3
        sign = 1.0 if (k // 3) % 2 == 0 else -1.0
        px, py = rng.uniform(4, 76), rng.uniform(4, 60)
        if kind == 0:  # p(t) = p_min (1 +- 0.5e-4) with Sigma_44 = s_t^2 (identity rotation pair)
            st = 0.1
            dt = st * math.sqrt(-2.0 * math.log(o["p_min"] * (1.0 + sign * 0.5e-4)))
            g = one_gaussian(_point_at(v, px, py, 3.0) + [t - dt], np.log([0.03, 0.03, 0.03, st]), logit=2.0,
                             shs=rng.normal(0, 1, 3))
        elif kind == 1:  # camera depth = near_z (1 +- 0.5e-4)
            d = o["near_z"] * (1.0 + sign * 0.5e-4)
            g = one_gaussian(_point_at(v, px, py, d) + [t], np.log([0.002, 0.002, 0.002, 1.0]), logit=2.0,
                             shs=rng.normal(0, 1, 3))
        else:  # alpha_eff = sigmoid(logit) p = alpha_min (1 +- 0.5e-4), p = 1
            a = amin * (1.0 + sign * 0.5e-4)
            g = one_gaussian(_point_at(v, px, py, 2.5) + [t], np.log([0.03, 0.03, 0.03, 1.0]),
                             logit=math.log(a / (1.0 - a)), shs=rng.normal(0, 1, 3))
        planted.append(g)
    bgG = I.gaussians(1500, 62, 0, 0)
    bgG["mu"][3] = t
    G = concat([{k: (bgG[k] if k in ("sh_degree", "n_freq", "period") else bgG[k].astype(np.float64))
                 for k in bgG}] + planted)
    base = oracle.render(G, v)
    flagged_cull = (base["flags"] & 32) != 0
    assert flagged_cull.sum() > 20  # the planted culls are flagged where they could be blended
    moved = {"p_min": 0, "near_z": 0, "alpha_min": 0}
    for key in moved:
        for f in (1 + 0.9e-4, 1 - 0.9e-4):
            _flip_check(oracle, G, v, base, {key: o[key] * f}, key, moved)
    assert all(m > 0 for m in moved.values()), moved  # each kind of cull did flip
    assert (base["amb_image"] > 0).mean() < 0.3


def test_ambiguity_bound_covers_depth_ties(oracle):
    """The bound's depth near-tie term (R8: equal depths are ordered by
    index), pinned by swapping the order of overlapping splats of equal
    depth: each pair sits at one world z in front of a camera looking down
    -z (so both depths are the same double), and the scene is rendered with
    the pair's indices in both orders.  The image moves by no more than the
    bound of either render, T does not move (both orders remove the same
    light), and the tie is flagged as such (cause bit 4)."""
    t = 0.5
    v = I.view((0.0, 0.0, 4.0), 64, 48, t, bg=(0.2, 0.2, 0.2))
    rng = np.random.default_rng(72)
    pairs = []
    for k in range(24):
        px, py = rng.uniform(6, 56), rng.uniform(6, 42)
        d = 2.0 + 0.05 * k  # pairs at distinct depths: only the two splats of a pair are tied
        pairs.append([one_gaussian(_point_at(v, px + dx, py, d) + [t], np.log([0.02, 0.02, 0.02, 1.0]), logit=1.5,
                                   shs=rng.normal(0, 1.5, 3)) for dx in (0.0, 1.5)])
    rf = oracle.render(concat([g for a, b in pairs for g in (a, b)]), v)
    rb = oracle.render(concat([g for a, b in pairs for g in (b, a)]), v)
    d = np.abs(rf["image"] - rb["image"]).max(axis=0)
    assert (d > 1e-6).sum() > 50  # the order matters on many pixels
    assert np.all(((rf["flags"] & 4) != 0)[d > 1e-5]) and np.all(((rb["flags"] & 4) != 0)[d > 1e-5])
    for r in (rf, rb):
        assert np.all(d <= 1.01 * r["amb_image"] + 1e-12), float((d - r["amb_image"]).max())
    assert np.abs(rf["T"] - rb["T"]).max() < 1e-12


def test_eq4_off_axis_jacobian_by_differences(oracle):
    """Eq. 3-4 off the optical axis, against the mathematics rather than a
    restated Jacobian: J = d(u, v)/d(X, Y, Z) taken by central differences of
    the pinhole map (u, v) = (fx X/Z + cx, fy Y/Z + cy), and the 2D mean by
    the homogeneous product K (W x + tau); the oracle's 2D covariance must
    equal J W Sigma_{xyz|t} W^T J^T + dilation I (clamp off) at points up to
    ~30 degrees off axis in every direction, with a full 4D rotation."""
    rng = np.random.default_rng(73)
    v = I.view((0.7, -0.4, 3.6), 120, 90, 0.4)
    vm = np.asarray(v["viewmat"]).reshape(3, 4)
    W, tau = vm[:, :3], vm[:, 3]
    Kmat = np.array([[v["fx"], 0, v["cx"]], [0, v["fy"], v["cy"]], [0, 0, 1.0]])
    opts = dict(clamp_fov=0.0, dilation=0.3)

    def pinhole(xc):
        return np.array([v["fx"] * xc[0] / xc[2] + v["cx"], v["fy"] * xc[1] / xc[2] + v["cy"]])

    checked = 0
    for k in range(40):
        # a camera-space point well off axis, mapped back to world coordinates
        Z = rng.uniform(1.5, 5.0)
        xc = np.array([rng.uniform(-0.6, 0.6) * Z, rng.uniform(-0.6, 0.6) * Z, Z])
        xw = W.T @ (xc - tau)
        g = one_gaussian(list(xw) + [0.4 + rng.uniform(-0.05, 0.05)], rng.normal(-2.5, 0.3, 4),
                         ql=unit(rng), qr=unit(rng), logit=3.0)
        s = oracle.project(g, 0, v, opts)
        if s.depth <= 0.0 or s.cull in (2, 4):
            continue
        x3 = np.array(s.xc)
        J = np.zeros((2, 3))
        for i in range(3):
            h = 1e-6 * max(1.0, abs(x3[i]))
            e = np.zeros(3)
            e[i] = h
            J[:, i] = (pinhole(x3 + e) - pinhole(x3 - e)) / (2 * h)
        S3 = np.array(s.Sigma3).reshape(3, 3)
        want = J @ W @ S3 @ W.T @ J.T + 0.3 * np.eye(2)
        got = np.array([[s.cov2d[0], s.cov2d[1]], [s.cov2d[1], s.cov2d[2]]])
        np.testing.assert_allclose(got, want, rtol=1e-7, atol=1e-9 * np.abs(want).max())
        hom = Kmat @ (W @ np.array(s.mu3) + tau)
        np.testing.assert_allclose([s.u, s.v], hom[:2] / hom[2], rtol=1e-12, atol=1e-9)
        assert abs(x3[0] / x3[2]) > 0.05 or abs(x3[1] / x3[2]) > 0.05  # off axis
        checked += 1
    assert checked >= 30


def test_temporal_filter_culls_below_threshold(oracle):
    """p(t) < 0.05 removes the Gaussian entirely (Sec. 4.2)."""
    st = 0.1
    # p = exp(-0.5 (dt/st)^2) = 0.04 and 0.06
    for p_want, visible in ((0.04, 0), (0.06, 1)):
        dt = st * math.sqrt(-2 * math.log(p_want))
        g = one_gaussian([0, 0, 0, 0.5 - dt], np.log([0.2, 0.2, 0.2, st]), logit=5.0)
        v = I.view((0.0, 0.0, 4.0), 9, 9, 0.5)
        s = oracle.project(g, 0, v)
        assert s.visible == visible
        assert abs(s.p_t - p_want) < 1e-12


def test_fourier_period_and_plain_sh_reduction(oracle):
    """Eq. 11: colour is T-periodic in dt and with K = 0 equals sum k Y(d) + 0.5."""
    rng = np.random.default_rng(9)
    L, K, T = 2, 2, 0.8
    shs = rng.normal(0, 0.2, size=3 * 9 * 3)
    ql = unit(rng)
    qr = ql * np.array([1, 1, 1, -1])  # block-diagonal: mu3 does not move with t
    base = dict(log_s=np.log([0.1, 0.1, 0.1, 5.0]), ql=ql, qr=qr, logit=2.0, shs=shs, L=L, K=K, period=T)
    v = I.view((0.5, -0.3, 4.0), 16, 16, 0.5)
    a = oracle.project(one_gaussian([0.1, 0.2, 0.0, 0.3], **base), 0, v)
    b = oracle.project(one_gaussian([0.1, 0.2, 0.0, 0.3 - T], **base), 0, v)
    np.testing.assert_allclose(list(a.color_raw), list(b.color_raw), atol=1e-12)
    g0 = one_gaussian([0.1, 0.2, 0.0, 0.3], np.log([0.1, 0.1, 0.1, 5.0]), ql, qr, 2.0, shs[:27], L=L, K=0)
    s0 = oracle.project(g0, 0, v)
    C = -np.asarray(v["viewmat"]).reshape(3, 4)[:, :3].T @ np.asarray(v["viewmat"]).reshape(3, 4)[:, 3]
    d = np.array(s0.mu3) - C
    Y = _real_sh_scipy(L, d / np.linalg.norm(d))
    want = [shs[:27].reshape(9, 3)[:, ch] @ Y for ch in range(3)]
    np.testing.assert_allclose(list(s0.color_raw), want, atol=1e-12)


# ------------------------------------------------------------------ I3: reduction to static 3DGS
def static_3dgs_render(mu3, Sig3, opacity, colors, view, opts):
    """Independent brute-force 3DGS renderer (Eq. 2 with the fixed product,
    Eq. 3, Eq. 4), numpy, for the space-time-independent special case."""
    vm = np.asarray(view["viewmat"]).reshape(3, 4)
    W, tau = vm[:, :3], vm[:, 3]
    fx, fy, cx, cy = view["fx"], view["fy"], view["cx"], view["cy"]
    Wd, Ht = view["width"], view["height"]
    recs = []
    for i in range(mu3.shape[0]):
        xc = W @ mu3[i] + tau
        if xc[2] < opts["near_z"]:
            continue
        X, Y, Z = xc
        J = np.array([[fx / Z, 0, -fx * X / Z ** 2], [0, fy / Z, -fy * Y / Z ** 2]])
        C2 = J @ W @ Sig3[i] @ W.T @ J.T + opts["dilation"] * np.eye(2)
        recs.append((Z, i, fx * X / Z + cx, fy * Y / Z + cy, np.linalg.inv(C2)))
    recs.sort(key=lambda r: (r[0], r[1]))
    ys, xs = np.mgrid[0:Ht, 0:Wd].astype(float)
    img = np.zeros((3, Ht, Wd))
    T = np.ones((Ht, Wd))
    alive = np.ones((Ht, Wd), bool)
    for Z, i, u, v, Q in recs:
        if opacity[i] < opts["alpha_min"]:
            continue
        dx, dy = xs - u, ys - v
        q = Q[0, 0] * dx * dx + 2 * Q[0, 1] * dx * dy + Q[1, 1] * dy * dy
        a = np.minimum(opts["alpha_max"], opacity[i] * np.exp(-0.5 * q))
        use = alive & (a >= opts["alpha_min"])
        Tn = T * (1 - a)
        stop = use & (Tn < opts["T_min"])
        alive &= ~stop
        use &= ~stop
        for ch in range(3):
            img[ch] += np.where(use, colors[i, ch] * a * T, 0.0)
        T = np.where(use, Tn, T)
    return img + T[None] * np.asarray(view["bg"])[:, None, None], T


def test_reduction_to_static_3dgs(oracle):
    """I3 / No-4DRot (Sec. 3.2): with a block-diagonal rotation the 4D render
    equals a static 3DGS render with opacity scaled by exp(-(t-mu_t)^2 / (2 s_t^2))."""
    rng = np.random.default_rng(10)
    n = 48
    ql = rng.normal(size=(4, n))
    ql /= np.linalg.norm(ql, axis=0)
    qr = ql * np.array([1, 1, 1, -1])[:, None]
    mu = np.concatenate([rng.uniform(-0.8, 0.8, size=(3, n)), rng.uniform(0.3, 0.7, size=(1, n))])
    log_s = np.concatenate([rng.normal(-2.5, 0.3, size=(3, n)), rng.normal(-1.5, 0.3, size=(1, n))])
    logit = rng.normal(size=n)
    K, T = 1, 1.0
    shs = rng.normal(0, 0.3, size=(3 * 1 * 2, n))
    g = dict(mu=mu, log_s=log_s, ql=ql, qr=qr, logit=logit, shs=shs, sh_degree=0, n_freq=K, period=T)
    t = 0.5
    v = I.view((0.3, -0.2, 4.0), 40, 32, t, bg=(0.2, 0.1, 0.0))
    opts = dict(I.DEFAULT_OPTIONS, clamp_fov=0.0)
    r = oracle.render(g, v, opts)
    # static path
    mu3 = mu[:3].T
    Sig3 = np.zeros((n, 3, 3))
    op = np.zeros(n)
    colors = np.zeros((n, 3))
    for i in range(n):
        R3 = oracle.rotation4(ql[:, i], qr[:, i])[:3, :3]
        Sig3[i] = R3 @ np.diag(np.exp(2 * log_s[:3, i])) @ R3.T
        p = math.exp(-0.5 * (t - mu[3, i]) ** 2 / math.exp(2 * log_s[3, i]))
        op[i] = (1 / (1 + math.exp(-logit[i]))) * p if p >= opts["p_min"] else 0.0
        dt = t - mu[3, i]
        for ch in range(3):
            raw = sum(math.cos(2 * math.pi * f * dt / T) * shs[f * 3 + ch, i] * Y00 for f in range(K + 1))
            colors[i, ch] = max(raw + 0.5, 0.0)
    img, Ts = static_3dgs_render(mu3, Sig3, op, colors, v, opts)
    ok = r["flags"] == 0
    assert ok.mean() > 0.95
    np.testing.assert_allclose(r["image"][:, ok], img[:, ok], atol=1e-10)
    np.testing.assert_allclose(r["T"][ok], Ts[ok], atol=1e-10)


def test_prefilter_is_exact(oracle):
    """The R7 support bound only skips splats whose alpha is below alpha_min."""
    c = I.config(0, n=400)
    v = c["views"][0]
    a = oracle.render(c["gaussians"], v, prefilter=False)
    b = oracle.render(c["gaussians"], v, prefilter=True)
    np.testing.assert_array_equal(a["image"], b["image"])
    np.testing.assert_array_equal(a["n_contrib"], b["n_contrib"])


# ------------------------------------------------------------------ O9: hand-derived gradient
def _loss(oracle, g, views, weights, opts):
    return sum(float(np.sum(w * oracle.render(g, v, opts)["image"])) for v, w in zip(views, weights))


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_central_differences(oracle, seed):
    """O9: analytic gradient of sum(w * image) equals FP64 central differences
    for every parameter kind, on parameters whose perturbation changes no
    discrete decision (checked by comparing two step sizes)."""
    rng = np.random.default_rng(100 + seed)
    g = I.gaussians(24, 777 + seed, 2, 2, period=1.0)
    g = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) else v) for k, v in g.items()}
    g["mu"][:3] *= 0.6
    g["log_s"][:3] += 1.0  # larger splats: more pixels per splat
    views = [I.view((0.4, 0.3, 3.5), 24, 20, 0.45, bg=(0.3, 0.2, 0.1)),
             I.view((-1.0, 0.5, 3.0), 20, 24, 0.55)]
    opts = dict(I.DEFAULT_OPTIONS, clamp_fov=1.3)
    weights = [rng.normal(size=(3, v["height"], v["width"])) for v in views]
    grads = None
    for v, w in zip(views, weights):
        gg = oracle.backward(g, v, w, opts)
        gg.pop("grad2d")
        grads = gg if grads is None else {k: grads[k] + gg[k] for k in grads}
    checked = 0
    for key in ("mu", "log_s", "ql", "qr", "logit", "shs"):
        arr = g[key]
        idxs = [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(12)]
        for idx in idxs:
            x0 = arr[idx]
            fds = []
            for h in (1e-6, 2e-6):
                arr[idx] = x0 + h
                lp = _loss(oracle, g, views, weights, opts)
                arr[idx] = x0 - h
                lm = _loss(oracle, g, views, weights, opts)
                arr[idx] = x0
                fds.append((lp - lm) / (2 * h))
            if abs(fds[0] - fds[1]) > 1e-6 * max(1.0, abs(fds[0])):
                continue  # a discrete decision flipped inside the stencil
            an = grads[key][idx]
            assert abs(an - fds[0]) <= 1e-6 * max(1.0, abs(fds[0])), (key, idx, an, fds[0])
            checked += 1
    assert checked >= 50


def test_render_values_uses_the_image_weights(oracle):
    """orc_render_values (depth and flow maps) composites with the walk of
    Eq. 6: a constant value c gives c (1 - T_final) (the weights alpha_i T_i
    sum to 1 - T_final), and the splats' own colours give the image without
    its background term."""
    G = I.gaussians(1500, 71, 2, 1)
    v = I.view((0.3, 0.1, 3.5), 48, 40, 0.4, bg=(0.2, 0.5, 0.8))
    ref = oracle.render(G, v)
    n = G["logit"].shape[0]
    c = np.array([2.5, -1.0, 0.25])
    out = oracle.render_values(G, v, np.tile(c, (n, 1)))
    assert np.abs(out - c[:, None, None] * (1.0 - ref["T"])[None]).max() < 1e-12
    col = oracle.project_all(G, v)["color"]
    out = oracle.render_values(G, v, col)
    bg = np.array(v["bg"])[:, None, None] * ref["T"][None]
    assert np.abs(out - (ref["image"] - bg)).max() < 1e-12
    assert (1.0 - ref["T"]).max() > 0.5  # not an empty image


def test_aux_flow_is_the_projected_displacement(oracle):
    """aux_values: zero flow without space-time coupling (q_l = q_r = 1); with
    an x-t rotation the conditional mean moves by Sigma_xt / Sigma_tt per unit
    of t (Eq. 9) and the flow is the pinhole projection of that move."""
    v = I.view((0.0, 0.0, 4.0), 64, 64, 0.5)
    dt = 0.01
    one = np.array([1.0, 0.0, 0.0, 0.0])
    G = I.gaussians(3, 72, 0, 0)
    G["mu"][:] = np.array([[0.1, -0.2, 0.0, 0.5]] * 3).T
    G["ql"][:] = one[:, None]
    G["qr"][:] = one[:, None]
    G["log_s"][:] = np.log(np.array([0.3, 0.2, 0.2, 0.1]))[:, None]  # anisotropic in x and t
    aux = oracle.aux_values(G, v, dt)
    assert np.abs(aux[:, 1:]).max() < 1e-12
    # rotation by th in the x-t plane: Sigma_xt / Sigma_tt = (s_x^2 - s_t^2) sin cos / (s_x^2 sin^2 + s_t^2 cos^2)
    th = 0.4
    q = np.array([np.cos(th / 2), 0, 0, np.sin(th / 2)])
    G["ql"][:] = q[:, None]
    G["qr"][:] = q[:, None]
    R = oracle.rotation4(G["ql"][:, 0], G["qr"][:, 0])  # the stored (float32) quaternions
    Sigma = R @ np.diag(np.exp(2 * G["log_s"][:, 0].astype(np.float64))) @ R.T
    vel = Sigma[:3, 3] / Sigma[3, 3]
    aux = oracle.aux_values(G, v, dt)
    Vm = np.asarray(v["viewmat"]).reshape(3, 4)
    mu3, _, _ = oracle.condition(G["mu"][:, 0], Sigma, v["t"])
    x0, x1 = Vm[:, :3] @ mu3 + Vm[:, 3], Vm[:, :3] @ (mu3 + vel * dt) + Vm[:, 3]
    want = np.array([v["fx"] * (x1[0] / x1[2] - x0[0] / x0[2]), v["fy"] * (x1[1] / x1[2] - x0[1] / x0[2])])
    assert np.abs(aux[0, 1:] - want).max() < 1e-12 and np.abs(want).max() > 1e-3
