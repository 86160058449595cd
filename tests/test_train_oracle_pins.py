"""Pins of the training-step oracle (loss and Adam) against things other than
itself: scipy's correlation, identities and closed forms of SSIM, a
per-pixel brute force of the SSIM definition, central differences for the
hand-derived gradient, and Adam's first step in closed form."""
import math

import numpy as np
import pytest

from oracle import train_oracle as T


def test_gaussian_window_taps():
    g = T.gaussian_taps()
    assert g.shape == (11,) and abs(g.sum() - 1.0) < 1e-15
    assert np.allclose(g, g[::-1], rtol=0, atol=1e-17)
    assert abs(g[6] / g[5] - math.exp(-1.0 / (2 * 1.5 ** 2))) < 1e-15


def test_window_sum_is_scipy_correlate_with_zero_padding():
    scipy_ndimage = pytest.importorskip("scipy.ndimage")
    r = np.random.default_rng(1)
    img = r.uniform(size=(23, 17))
    g = T.gaussian_taps()
    want = scipy_ndimage.correlate(img, np.outer(g, g), mode="constant", cval=0.0)
    assert np.abs(T.window_sum(img) - want).max() < 1e-14


def test_ssim_of_an_image_with_itself_is_one_and_stationary():
    r = np.random.default_rng(2)
    x = r.uniform(size=(3, 14, 19))
    assert np.abs(T.ssim_map(x[0], x[0]) - 1.0).max() < 1e-12
    loss, (g,) = T.loss_l1_dssim([x], [x.copy()])
    assert abs(loss) < 1e-12 and np.abs(g).max() < 1e-12


def test_ssim_of_constant_images_closed_form():
    a, b = 0.3, 0.7
    s = T.ssim_map(np.full((40, 40), a), np.full((40, 40), b))
    interior = s[5:-5, 5:-5]  # the window lies inside the image: unit mass, zero variance
    want = (2 * a * b + T.C1) / (a * a + b * b + T.C1)
    assert np.abs(interior - want).max() < 1e-12
    # at a corner the window keeps only part of its mass (zero padding): a different value
    assert abs(s[0, 0] - want) > 1e-3


def test_ssim_brute_force_per_pixel():
    r = np.random.default_rng(3)
    x, y = r.uniform(size=(13, 11)), r.uniform(size=(13, 11))
    g = T.gaussian_taps()
    s = T.ssim_map(x, y)
    for (py, px) in ((0, 0), (6, 5), (12, 10), (3, 9)):
        mx = my = exx = eyy = exy = 0.0
        for dy in range(-5, 6):
            for dx in range(-5, 6):
                qy, qx = py + dy, px + dx
                if 0 <= qy < 13 and 0 <= qx < 11:
                    wt = g[dy + 5] * g[dx + 5]
                    mx += wt * x[qy, qx]
                    my += wt * y[qy, qx]
                    exx += wt * x[qy, qx] ** 2
                    eyy += wt * y[qy, qx] ** 2
                    exy += wt * x[qy, qx] * y[qy, qx]
        vx, vy, cxy = exx - mx * mx, eyy - my * my, exy - mx * my
        want = (2 * mx * my + T.C1) * (2 * cxy + T.C2) / ((mx * mx + my * my + T.C1) * (vx + vy + T.C2))
        assert abs(s[py, px] - want) < 1e-13


def test_loss_gradient_by_central_differences():
    r = np.random.default_rng(4)
    ims = [r.uniform(size=(3, 9, 7)), r.uniform(size=(3, 6, 10))]
    tgs = [r.uniform(size=(3, 9, 7)), r.uniform(size=(3, 6, 10))]
    _, grads = T.loss_l1_dssim(ims, tgs, 0.2)
    h = 1e-6
    checked = 0
    for _ in range(60):
        vi = int(r.integers(0, 2))
        idx = tuple(int(r.integers(0, s)) for s in ims[vi].shape)
        if abs(ims[vi][idx] - tgs[vi][idx]) < 10 * h:
            continue  # the L1 kink
        p = [a.copy() for a in ims]
        m = [a.copy() for a in ims]
        p[vi][idx] += h
        m[vi][idx] -= h
        fd = (T.loss_l1_dssim(p, tgs, 0.2)[0] - T.loss_l1_dssim(m, tgs, 0.2)[0]) / (2 * h)
        an = grads[vi][idx]
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-10, (vi, idx, fd, an)
        checked += 1
    assert checked >= 50


def test_adam_first_step_closed_form():
    # m0 = v0 = 0: the bias-corrected moments are g and g^2, so the step is lr g / (|g| + eps)
    r = np.random.default_rng(5)
    p0, g = r.normal(size=50), r.normal(size=50)
    lr, eps = 1e-3, 1e-8
    p1, m1, v1 = T.adam_step(p0, np.zeros(50), np.zeros(50), g, 1, lr, 0.9, 0.999, eps)
    assert np.abs(p1 - (p0 - lr * g / (np.abs(g) + eps))).max() < 1e-15
    assert np.allclose(m1, 0.1 * g, rtol=1e-12, atol=0) and np.allclose(v1, 0.001 * g * g, rtol=1e-12, atol=0)


def test_adam_second_step_by_hand():
    # scalar, g1 = 2, g2 = -1, beta1 = 0.9, beta2 = 0.999, lr = 0.1, eps = 0
    p, m, v = T.adam_step(1.0, 0.0, 0.0, 2.0, 1, 0.1, 0.9, 0.999, 1e-300)
    p, m, v = T.adam_step(p, m, v, -1.0, 2, 0.1, 0.9, 0.999, 1e-300)
    m_want = 0.9 * 0.2 + 0.1 * -1.0                   # 0.08
    v_want = 0.999 * 0.004 + 0.001 * 1.0               # 0.004996
    p_want = (1.0 - 0.1) - 0.1 * (m_want / (1 - 0.81)) / math.sqrt(v_want / (1 - 0.998001))
    assert abs(m - m_want) < 1e-15 and abs(v - v_want) < 1e-15 and abs(p - p_want) < 1e-12
