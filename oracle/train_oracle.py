"""FP64 oracle of the training step around the renderer: test infrastructure.

Only tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline may
import this module; nothing on the product path does.  Plain numpy in double
precision, written from the definitions (no blocking, no fusion):

* the photometric loss the paper trains with (Sec. 3.3; the setting of Sec.
  4.1 adopts 3D Gaussian splatting's loss): L = (1 - lambda) L1 +
  lambda (1 - SSIM), as a mean over all pixels and channels of the batch;
  SSIM is the structural similarity of Wang et al. (2004) with an 11x11
  Gaussian window (sigma 1.5, normalised), zero padding, C1 = 0.01^2,
  C2 = 0.03^2;
* its gradient w.r.t. the rendered images, derived by hand (chain rule
  through the window moments);
* Adam (Kingma and Ba, 2015, Algorithm 1, with bias correction), the
  optimiser the paper trains with.
"""
from __future__ import annotations

import numpy as np

RADIUS = 5
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def gaussian_taps() -> np.ndarray:
    """exp(-i^2 / (2 sigma^2)) for i = -5..5, normalised to sum 1."""
    i = np.arange(-RADIUS, RADIUS + 1, dtype=np.float64)
    g = np.exp(-(i * i) / (2.0 * SIGMA * SIGMA))
    return g / g.sum()


def window_sum(img: np.ndarray) -> np.ndarray:
    """sum_{dy,dx} w(dy, dx) img(y + dy, x + dx), w = g g^T, zero outside the image."""
    g = gaussian_taps()
    h, w = img.shape
    pad = np.zeros((h + 2 * RADIUS, w + 2 * RADIUS))
    pad[RADIUS:RADIUS + h, RADIUS:RADIUS + w] = img
    out = np.zeros((h, w))
    for dy in range(2 * RADIUS + 1):
        for dx in range(2 * RADIUS + 1):
            out += g[dy] * g[dx] * pad[dy:dy + h, dx:dx + w]
    return out


def ssim_terms(x: np.ndarray, y: np.ndarray):
    """SSIM map of one channel and the pieces of its gradient."""
    mx, my = window_sum(x), window_sum(y)
    exx, eyy, exy = window_sum(x * x), window_sum(y * y), window_sum(x * y)
    a1 = 2 * mx * my + C1
    a2 = 2 * (exy - mx * my) + C2
    b1 = mx * mx + my * my + C1
    b2 = (exx - mx * mx) + (eyy - my * my) + C2
    s = a1 * a2 / (b1 * b2)
    # partials of s w.r.t. the window moments of x (mu_x, e_xx, e_xy), the others held fixed
    s_mu = (2 * my * (a2 - a1) - 2 * mx * s * (b2 - b1)) / (b1 * b2)
    s_xx = -s / b2
    s_xy = 2 * a1 / (b1 * b2)
    return s, s_mu, s_xx, s_xy


def ssim_map(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    return ssim_terms(x, y)[0]


def loss_l1_dssim(images: list, targets: list, lam: float = 0.2):
    """(L, [dL/dimage per view]) for images/targets given as [3, H, W] arrays."""
    count = sum(im.size for im in images)
    total = 0.0
    grads = []
    for im, tg in zip(images, targets):
        im = np.asarray(im, dtype=np.float64)
        tg = np.asarray(tg, dtype=np.float64)
        g = np.zeros_like(im)
        for ch in range(im.shape[0]):
            x, y = im[ch], tg[ch]
            s, s_mu, s_xx, s_xy = ssim_terms(x, y)
            total += np.sum((1 - lam) * np.abs(x - y) + lam * (1 - s))
            # d sum(s)/dx(p) = sum_q w(q - p) [s_mu(q) + 2 x(p) s_xx(q) + y(p) s_xy(q)]  (w symmetric)
            dssim = window_sum(s_mu) + 2 * x * window_sum(s_xx) + y * window_sum(s_xy)
            g[ch] = ((1 - lam) * np.sign(x - y) - lam * dssim) / count
        grads.append(g)
    return total / count, grads


def adam_step(p, m, v, g, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-15):
    """One Adam step at step number t (1-based); returns new (p, m, v)."""
    p, m, v, g = (np.asarray(a, dtype=np.float64) for a in (p, m, v, g))
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mhat = m / (1 - beta1 ** t)
    vhat = v / (1 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
