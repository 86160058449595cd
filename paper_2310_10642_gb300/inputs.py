"""Seeded synthetic inputs: 4D Gaussian parameters and pinhole cameras.

This module only draws random numbers and builds cameras.  It contains none of
the rendering arithmetic, so the CUDA path and the CPU oracle can both be fed
from it without sharing any of the method.  Every draw uses numpy's Philox
counter-based generator, seeded per workload.

Parameter layout (structure of arrays, float32):
  mu     [4, N]   (x, y, z, t)
  log_s  [4, N]   log of (s_x, s_y, s_z, s_t)
  ql     [4, N]   left quaternion (a, b, c, d), unnormalised
  qr     [4, N]   right quaternion (p, q, r, s), unnormalised
  logit  [N]      opacity logit
  shs    [3*(L+1)^2*(K+1), N]  4D spherindrical coefficients, row
                  (f*(L+1)^2 + j)*3 + ch for Fourier order f, SH index
                  j = l^2 + l + m and colour channel ch

Workload shapes follow the paper's settings: D-NeRF style clouds of 100k
points in a cube, Plenoptic-Video-like 1352x1014 frames over 300 timestamps,
time scale initialised around the scene duration.  No dataset item is used.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 20231016


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def n_coef(sh_degree: int, n_freq: int) -> int:
    return (sh_degree + 1) ** 2 * (n_freq + 1)


def gaussians(n: int, seed: int, sh_degree: int, n_freq: int, period: float = 1.0, clustered: bool = False,
              n_blobs: int = 64, blob_sigma: float = 0.1, cluster_frac: float = 0.7,
              log_s_xyz=(-3.0, 0.5), log_s_t=(-2.0, 0.5), sh_sigma: float = 0.2) -> dict:
    """Draws N Gaussians: means uniform in [-1,1]^3 x [0,1] (or 70% from
    n_blobs spatial blobs), log scales normal, quaternions normal in R^4
    (uniform on S^3 after normalisation), logit N(0,1), coefficients N(0, sh_sigma)."""
    r = rng(seed)
    mu = np.empty((4, n), np.float32)
    if clustered:
        centres = r.uniform(-1.0, 1.0, size=(n_blobs, 3))
        n_cl = int(round(cluster_frac * n))
        which = r.integers(0, n_blobs, size=n_cl)
        pts = centres[which] + r.normal(0.0, blob_sigma, size=(n_cl, 3))
        uni = r.uniform(-1.0, 1.0, size=(n - n_cl, 3))
        xyz = np.concatenate([pts, uni], axis=0)
        xyz = xyz[r.permutation(n)]
        mu[:3] = xyz.T
    else:
        mu[:3] = r.uniform(-1.0, 1.0, size=(3, n))
    mu[3] = r.uniform(0.0, 1.0, size=n) * period
    log_s = np.empty((4, n), np.float32)
    log_s[:3] = r.normal(log_s_xyz[0], log_s_xyz[1], size=(3, n))
    log_s[3] = r.normal(log_s_t[0], log_s_t[1], size=n)
    ql = r.normal(size=(4, n)).astype(np.float32)
    qr = r.normal(size=(4, n)).astype(np.float32)
    logit = r.normal(size=n).astype(np.float32)
    shs = r.normal(0.0, sh_sigma, size=(3 * n_coef(sh_degree, n_freq), n)).astype(np.float32)
    return dict(mu=mu, log_s=log_s, ql=ql, qr=qr, logit=logit, shs=shs, sh_degree=int(sh_degree),
                n_freq=int(n_freq), period=float(period))


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World->camera [W | tau] (3x4, row-major) for an OpenCV camera:
    +x right, +y down, +z forward."""
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    right = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(right) < 1e-9:
        right = np.cross(f, np.array([0.0, 0.0, 1.0]))
    right /= np.linalg.norm(right)
    down = np.cross(f, right)
    W = np.stack([right, down, f])
    tau = -W @ eye
    return np.concatenate([W, tau[:, None]], axis=1)


def view(eye, width: int, height: int, t: float, fov_x_deg: float = 50.0, target=(0.0, 0.0, 0.0),
         bg=(0.0, 0.0, 0.0)) -> dict:
    """Pinhole camera with a horizontal field of view, square pixels and the
    principal point at the image centre ((W-1)/2, (H-1)/2)."""
    fx = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    return dict(viewmat=look_at(eye, target).reshape(12), fx=fx, fy=fx, cx=(width - 1) * 0.5,
                cy=(height - 1) * 0.5, width=int(width), height=int(height), t=float(t),
                bg=tuple(float(b) for b in bg))


def fibonacci_sphere(k: int, radius: float) -> np.ndarray:
    i = np.arange(k) + 0.5
    phi = np.arccos(1.0 - 2.0 * i / k)
    theta = math.pi * (1.0 + 5.0 ** 0.5) * i
    return radius * np.stack([np.cos(theta) * np.sin(phi), np.cos(phi), np.sin(theta) * np.sin(phi)], axis=1)


def arc_eyes(k: int, radius: float = 4.0, az_deg=(-30.0, 30.0), elev_deg: float = 10.0) -> np.ndarray:
    az = np.radians(np.linspace(az_deg[0], az_deg[1], k))
    el = math.radians(elev_deg)
    return radius * np.stack([np.sin(az) * math.cos(el), -np.full(k, math.sin(el)), np.cos(az) * math.cos(el)], axis=1)


DEFAULT_OPTIONS = dict(p_min=0.05, near_z=0.2, alpha_min=1.0 / 255.0, alpha_max=0.99, T_min=1e-4,
                       dilation=0.3, clamp_fov=1.3)


def config(k: int, n: int | None = None, n_views: int | None = None, scale: float = 1.0) -> dict:
    """Workload k of the benchmark ladder.  ``n`` and ``n_views`` shrink a
    workload for tests; ``scale`` shrinks image sizes (for tests only).

    0: 2,000 Gaussians, L=1, K=1, one 128x128 camera at distance 4, t = 0.5
    1: 100k Gaussians, L=3, K=2, 16 cameras on a sphere of radius 4, 800x800,
       t ~ U[0,1] per view
    2: 300k Gaussians, L=3, K=2, 300 frames; 20 arc cameras x 4 timestamps at
       1352x1014 plus 20 views at 676x507
    3: 1M clustered Gaussians, L=3, K=2; 20 arc cameras at 1352x1014, one
       window of timestamps out of 300 frames
    4: 3M clustered Gaussians, L=3, K=2; 4 views at 1352x1014 + 4 at 800x800
    """
    seed = SEED_BASE + k
    r = rng(seed + 1000)
    S = lambda w, h: (max(1, int(round(w * scale))), max(1, int(round(h * scale))))
    if k == 0:
        G = gaussians(n or 2000, seed, 1, 1)
        w, h = S(128, 128)
        views = [view((0.0, 0.0, 4.0), w, h, 0.5)]
    elif k == 1:
        G = gaussians(n or 100_000, seed, 3, 2)
        kv = n_views or 16
        eyes = fibonacci_sphere(16, 4.0)[:kv]
        ts = r.uniform(0.0, 1.0, size=16)[:kv]
        w, h = S(800, 800)
        views = [view(e, w, h, float(t)) for e, t in zip(eyes, ts)]
    elif k == 2:
        G = gaussians(n or 300_000, seed, 3, 2)
        eyes = arc_eyes(20)
        frames = np.arange(300) / 299.0
        tsel = frames[np.sort(r.choice(300, size=4, replace=False))]
        w1, h1 = S(1352, 1014)
        w2, h2 = S(676, 507)
        views = [view(e, w1, h1, float(t)) for t in tsel for e in eyes]
        views += [view(e, w2, h2, float(frames[r.integers(0, 300)])) for e in eyes]
        if n_views:
            views = views[:n_views]
    elif k == 3:
        G = gaussians(n or 1_000_000, seed, 3, 2, clustered=True)
        eyes = arc_eyes(20)
        frames = np.arange(300) / 299.0
        f0 = int(r.integers(0, 300))
        w, h = S(1352, 1014)
        views = [view(e, w, h, float(frames[(f0 + 15 * i) % 300])) for i, e in enumerate(eyes)]
        if n_views:
            views = views[:n_views]
    elif k == 4:
        G = gaussians(n or 3_000_000, seed, 3, 2, clustered=True)
        eyes = fibonacci_sphere(8, 4.0)
        ts = r.uniform(0.0, 1.0, size=8)
        w1, h1 = S(1352, 1014)
        w2, h2 = S(800, 800)
        views = [view(e, *(S(1352, 1014) if i < 4 else S(800, 800)), float(t))
                 for i, (e, t) in enumerate(zip(eyes, ts))]
        if n_views:
            views = views[:n_views]
    else:
        raise ValueError(f"unknown workload {k}")
    return dict(gaussians=G, views=views, options=dict(DEFAULT_OPTIONS))


def random_target(views: list, seed: int) -> list:
    """Seeded U[0,1] target images [3, H, W] for an L1 loss."""
    r = rng(seed)
    return [r.uniform(0.0, 1.0, size=(3, v["height"], v["width"])).astype(np.float32) for v in views]
