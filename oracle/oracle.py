"""ctypes wrapper around the FP64 CPU oracle in ``fgs4d_oracle.c``.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  The product path never does, and
this module imports nothing from the product package.

Every function takes the Gaussian parameters as a dict of numpy arrays in the
structure-of-arrays layout of the boundary (``mu``/``log_s``/``ql``/``qr`` are
``[4, N]``, ``logit`` is ``[N]``, ``shs`` is ``[3*(L+1)^2*(K+1), N]`` with row
``(f*(L+1)^2 + j)*3 + ch``), plus ``sh_degree``, ``n_freq`` and ``period``.
Values are converted to float64 before the call.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fgs4d_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfgs4d_oracle.so")
_lock = threading.Lock()
_lib = None

DEFAULT_OPTIONS = dict(p_min=0.05, near_z=0.2, alpha_min=1.0 / 255.0, alpha_max=0.99,
                       T_min=1e-4, dilation=0.3, clamp_fov=1.3)


def build(force: bool = False) -> str:
    """Compiles the oracle with gcc (plain -O2, IEEE semantics, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Gaussians(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("sh_degree", ctypes.c_int), ("n_freq", ctypes.c_int),
                ("period", ctypes.c_double),
                ("mu", ctypes.c_void_p), ("log_s", ctypes.c_void_p), ("ql", ctypes.c_void_p),
                ("qr", ctypes.c_void_p), ("logit", ctypes.c_void_p), ("shs", ctypes.c_void_p)]


class _View(ctypes.Structure):
    _fields_ = [("viewmat", ctypes.c_double * 12), ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("width", ctypes.c_int),
                ("height", ctypes.c_int), ("t", ctypes.c_double), ("bg", ctypes.c_double * 3)]


class _Options(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in
                ("p_min", "near_z", "alpha_min", "alpha_max", "T_min", "dilation", "clamp_fov")]


class Splat(ctypes.Structure):
    _fields_ = [("visible", ctypes.c_int), ("cull", ctypes.c_int), ("borderline", ctypes.c_int),
                ("p_t", ctypes.c_double), ("mu3", ctypes.c_double * 3), ("Sigma3", ctypes.c_double * 9),
                ("xc", ctypes.c_double * 3), ("u", ctypes.c_double), ("v", ctypes.c_double),
                ("depth", ctypes.c_double), ("cov2d", ctypes.c_double * 3), ("conic", ctypes.c_double * 3),
                ("alpha", ctypes.c_double), ("alpha_eff", ctypes.c_double), ("color", ctypes.c_double * 3),
                ("color_raw", ctypes.c_double * 3), ("radius", ctypes.c_double)]


class _Grads(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in ("mu", "log_s", "ql", "qr", "logit", "shs")]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            L.orc_quat_left.argtypes = [dp, dp]
            L.orc_quat_right.argtypes = [dp, dp]
            L.orc_rotation4.argtypes = [dp, dp, dp]
            L.orc_covariance4.argtypes = [dp, dp, dp, dp]
            L.orc_condition.argtypes = [dp, dp, ctypes.c_double, dp, dp, dp]
            L.orc_sh_basis.argtypes = [ctypes.c_int, dp, dp, ctypes.c_void_p]
            L.orc_project.argtypes = [ctypes.POINTER(_Gaussians), ctypes.c_int64, ctypes.POINTER(_View),
                                      ctypes.POINTER(_Options), ctypes.POINTER(Splat)]
            L.orc_project.restype = ctypes.c_int
            L.orc_render.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_View), ctypes.POINTER(_Options),
                                     ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_render.restype = ctypes.c_int64
            L.orc_render_values.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_View),
                                            ctypes.POINTER(_Options), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
            L.orc_project_backward.argtypes = [ctypes.POINTER(_Gaussians), ctypes.c_int64, ctypes.POINTER(_View),
                                               ctypes.POINTER(_Options), dp, ctypes.POINTER(_Grads)]
            L.orc_backward.argtypes = [ctypes.POINTER(_Gaussians), ctypes.POINTER(_View), ctypes.POINTER(_Options),
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_void_p, ctypes.POINTER(_Grads), ctypes.c_void_p]
            L.orc_splat_size.restype = ctypes.c_int
            assert L.orc_splat_size() == ctypes.sizeof(Splat), "oracle splat struct mismatch"
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class _Packed:
    """Keeps the float64 copies alive while the C structure points at them."""

    def __init__(self, params: dict):
        self.arrays = {k: _f64(params[k]) for k in ("mu", "log_s", "ql", "qr", "logit", "shs")}
        n = self.arrays["logit"].shape[0]
        L, K = int(params["sh_degree"]), int(params["n_freq"])
        assert self.arrays["shs"].shape == (3 * (L + 1) ** 2 * (K + 1), n), "shs layout mismatch"
        for k in ("mu", "log_s", "ql", "qr"):
            assert self.arrays[k].shape == (4, n), f"{k} must be [4, N]"
        self.struct = _Gaussians(n, L, K, float(params.get("period", 1.0)),
                                 *[self.arrays[k].ctypes.data for k in ("mu", "log_s", "ql", "qr", "logit", "shs")])
        self.n = n


def _view(view: dict) -> _View:
    v = _View()
    vm = np.asarray(view["viewmat"], dtype=np.float64).reshape(12)
    for i in range(12):
        v.viewmat[i] = vm[i]
    v.fx, v.fy, v.cx, v.cy = (float(view[k]) for k in ("fx", "fy", "cx", "cy"))
    v.width, v.height = int(view["width"]), int(view["height"])
    v.t = float(view["t"])
    bg = view.get("bg", (0.0, 0.0, 0.0))
    for i in range(3):
        v.bg[i] = float(bg[i])
    return v


def _options(opts: dict | None) -> _Options:
    o = dict(DEFAULT_OPTIONS)
    if opts:
        o.update({k: v for k, v in opts.items() if k in DEFAULT_OPTIONS})
    return _Options(*[float(o[k]) for k in ("p_min", "near_z", "alpha_min", "alpha_max", "T_min",
                                             "dilation", "clamp_fov")])


# ---------------------------------------------------------------- small steps
def quat_left(q) -> np.ndarray:
    out = np.zeros(16)
    lib().orc_quat_left(_dp(_f64(q)), _dp(out))
    return out.reshape(4, 4)


def quat_right(q) -> np.ndarray:
    out = np.zeros(16)
    lib().orc_quat_right(_dp(_f64(q)), _dp(out))
    return out.reshape(4, 4)


def rotation4(ql, qr) -> np.ndarray:
    out = np.zeros(16)
    lib().orc_rotation4(_dp(_f64(ql)), _dp(_f64(qr)), _dp(out))
    return out.reshape(4, 4)


def covariance4(log_s, ql, qr) -> np.ndarray:
    out = np.zeros(16)
    lib().orc_covariance4(_dp(_f64(log_s)), _dp(_f64(ql)), _dp(_f64(qr)), _dp(out))
    return out.reshape(4, 4)


def condition(mu, Sigma, t):
    mu3, S3, p = np.zeros(3), np.zeros(9), np.zeros(1)
    lib().orc_condition(_dp(_f64(mu)), _dp(_f64(Sigma).reshape(16)), float(t), _dp(mu3), _dp(S3), _dp(p))
    return mu3, S3.reshape(3, 3), float(p[0])


def sh_basis(L: int, d, with_grad: bool = False):
    nb = (L + 1) ** 2
    Y = np.zeros(nb)
    dY = np.zeros(3 * nb) if with_grad else None
    lib().orc_sh_basis(int(L), _dp(_f64(d)), _dp(Y), dY.ctypes.data if with_grad else None)
    return (Y, dY.reshape(nb, 3)) if with_grad else Y


def project(params: dict, g: int, view: dict, opts: dict | None = None) -> Splat:
    P = _Packed(params)
    s = Splat()
    lib().orc_project(ctypes.byref(P.struct), int(g), ctypes.byref(_view(view)), ctypes.byref(_options(opts)),
                      ctypes.byref(s))
    return s


def project_all(params: dict, view: dict, opts: dict | None = None) -> dict:
    """Per-Gaussian slice/projection records as numpy arrays (visible, u, v, ...)."""
    P = _Packed(params)
    n = P.n
    S = (Splat * max(n, 1))()
    img = np.zeros((3, 1, 1))
    lib().orc_render(ctypes.byref(P.struct), ctypes.byref(_view(view)), ctypes.byref(_options(opts)), 0, 0, 1, 1, 1,
                     img.ctypes.data, None, None, None, ctypes.cast(S, ctypes.c_void_p), None, None)
    out = {}
    for name, _ in Splat._fields_:
        vals = [getattr(S[i], name) for i in range(n)]
        if isinstance(vals[0] if n else 0, (int, float)):
            out[name] = np.array(vals)
        else:
            out[name] = np.array([list(v) for v in vals]) if n else np.zeros((0,))
    return out


# ---------------------------------------------------------------- render / backward
def _window(view, window):
    if window is None:
        return 0, 0, int(view["width"]), int(view["height"])
    x0, y0, w, h = window
    return int(x0), int(y0), int(w), int(h)


def render(params: dict, view: dict, opts: dict | None = None, window=None, prefilter: bool = False) -> dict:
    """Eq. 6 per pixel over all splats.  Returns image [3,h,w], T [h,w],
    n_contrib [h,w], flags [h,w] (bit 0: image borderline, bit 1: gradient
    borderline; bits 2..5: cause of bit 0 -- depth near-tie, early stop,
    alpha_min skip, Gaussian-level cull), seq_hash [h,w] (order-sensitive
    hash of the contributor sequence), amb_image / amb_T [h,w] (how far a
    valid single-precision evaluation may land from this result because of
    the flagged decisions) and the number of visible splats."""
    P = _Packed(params)
    x0, y0, w, h = _window(view, window)
    img = np.zeros((3, h, w))
    T = np.zeros((h, w))
    nc = np.zeros((h, w), dtype=np.int32)
    fl = np.zeros((h, w), dtype=np.uint8)
    sh = np.zeros((h, w), dtype=np.uint64)
    amb = np.zeros((2, h, w))
    nvis = lib().orc_render(ctypes.byref(P.struct), ctypes.byref(_view(view)), ctypes.byref(_options(opts)),
                            x0, y0, w, h, int(bool(prefilter)), img.ctypes.data, T.ctypes.data, nc.ctypes.data,
                            fl.ctypes.data, None, sh.ctypes.data, amb.ctypes.data)
    return dict(image=img, T=T, n_contrib=nc, flags=fl, seq_hash=sh, amb_image=amb[0], amb_T=amb[1],
                n_visible=int(nvis))


def render_values(params: dict, view: dict, values: np.ndarray, opts: dict | None = None, window=None,
                  prefilter: bool = False) -> np.ndarray:
    """Eq. 6 compositing of per-Gaussian values [n, 3] (in place of the
    colours, background 0) with the image's walk: [3, h, w]."""
    P = _Packed(params)
    x0, y0, w, h = _window(view, window)
    vals = np.ascontiguousarray(np.asarray(values, dtype=np.float64).reshape(P.n, 3))
    out = np.zeros((3, h, w))
    lib().orc_render_values(ctypes.byref(P.struct), ctypes.byref(_view(view)), ctypes.byref(_options(opts)), x0, y0,
                            w, h, int(bool(prefilter)), vals.ctypes.data, out.ctypes.data)
    return out


def aux_values(params: dict, view: dict, flow_dt: float, opts: dict | None = None) -> np.ndarray:
    """Per-Gaussian [n, 3]: the camera depth of mu_{xyz|t}, and the
    displacement (du, dv) of its projection from t to t + flow_dt, with the
    conditional mean of Eq. 9 at t + flow_dt (0 where that mean is behind the
    camera)."""
    rec = project_all(params, view, opts)
    n = len(rec["u"])
    Vm = np.asarray(view["viewmat"], dtype=np.float64).reshape(3, 4)
    W, tau = Vm[:, :3], Vm[:, 3]
    out = np.zeros((n, 3))
    for g in range(n):
        out[g, 0] = rec["depth"][g]
        Sigma = covariance4(params["log_s"][:, g], params["ql"][:, g], params["qr"][:, g])
        mu3, _, _ = condition(params["mu"][:, g], Sigma, float(view["t"]) + flow_dt)
        xc = W @ mu3 + tau
        if xc[2] > 0:
            out[g, 1] = view["fx"] * xc[0] / xc[2] + view["cx"] - rec["u"][g]
            out[g, 2] = view["fy"] * xc[1] / xc[2] + view["cy"] - rec["v"][g]
    return out


def _new_grads(P: _Packed):
    g = {k: np.zeros_like(P.arrays[k]) for k in ("mu", "log_s", "ql", "qr", "logit", "shs")}
    s = _Grads(*[g[k].ctypes.data for k in ("mu", "log_s", "ql", "qr", "logit", "shs")])
    return g, s


def backward(params: dict, view: dict, dL_dimage: np.ndarray, opts: dict | None = None, window=None,
             prefilter: bool = False) -> dict:
    """Gradient of sum(dL_dimage * image) w.r.t. the raw parameters, plus the
    per-Gaussian 2D splat gradient ``grad2d`` [N, 9] (u, v, a, b, c, alpha_eff, rgb)."""
    P = _Packed(params)
    x0, y0, w, h = _window(view, window)
    dLd = _f64(dL_dimage).reshape(3, h, w)
    g, s = _new_grads(P)
    g2 = np.zeros((P.n, 9))
    lib().orc_backward(ctypes.byref(P.struct), ctypes.byref(_view(view)), ctypes.byref(_options(opts)), x0, y0, w, h,
                       int(bool(prefilter)), dLd.ctypes.data, ctypes.byref(s), g2.ctypes.data)
    g["grad2d"] = g2
    return g


def project_backward(params: dict, g: int, view: dict, g2d, opts: dict | None = None) -> dict:
    P = _Packed(params)
    grads, s = _new_grads(P)
    lib().orc_project_backward(ctypes.byref(P.struct), int(g), ctypes.byref(_view(view)),
                               ctypes.byref(_options(opts)), _dp(_f64(g2d)), ctypes.byref(s))
    return grads


def render_views(params: dict, views: list, opts: dict | None = None, prefilter: bool = False) -> list:
    return [render(params, v, opts, prefilter=prefilter) for v in views]


def backward_views(params: dict, views: list, dL_dimages: list, opts: dict | None = None,
                   prefilter: bool = False) -> dict:
    total = None
    for v, d in zip(views, dL_dimages):
        g = backward(params, v, d, opts, prefilter=prefilter)
        g.pop("grad2d")
        if total is None:
            total = g
        else:
            for k in total:
                total[k] += g[k]
    return total
