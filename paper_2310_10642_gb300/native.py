"""ctypes binding of libfgs4d (include/fgs4d.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: all of it runs in the CUDA kernels of ``csrc/``.
If the library has not been built, or cannot be loaded, ``lib()`` raises:
there is no CPU fallback.

``build()`` compiles the library in-tree with nvcc for sm_103a.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_INCLUDE = os.path.join(os.path.dirname(_HERE), "include")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libfgs4d.so")
SOURCES = ["api.cu", "slice_project.cu", "bin_sort.cu", "render.cu", "train.cu"]
HEADERS = ["fgs4d_internal.cuh"]
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]

MAX_VIEWS = 128
TILE = 16
F32, BF16 = 0, 1
ROT_4D, ROT_SPATIAL, ROT_STATIC = 0, 1, 2
STATUS_PAIR_OVERFLOW = 1
STATUS_NONFINITE = 2

_lock = threading.Lock()
_lib = None


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(out: str, deps: list) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles csrc/*.cu for sm_103a into _build/libfgs4d.so (parallel, in-tree)."""
    os.makedirs(_BUILD, exist_ok=True)
    hdrs = [os.path.join(_CSRC, h) for h in HEADERS] + [os.path.join(_INCLUDE, "fgs4d.h")]
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(_CSRC, src)
        o = os.path.join(_BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            jobs.append([_nvcc(), *ARCH_FLAGS, *NVCC_FLAGS, "-I", _INCLUDE, "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return r.stderr

    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            list(ex.map(run, jobs))
    if force or _stale(LIB_PATH, objs):
        tmp = LIB_PATH + f".{os.getpid()}.tmp"
        run([_nvcc(), *ARCH_FLAGS, "-shared", "-o", tmp, *objs])
        os.replace(tmp, LIB_PATH)
    return LIB_PATH


# ---------------------------------------------------------------- C structures
class Gaussians(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_void_p), ("log_scale", ctypes.c_void_p), ("q_left", ctypes.c_void_p),
                ("q_right", ctypes.c_void_p), ("opacity_logit", ctypes.c_void_p), ("shs", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("sh_degree", ctypes.c_int), ("n_freq", ctypes.c_int),
                ("period", ctypes.c_float), ("shs_dtype", ctypes.c_int), ("rotation", ctypes.c_int)]


class View(ctypes.Structure):
    _fields_ = [("viewmat", ctypes.c_float * 12), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("t", ctypes.c_float), ("bg", ctypes.c_float * 3)]


class Options(ctypes.Structure):
    _fields_ = [("p_min", ctypes.c_float), ("near_z", ctypes.c_float), ("alpha_min", ctypes.c_float),
                ("alpha_max", ctypes.c_float), ("T_min", ctypes.c_float), ("dilation", ctypes.c_float),
                ("clamp_fov", ctypes.c_float), ("record_fp16", ctypes.c_int), ("schur_cond", ctypes.c_float),
                ("conic_cond", ctypes.c_float), ("tile_size", ctypes.c_int), ("batch_depth", ctypes.c_int),
                ("aux_channels", ctypes.c_int), ("flow_dt", ctypes.c_float), ("bin_size", ctypes.c_int),
                ("accumulate_grads", ctypes.c_int)]


class GaussianGrads(ctypes.Structure):
    _fields_ = [("mu", ctypes.c_void_p), ("log_scale", ctypes.c_void_p), ("q_left", ctypes.c_void_p),
                ("q_right", ctypes.c_void_p), ("opacity_logit", ctypes.c_void_p), ("shs", ctypes.c_void_p),
                ("mean2d_abs", ctypes.c_void_p), ("mu_t_abs", ctypes.c_void_p)]


class Counters(ctypes.Structure):
    _fields_ = [("n_visible", ctypes.c_uint32), ("n_pairs", ctypes.c_uint32), ("status", ctypes.c_uint32),
                ("pair_capacity", ctypes.c_uint32)]


class AdamGroup(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("exp_avg", ctypes.c_void_p), ("exp_avg_sq", ctypes.c_void_p),
                ("grad", ctypes.c_void_p), ("param_bf16", ctypes.c_void_p), ("count", ctypes.c_int64),
                ("lr_index", ctypes.c_int)]


class StateLayoutInfo(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("counters", "records", "tiles_touched", "ranges", "pair_vals",
                                                "record_bytes", "n_splats", "total_tiles", "pair_capacity",
                                                "grad2d")]


EXPORTS = ["fgs4d_abi_version", "fgs4d_launch_count", "fgs4d_status_string", "fgs4d_default_options", "fgs4d_state_size",
           "fgs4d_total_pixels", "fgs4d_slice_project", "fgs4d_bin_sort", "fgs4d_render", "fgs4d_render_backward",
           "fgs4d_state_layout", "fgs4d_read_counters", "fgs4d_render_backward_noalloc", "fgs4d_render_stats",
           "fgs4d_render_backward_2d", "fgs4d_project_backward",
           "fgs4d_loss_scratch_size", "fgs4d_loss_l1_dssim", "fgs4d_adam_step", "fgs4d_sample_split",
           "fgs4d_render_aux"]
NOALLOC_MAX_SPLATS = 262144


class Fgs4dError(RuntimeError):
    def __init__(self, fn: str, code: int):
        msg = lib().fgs4d_status_string(code).decode() if _lib is not None else str(code)
        super().__init__(f"{fn} failed: {msg} (status {code})")
        self.code = code


def lib(path: str | None = None) -> ctypes.CDLL:
    """Loads libfgs4d.so (raises if it is missing: no fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise RuntimeError(f"libfgs4d is not built ({p}); run paper_2310_10642_gb300.native.build()")
            L = ctypes.CDLL(p)
            vp, i64, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
            L.fgs4d_abi_version.restype = ci
            L.fgs4d_launch_count.restype = ctypes.c_uint64
            L.fgs4d_status_string.argtypes = [ci]
            L.fgs4d_status_string.restype = ctypes.c_char_p
            L.fgs4d_default_options.argtypes = [ctypes.POINTER(Options)]
            L.fgs4d_state_size.argtypes = [i64, ctypes.POINTER(View), ci, i64, ctypes.POINTER(Options),
                                           ctypes.POINTER(ctypes.c_size_t)]
            L.fgs4d_total_pixels.argtypes = [ctypes.POINTER(View), ci]
            L.fgs4d_total_pixels.restype = i64
            L.fgs4d_slice_project.argtypes = [ctypes.POINTER(Gaussians), ctypes.POINTER(View), ci,
                                              ctypes.POINTER(Options), vp, ctypes.c_size_t, vp]
            L.fgs4d_bin_sort.argtypes = [i64, ctypes.POINTER(View), ci, ctypes.POINTER(Options), vp, ctypes.c_size_t,
                                         vp]
            L.fgs4d_render.argtypes = [i64, ctypes.POINTER(View), ci, ctypes.POINTER(Options), vp, ctypes.c_size_t,
                                       vp, vp, vp, vp]
            L.fgs4d_render_backward.argtypes = [ctypes.POINTER(Gaussians), ctypes.POINTER(View), ci,
                                                ctypes.POINTER(Options), vp, ctypes.c_size_t, vp, vp, vp,
                                                ctypes.POINTER(GaussianGrads), vp]
            L.fgs4d_render_stats.argtypes = [i64, ctypes.POINTER(View), ci, ctypes.POINTER(Options), vp,
                                             ctypes.c_size_t, vp, vp, vp, vp, vp]
            L.fgs4d_render_stats.restype = ci
            L.fgs4d_render_backward_2d.argtypes = [i64, ctypes.POINTER(View), ci, ctypes.POINTER(Options), vp,
                                                   ctypes.c_size_t, vp, vp, vp, vp]
            L.fgs4d_project_backward.argtypes = [ctypes.POINTER(Gaussians), ctypes.POINTER(View), ci,
                                                 ctypes.POINTER(Options), vp, ctypes.c_size_t,
                                                 ctypes.POINTER(GaussianGrads), vp]
            L.fgs4d_read_counters.argtypes = [vp, ctypes.POINTER(Counters), vp]
            L.fgs4d_render_aux.argtypes = [i64, ctypes.POINTER(View), ci, ctypes.POINTER(Options), vp,
                                           ctypes.c_size_t, vp, vp]
            L.fgs4d_render_aux.restype = ci
            L.fgs4d_sample_split.argtypes = [ctypes.POINTER(Gaussians), vp, vp, i64, vp, vp]
            L.fgs4d_sample_split.restype = ci
            L.fgs4d_loss_scratch_size.argtypes = [ctypes.POINTER(View), ci]
            L.fgs4d_loss_scratch_size.restype = ctypes.c_size_t
            L.fgs4d_loss_l1_dssim.argtypes = [ctypes.POINTER(View), ci, vp, vp, ctypes.c_float, vp, vp, vp,
                                              ctypes.c_size_t, vp]
            L.fgs4d_loss_l1_dssim.restype = ci
            L.fgs4d_adam_step.argtypes = [ctypes.POINTER(AdamGroup), ci, vp, ctypes.c_float, ctypes.c_float,
                                          ctypes.c_float, vp, vp, vp]
            L.fgs4d_adam_step.restype = ci
            L.fgs4d_render_backward_noalloc.argtypes = L.fgs4d_render_backward.argtypes
            L.fgs4d_render_backward_noalloc.restype = ci
            L.fgs4d_state_layout.argtypes = [i64, ctypes.POINTER(View), ci, ctypes.POINTER(Options), ctypes.c_size_t,
                                             ctypes.POINTER(StateLayoutInfo)]
            for fn in ("fgs4d_state_size", "fgs4d_slice_project", "fgs4d_bin_sort", "fgs4d_render",
                       "fgs4d_render_backward", "fgs4d_read_counters", "fgs4d_state_layout",
                       "fgs4d_render_backward_2d", "fgs4d_project_backward"):
                getattr(L, fn).restype = ci
            assert L.fgs4d_abi_version() == 5, "libfgs4d ABI version mismatch"
            _lib = L
    return _lib


def _check(fn: str, code: int):
    if code != 0:
        raise Fgs4dError(fn, code)


# ---------------------------------------------------------------- marshalling
def make_views(views: list) -> ctypes.Array:
    arr = (View * len(views))()
    for i, v in enumerate(views):
        vm = [float(x) for x in list(v["viewmat"])]
        for k in range(12):
            arr[i].viewmat[k] = vm[k]
        arr[i].fx, arr[i].fy, arr[i].cx, arr[i].cy = (float(v[k]) for k in ("fx", "fy", "cx", "cy"))
        arr[i].width, arr[i].height = int(v["width"]), int(v["height"])
        arr[i].t = float(v["t"])
        bg = v.get("bg", (0.0, 0.0, 0.0))
        for k in range(3):
            arr[i].bg[k] = float(bg[k])
    return arr


def make_options(opts: dict | None = None) -> Options:
    o = Options()
    lib().fgs4d_default_options(ctypes.byref(o))
    for k, val in (opts or {}).items():
        if hasattr(o, k) and k in dict(Options._fields_):
            setattr(o, k, type(getattr(o, k))(val))
    return o


def fgs4d_default_options() -> Options:
    return make_options(None)


def fgs4d_state_size(n: int, views, n_views: int, pair_capacity: int, opts: Options) -> int:
    out = ctypes.c_size_t(0)
    _check("fgs4d_state_size", lib().fgs4d_state_size(int(n), views, int(n_views), int(pair_capacity),
                                                       ctypes.byref(opts), ctypes.byref(out)))
    return int(out.value)


def fgs4d_total_pixels(views, n_views: int) -> int:
    return int(lib().fgs4d_total_pixels(views, int(n_views)))


def fgs4d_slice_project(g: Gaussians, views, n_views: int, opts: Options, state: int, state_bytes: int, stream: int):
    _check("fgs4d_slice_project", lib().fgs4d_slice_project(ctypes.byref(g), views, int(n_views), ctypes.byref(opts),
                                                             state, state_bytes, stream))


def fgs4d_bin_sort(n: int, views, n_views: int, opts: Options, state: int, state_bytes: int, stream: int):
    _check("fgs4d_bin_sort", lib().fgs4d_bin_sort(int(n), views, int(n_views), ctypes.byref(opts), state,
                                                   state_bytes, stream))


def fgs4d_render(n: int, views, n_views: int, opts: Options, state: int, state_bytes: int, image: int,
                 final_T: int, n_last: int, stream: int):
    _check("fgs4d_render", lib().fgs4d_render(int(n), views, int(n_views), ctypes.byref(opts), state, state_bytes,
                                               image, final_T, n_last, stream))


def fgs4d_render_backward_2d(n: int, views, n_views: int, opts: Options, state: int, state_bytes: int,
                             final_T: int, n_last: int, dL_dimage: int, stream: int):
    _check("fgs4d_render_backward_2d", lib().fgs4d_render_backward_2d(int(n), views, int(n_views), ctypes.byref(opts),
                                                                       state, state_bytes, final_T, n_last, dL_dimage,
                                                                       stream))


def fgs4d_project_backward(g: Gaussians, views, n_views: int, opts: Options, state: int, state_bytes: int,
                           grads: GaussianGrads, stream: int):
    _check("fgs4d_project_backward", lib().fgs4d_project_backward(ctypes.byref(g), views, int(n_views),
                                                                   ctypes.byref(opts), state, state_bytes,
                                                                   ctypes.byref(grads), stream))


def fgs4d_render_aux(n: int, views, n_views: int, opts: Options, state: int, state_bytes: int, aux_image: int,
                     stream: int):
    _check("fgs4d_render_aux", lib().fgs4d_render_aux(int(n), views, int(n_views), ctypes.byref(opts), state,
                                                       state_bytes, aux_image, stream))


def fgs4d_sample_split(g: Gaussians, index: int, z: int, m: int, out_mu: int, stream: int):
    _check("fgs4d_sample_split", lib().fgs4d_sample_split(ctypes.byref(g), index, z, int(m), out_mu, stream))


def fgs4d_loss_scratch_size(views, n_views: int) -> int:
    return int(lib().fgs4d_loss_scratch_size(views, int(n_views)))


def fgs4d_loss_l1_dssim(views, n_views: int, image: int, target: int, lam: float, loss: int, dL_dimage: int,
                        scratch: int, scratch_bytes: int, stream: int):
    _check("fgs4d_loss_l1_dssim", lib().fgs4d_loss_l1_dssim(views, int(n_views), image, target, float(lam), loss,
                                                             dL_dimage, scratch, scratch_bytes, stream))


def fgs4d_adam_step(groups: list, lrs: int, beta1: float, beta2: float, eps: float, step: int, bias: int,
                    stream: int):
    arr = (AdamGroup * len(groups))(*groups)
    _check("fgs4d_adam_step", lib().fgs4d_adam_step(arr, len(groups), lrs, float(beta1), float(beta2), float(eps),
                                                     step, bias, stream))


def fgs4d_render_stats(n: int, views, n_views: int, opts: Options, state: int, state_bytes: int, image: int,
                       final_T: int, n_last: int, stats: int, stream: int):
    _check("fgs4d_render_stats", lib().fgs4d_render_stats(int(n), views, int(n_views), ctypes.byref(opts), state,
                                                           state_bytes, image, final_T, n_last, stats, stream))


def fgs4d_render_backward(g: Gaussians, views, n_views: int, opts: Options, state: int, state_bytes: int,
                          final_T: int, n_last: int, dL_dimage: int, grads: GaussianGrads, stream: int):
    _check("fgs4d_render_backward", lib().fgs4d_render_backward(ctypes.byref(g), views, int(n_views),
                                                                 ctypes.byref(opts), state, state_bytes, final_T,
                                                                 n_last, dL_dimage, ctypes.byref(grads), stream))


def fgs4d_read_counters(state: int, stream: int) -> Counters:
    c = Counters()
    _check("fgs4d_read_counters", lib().fgs4d_read_counters(state, ctypes.byref(c), stream))
    return c


def fgs4d_state_layout(n: int, views, n_views: int, opts: Options, state_bytes: int) -> StateLayoutInfo:
    out = StateLayoutInfo()
    _check("fgs4d_state_layout", lib().fgs4d_state_layout(int(n), views, int(n_views), ctypes.byref(opts),
                                                           int(state_bytes), ctypes.byref(out)))
    return out


def fgs4d_launch_count() -> int:
    return int(lib().fgs4d_launch_count())


def fgs4d_render_backward_noalloc(g: Gaussians, views, n_views: int, opts: Options, state: int, state_bytes: int,
                                  final_T: int, n_last: int, dL_dimage: int, grads: GaussianGrads, stream: int):
    """Backward pass whose scratch lives in the library's static device array
    (at most NOALLOC_MAX_SPLATS (view, Gaussian) splats); allocates nothing."""
    _check("fgs4d_render_backward_noalloc",
           lib().fgs4d_render_backward_noalloc(ctypes.byref(g), views, int(n_views), ctypes.byref(opts), state,
                                               state_bytes, final_T, n_last, dL_dimage, ctypes.byref(grads), stream))
