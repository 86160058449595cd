"""PyTorch front end of libfgs4d: device buffers, streams and autograd.

``Frame`` owns the per-frame state for one (number of Gaussians, views,
options) configuration and calls the four C entry points in order.  PyTorch
only allocates memory and supplies the stream; every step of the rendering
routine and of its adjoint runs in the CUDA kernels behind the C ABI.

``render(params, views)`` is the differentiable entry point: it returns the
list of [3, H, W] images and, through ``Render4DGS``, back-propagates into the
raw parameters (mu, log_s, ql, qr, logit, shs) with transmittance recomputed
in the backward kernels rather than stored per splat.
"""
from __future__ import annotations

import torch

from . import native as N

PARAM_KEYS = ("mu", "log_s", "ql", "qr", "logit", "shs")


def params_to_device(params: dict, device="cuda", shs_dtype=torch.float32) -> dict:
    """Copies numpy/torch parameters (the inputs-module layout) to the device."""
    out = {}
    for k in PARAM_KEYS:
        t = torch.as_tensor(params[k])
        dt = shs_dtype if k == "shs" else torch.float32
        out[k] = t.to(device=device, dtype=dt).contiguous()
    for k in ("sh_degree", "n_freq", "period"):
        out[k] = params[k]
    if "rotation" in params:
        out["rotation"] = int(params["rotation"])
    return out


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def gaussians_struct(p: dict) -> N.Gaussians:
    shs = p["shs"]
    if shs.dtype == torch.bfloat16:
        dtype = N.BF16
    elif shs.dtype == torch.float32:
        dtype = N.F32
    else:
        raise TypeError("shs must be float32 or bfloat16")
    for k in PARAM_KEYS:
        t = p[k]
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{k} must be a contiguous CUDA tensor")
    n = p["logit"].shape[0]
    return N.Gaussians(_ptr(p["mu"]), _ptr(p["log_s"]), _ptr(p["ql"]), _ptr(p["qr"]), _ptr(p["logit"]),
                       _ptr(p["shs"]), n, int(p["sh_degree"]), int(p["n_freq"]), float(p.get("period", 1.0)), dtype,
                       int(p.get("rotation", N.ROT_4D)))


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Frame:
    """State and output buffers for rendering ``n`` Gaussians into ``views``.

    pair_capacity: room for (splat, tile) pairs; ``None`` picks an estimate
    and ``forward(check=True)`` grows it when the device reports overflow.
    """

    def __init__(self, n: int, views: list, options: dict | None = None, pair_capacity: int | None = None,
                 device="cuda", outputs: tuple | None = None):
        """outputs: optional (image, final_T, n_last) device tensors of the
        packed sizes to render into (e.g. views of a larger packed buffer)."""
        if len(views) < 1 or len(views) > N.MAX_VIEWS:
            raise ValueError(f"1..{N.MAX_VIEWS} views per frame")
        self.n = int(n)
        self.views = list(views)
        self.nv = len(views)
        self.device = torch.device(device)
        self.c_views = N.make_views(self.views)
        self.c_opts = N.make_options(options)
        self.total_pixels = N.fgs4d_total_pixels(self.c_views, self.nv)
        self.pix_offsets = []
        off = 0
        for v in self.views:
            self.pix_offsets.append(off)
            off += int(v["width"]) * int(v["height"])
        if pair_capacity is None:
            tiles = sum(((int(v["width"]) + 15) // 16) * ((int(v["height"]) + 15) // 16) for v in self.views)
            pair_capacity = max(1 << 16, min(self.n * self.nv * 8, tiles * 4096))
        if outputs is not None:
            self.image, self.final_T, self.n_last = outputs
            if (self.image.numel() != 3 * self.total_pixels or self.final_T.numel() != self.total_pixels
                    or self.n_last.numel() != self.total_pixels or self.n_last.dtype != torch.int32):
                raise ValueError("outputs do not match the views' packed sizes")
        else:
            self.image = torch.empty(3 * self.total_pixels, device=self.device, dtype=torch.float32)
            self.final_T = torch.empty(self.total_pixels, device=self.device, dtype=torch.float32)
            self.n_last = torch.empty(self.total_pixels, device=self.device, dtype=torch.int32)
        self._alloc(int(pair_capacity))

    def _alloc(self, cap: int):
        self.pair_capacity = cap
        self.state_bytes = N.fgs4d_state_size(self.n, self.c_views, self.nv, cap, self.c_opts)
        self.state = torch.empty(self.state_bytes, device=self.device, dtype=torch.uint8)
        assert self.state.data_ptr() % 256 == 0

    # ---------------------------------------------------------------- stages
    def slice_project(self, params: dict, stream=None):
        g = gaussians_struct(params)
        if g.n != self.n:
            raise ValueError("number of Gaussians differs from the frame's")
        N.fgs4d_slice_project(g, self.c_views, self.nv, self.c_opts, self.state.data_ptr(), self.state_bytes,
                              _stream(stream))

    def bin_sort(self, stream=None):
        N.fgs4d_bin_sort(self.n, self.c_views, self.nv, self.c_opts, self.state.data_ptr(), self.state_bytes,
                         _stream(stream))

    def render(self, stream=None):
        N.fgs4d_render(self.n, self.c_views, self.nv, self.c_opts, self.state.data_ptr(), self.state_bytes,
                       self.image.data_ptr(), self.final_T.data_ptr(), self.n_last.data_ptr(), _stream(stream))

    def render_aux(self, stream=None) -> torch.Tensor:
        """Depth and flow maps (packed like the image: per view [3][H][W] =
        accumulated depth, flow u, flow v) over the current lists; the frame's
        options must have aux_channels=1 before slice_project."""
        if not hasattr(self, "aux_image"):
            self.aux_image = torch.empty(3 * self.total_pixels, device=self.device, dtype=torch.float32)
        N.fgs4d_render_aux(self.n, self.c_views, self.nv, self.c_opts, self.state.data_ptr(), self.state_bytes,
                           self.aux_image.data_ptr(), _stream(stream))
        return self.aux_image

    def render_stats(self, stream=None) -> dict:
        """render() plus the work counts of its walk (one synchronisation):
        pixel-splat pairs inside support boxes, pairs blended, sum of n_last,
        pairs the kernel evaluated."""
        st = torch.zeros(4, device=self.device, dtype=torch.int64)
        N.fgs4d_render_stats(self.n, self.c_views, self.nv, self.c_opts, self.state.data_ptr(), self.state_bytes,
                             self.image.data_ptr(), self.final_T.data_ptr(), self.n_last.data_ptr(), st.data_ptr(),
                             _stream(stream))
        box, blended, walked, evaluated = (int(x) for x in st.cpu())
        return dict(in_box=box, blended=blended, walked=walked, evaluated=evaluated)

    def counters(self, stream=None) -> N.Counters:
        return N.fgs4d_read_counters(self.state.data_ptr(), _stream(stream))

    def forward(self, params: dict, stream=None, check=True) -> torch.Tensor:
        """slice_project -> bin_sort -> render.

        check=True: reads the device counters (one synchronisation) and
        re-runs with a larger pair capacity on overflow.  check=False: no
        check.  check="deferred": no synchronisation once the capacity has
        been sized (the first call sizes it like check=True); the counters
        are copied to pinned host memory behind the render and inspected at
        the next call, or by ``status()``.  A deferred overflow grows the
        capacity for the following calls and is reported by ``status()``."""
        if check == "deferred":
            return self._forward_deferred(params, stream)
        for _ in range(4):
            self.slice_project(params, stream)
            self.bin_sort(stream)
            self.render(stream)
            if not check:
                return self.image
            c = self.counters(stream)
            if c.status & N.STATUS_PAIR_OVERFLOW:
                self._alloc(int(c.n_pairs * 1.25) + 1024)
                continue
            self.last_counters = c
            return self.image
        raise RuntimeError("pair capacity could not be sized")

    def _forward_deferred(self, params: dict, stream=None) -> torch.Tensor:
        if not hasattr(self, "last_counters"):
            return self.forward(params, stream, check=True)
        self._take_deferred(wait=False)
        self.slice_project(params, stream)
        self.bin_sort(stream)
        self.render(stream)
        s = stream if stream is not None else torch.cuda.current_stream()
        if not torch.cuda.is_current_stream_capturing():
            if not hasattr(self, "_host_counters"):
                self._host_counters = torch.empty(4, dtype=torch.int32).pin_memory()
                self._counter_event = torch.cuda.Event()
            with torch.cuda.stream(s):
                self._host_counters.copy_(self.state[:16].view(torch.int32), non_blocking=True)
            self._counter_event.record(s)
            self._pending = True
        return self.image

    def _take_deferred(self, wait: bool):
        """Reads the counters copied behind the last deferred forward once the
        copy has landed (waiting for it only with wait=True)."""
        if not getattr(self, "_pending", False):
            return
        if not wait and not self._counter_event.query():
            return
        self._counter_event.synchronize()
        self._pending = False
        h = [int(x) & 0xffffffff for x in self._host_counters.tolist()]
        c = N.Counters(h[0], h[1], h[2], h[3])
        self.last_counters = c
        if c.status & N.STATUS_PAIR_OVERFLOW:
            self.overflowed = True
            self._alloc(int(c.n_pairs * 1.25) + 1024)

    def status(self) -> N.Counters:
        """Counters of the last forward (waits for a deferred copy); raises if a
        deferred forward dropped (splat, tile) pairs since the last call."""
        self._take_deferred(wait=True)
        if getattr(self, "overflowed", False):
            self.overflowed = False
            raise RuntimeError("a deferred forward exceeded the pair capacity (its image lacks pairs); "
                               f"the capacity has grown to {self.pair_capacity}")
        return self.last_counters

    def _grads(self, params: dict, grads: dict | None, mean2d: bool):
        """mean2d: also the densification signals mean2d_abs (sum over views of
        |dL/dmu_2d|) and mu_t_abs (sum over views of |dL/dmu_t|)."""
        if grads is None:
            grads = {k: torch.empty(params[k].shape, device=self.device, dtype=torch.float32) for k in PARAM_KEYS}
        if mean2d:
            for k in ("mean2d_abs", "mu_t_abs"):
                if k not in grads:
                    grads[k] = torch.empty(self.n, device=self.device, dtype=torch.float32)
        gs = N.GaussianGrads(_ptr(grads["mu"]), _ptr(grads["log_s"]), _ptr(grads["ql"]), _ptr(grads["qr"]),
                             _ptr(grads["logit"]), _ptr(grads["shs"]), _ptr(grads.get("mean2d_abs")),
                             _ptr(grads.get("mu_t_abs")))
        return grads, gs

    def _dL(self, dL_dimage: torch.Tensor) -> torch.Tensor:
        dL = dL_dimage.contiguous()
        if dL.dtype != torch.float32 or dL.numel() != 3 * self.total_pixels:
            raise ValueError("dL_dimage must be float32 with the image's layout")
        return dL

    def backward(self, params: dict, dL_dimage: torch.Tensor, grads: dict | None = None, stream=None,
                 mean2d: bool = False) -> dict:
        """Gradients w.r.t. the raw parameters (both adjoint steps in one call)."""
        g = gaussians_struct(params)
        grads, gs = self._grads(params, grads, mean2d)
        dL = self._dL(dL_dimage)
        N.fgs4d_render_backward(g, self.c_views, self.nv, self.c_opts, self.state.data_ptr(), self.state_bytes,
                                self.final_T.data_ptr(), self.n_last.data_ptr(), dL.data_ptr(), gs, _stream(stream))
        return grads

    def backward_2d(self, dL_dimage: torch.Tensor, stream=None):
        """Adjoint of the compositing alone: per-splat 2D gradients into the state (see grad2d())."""
        dL = self._dL(dL_dimage)
        N.fgs4d_render_backward_2d(self.n, self.c_views, self.nv, self.c_opts, self.state.data_ptr(),
                                   self.state_bytes, self.final_T.data_ptr(), self.n_last.data_ptr(), dL.data_ptr(),
                                   _stream(stream))

    def project_backward(self, params: dict, grads: dict | None = None, stream=None, mean2d: bool = False) -> dict:
        """Second adjoint step: the state's 2D gradients to the raw parameters."""
        g = gaussians_struct(params)
        grads, gs = self._grads(params, grads, mean2d)
        N.fgs4d_project_backward(g, self.c_views, self.nv, self.c_opts, self.state.data_ptr(), self.state_bytes, gs,
                                 _stream(stream))
        return grads

    def step(self, params: dict, dL_dimage: torch.Tensor, grads: dict, stream=None):
        """One whole step on one stream: slice_project, bin_sort, render and
        both adjoint steps (no check of the pair capacity; size it first with
        forward())."""
        self.slice_project(params, stream)
        self.bin_sort(stream)
        self.render(stream)
        self.backward(params, dL_dimage, grads, stream)

    def grad2d(self) -> torch.Tensor:
        """[views, n, 9] view of the state: dL/d(u, v, a, b, c, alpha_eff, R, G, B) per splat, valid
        between backward_2d() and project_backward() (which reuses the section)."""
        info = self.layout()
        g = self.state[info.grad2d: info.grad2d + 48 * self.nv * self.n].view(torch.float32)
        return g.view(self.nv, self.n, 12)[:, :, :9]

    # ---------------------------------------------------------------- views of the packed outputs
    def split(self, packed: torch.Tensor, channels: int = 3) -> list:
        out = []
        for v, off in zip(self.views, self.pix_offsets):
            w, h = int(v["width"]), int(v["height"])
            out.append(packed[channels * off: channels * (off + w * h)].view(channels, h, w) if channels > 1
                       else packed[off: off + w * h].view(h, w))
        return out

    def pack(self, images: list) -> torch.Tensor:
        return torch.cat([im.reshape(-1) for im in images])

    def layout(self) -> N.StateLayoutInfo:
        return N.fgs4d_state_layout(self.n, self.c_views, self.nv, self.c_opts, self.state_bytes)


def split_views(views: list, groups: int) -> list:
    """Contiguous groups of views with balanced pixel counts: the first view
    index of every group after the first."""
    pix = [int(v["width"]) * int(v["height"]) for v in views]
    groups = max(1, min(int(groups), len(views)))
    total, cuts, acc = sum(pix), [], 0
    for i, q in enumerate(pix):
        if len(cuts) < groups - 1 and acc > 0 and acc + q / 2 > total * (len(cuts) + 1) / groups:
            cuts.append(i)
        acc += q
    return cuts


class SplitFrame:
    """The views of one batch as contiguous sub-batches, each a Frame of its
    own on a stream of its own: the groups run the whole step concurrently
    (one group's latency-bound stages -- slice/project, binning, projection
    adjoint -- overlap another's compositing kernels), rendering into one
    packed image.  The step zeroes the gradients once and every group's
    adjoint adds into them (option accumulate_grads).  Views are
    independent, so images, T and n_last are those of one Frame over all the
    views (n_last counts positions in each group's own lists); gradients
    differ only in the order of FP32 sums.  The streams fork from and join
    the caller's stream, so a step can be captured in a CUDA graph."""
    # (the groups' adjoints add into one set of gradients with accumulate_grads; their
    # per-Gaussian outputs take atomic adds, so the groups run without ordering)

    def __init__(self, n: int, views: list, options: dict | None = None, groups: int = 2,
                 pair_capacity: int | None = None, device="cuda", cuts: list | None = None):
        """cuts: the first view index of every group after the first (default:
        split_views(views, groups), groups balanced by pixel count)."""
        self.n = int(n)
        self.views = list(views)
        self.nv = len(self.views)
        self.device = torch.device(device)
        cuts = split_views(self.views, groups) if cuts is None else [int(c) for c in cuts]
        if cuts != sorted(set(cuts)) or (cuts and (cuts[0] < 1 or cuts[-1] >= self.nv)):
            raise ValueError("cuts must be increasing view indices in 1 .. len(views) - 1")
        bounds = [0] + cuts + [self.nv]
        self.parts = [(a, b) for a, b in zip(bounds[:-1], bounds[1:])]
        self.pix_offsets, off = [], 0
        for v in self.views:
            self.pix_offsets.append(off)
            off += int(v["width"]) * int(v["height"])
        self.total_pixels = off
        self.c_views = N.make_views(self.views)
        self.image = torch.empty(3 * off, device=self.device, dtype=torch.float32)
        self.final_T = torch.empty(off, device=self.device, dtype=torch.float32)
        self.n_last = torch.empty(off, device=self.device, dtype=torch.int32)
        self.frames, self.ranges = [], []
        for gi, (a, b) in enumerate(self.parts):
            p0 = self.pix_offsets[a]
            p1 = self.pix_offsets[b] if b < self.nv else off
            opts = dict(options or {}, accumulate_grads=1)
            outs = (self.image[3 * p0: 3 * p1], self.final_T[p0:p1], self.n_last[p0:p1])
            cap = None if pair_capacity is None else max(1 << 16, int(pair_capacity * (p1 - p0) / max(off, 1)))
            self.frames.append(Frame(n, self.views[a:b], opts, cap, device, outputs=outs))
            self.ranges.append((p0, p1))
        self.streams = [torch.cuda.Stream(device=self.device) for _ in self.frames]

    @property
    def groups(self) -> int:
        return len(self.frames)

    def _dL(self, dL_dimage: torch.Tensor, gi: int) -> torch.Tensor:
        p0, p1 = self.ranges[gi]
        return dL_dimage[3 * p0: 3 * p1]

    def forward(self, params: dict, stream=None, check: bool = True) -> torch.Tensor:
        """Every group's slice_project -> bin_sort -> render, concurrently;
        check=True sizes each group's pair capacity as Frame.forward does."""
        if check:
            for fr in self.frames:
                fr.forward(params, stream, check=True)
            return self.image
        cur = stream if stream is not None else torch.cuda.current_stream()
        for fr, s in zip(self.frames, self.streams):
            s.wait_stream(cur)
            fr.slice_project(params, s)
            fr.bin_sort(s)
            fr.render(s)
        for s in self.streams:
            cur.wait_stream(s)
        return self.image

    def step(self, params: dict, dL_dimage: torch.Tensor, grads: dict, stream=None):
        """One whole step: grads are zeroed, then every group runs its forward
        and both adjoint steps on its own stream, adding into grads
        (accumulate_grads: atomic adds, so the groups need no ordering)."""
        cur = stream if stream is not None else torch.cuda.current_stream()
        dL = dL_dimage.contiguous()
        with torch.cuda.stream(cur):
            for k in PARAM_KEYS:
                grads[k].zero_()
        for gi, (fr, s) in enumerate(zip(self.frames, self.streams)):
            s.wait_stream(cur)
            fr.slice_project(params, s)
            fr.bin_sort(s)
            fr.render(s)
            fr.backward_2d(self._dL(dL, gi), s)
            fr.project_backward(params, grads, s)
        for s in self.streams:
            cur.wait_stream(s)

    def backward(self, params: dict, dL_dimage: torch.Tensor, grads: dict | None = None, stream=None) -> dict:
        """The adjoint of the last forward: grads are zeroed, then every
        group's adjoint adds into them on its own stream."""
        if grads is None:
            grads = {k: torch.empty(params[k].shape, device=self.device, dtype=torch.float32) for k in PARAM_KEYS}
        cur = stream if stream is not None else torch.cuda.current_stream()
        dL = dL_dimage.contiguous()
        with torch.cuda.stream(cur):
            for k in PARAM_KEYS:
                grads[k].zero_()
        for gi, (fr, s) in enumerate(zip(self.frames, self.streams)):
            s.wait_stream(cur)
            fr.backward_2d(self._dL(dL, gi), s)
            fr.project_backward(params, grads, s)
        for s in self.streams:
            cur.wait_stream(s)
        return grads

    def counters(self) -> list:
        return [fr.counters() for fr in self.frames]

    def split(self, packed: torch.Tensor, channels: int = 3) -> list:
        out = []
        for v, off in zip(self.views, self.pix_offsets):
            w, h = int(v["width"]), int(v["height"])
            out.append(packed[channels * off: channels * (off + w * h)].view(channels, h, w) if channels > 1
                       else packed[off: off + w * h].view(h, w))
        return out


class Render4DGS(torch.autograd.Function):
    """images_packed = Render4DGS.apply(frame, mu, log_s, ql, qr, logit, shs)."""

    @staticmethod
    def forward(ctx, frame: Frame, mu, log_s, ql, qr, logit, shs, sh_degree: int, n_freq: int, period: float):
        params = dict(mu=mu.detach(), log_s=log_s.detach(), ql=ql.detach(), qr=qr.detach(), logit=logit.detach(),
                      shs=shs.detach(), sh_degree=sh_degree, n_freq=n_freq, period=period)
        # no synchronisation: the pair-capacity check is deferred (Frame.status)
        img = frame.forward(params, check="deferred").clone()
        ctx.frame = frame
        ctx.meta = (sh_degree, n_freq, period)
        ctx.save_for_backward(mu, log_s, ql, qr, logit, shs)
        return img

    @staticmethod
    def backward(ctx, dimg):
        mu, log_s, ql, qr, logit, shs = ctx.saved_tensors
        L, K, T = ctx.meta
        params = dict(mu=mu.detach(), log_s=log_s.detach(), ql=ql.detach(), qr=qr.detach(), logit=logit.detach(),
                      shs=shs.detach(), sh_degree=L, n_freq=K, period=T)
        g = ctx.frame.backward(params, dimg.float())
        gshs = g["shs"].to(shs.dtype)
        return None, g["mu"], g["log_s"], g["ql"], g["qr"], g["logit"], gshs, None, None, None


def render(params: dict, views: list, options: dict | None = None, frame: Frame | None = None):
    """Differentiable render of all views; returns (list of [3,H,W] images, frame)."""
    n = params["logit"].shape[0]
    if frame is None:
        frame = Frame(n, views, options, device=params["mu"].device)
    packed = Render4DGS.apply(frame, params["mu"], params["log_s"], params["ql"], params["qr"], params["logit"],
                              params["shs"], int(params["sh_degree"]), int(params["n_freq"]),
                              float(params.get("period", 1.0)))
    return frame.split(packed), frame
