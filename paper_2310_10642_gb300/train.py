"""One training step of 4DGS (Sec. 3.3), all of it in the library's kernels.

forward (fgs4d_slice_project, fgs4d_bin_sort, fgs4d_render) ->
loss and dL/dimage (fgs4d_loss_l1_dssim) -> adjoint (fgs4d_render_backward) ->
Adam over every parameter group (fgs4d_adam_step), which also refreshes the
BF16 copy of the 4DSH coefficients that the mixed-precision renderer reads.

The FP32 parameters are the master weights.  Learning rates and the step
counter live on the device, so ``capture()`` records the whole step once as a
CUDA graph and every ``replay()`` runs a full step (the host may change
``lrs`` in between).  Argument marshalling only: no arithmetic here.
"""
from __future__ import annotations

import torch

from . import native as N
from . import render as R

GROUPS = ("mu", "log_s", "ql", "qr", "logit", "shs")
# per-group learning rates in the spirit of the 3D Gaussian splatting setting
# the paper adopts; callers pass their own
DEFAULT_LRS = dict(mu=1.6e-4, log_s=5e-3, ql=1e-3, qr=1e-3, logit=5e-2, shs=2.5e-3)


class TrainStep:
    def __init__(self, params: dict, views: list, targets: torch.Tensor, options: dict | None = None,
                 mixed: bool = True, lrs: dict | None = None, lam: float = 0.2, betas=(0.9, 0.999), eps=1e-15,
                 pair_capacity: int | None = None, groups: int = 1):
        """params: FP32 device parameters (R.params_to_device); targets: packed
        [3 * total pixels] float32 like the rendered image.  groups > 1
        renders the views as that many groups on their own streams
        (R.SplitFrame): forward and adjoint of one group overlap another's."""
        self.master = params
        self.mixed = bool(mixed)
        self.lam = float(lam)
        self.betas = tuple(float(b) for b in betas)
        self.eps = float(eps)
        dev = params["mu"].device
        self.render_params = dict(params)
        self.shs_bf16 = None
        if self.mixed:
            self.shs_bf16 = params["shs"].to(torch.bfloat16)
            self.render_params["shs"] = self.shs_bf16
        opts = dict(options or {}, record_fp16=int(self.mixed))
        n = int(params["logit"].shape[0])
        if int(groups) > 1:
            self.frame = R.SplitFrame(n, views, opts, groups=int(groups), pair_capacity=pair_capacity, device=dev)
        else:
            self.frame = R.Frame(n, views, opts, pair_capacity=pair_capacity, device=dev)
        self.frame.forward(self.render_params, check=True)
        for fr in getattr(self.frame, "frames", [self.frame]):
            c = fr.last_counters
            if c.n_pairs * 1.2 > fr.pair_capacity:  # headroom for the parameters to move
                fr._alloc(int(c.n_pairs * 1.3) + 4096)
        self.targets = targets.contiguous()
        if self.targets.numel() != 3 * self.frame.total_pixels:
            raise ValueError("targets must have the packed image layout")
        self.grads = {k: torch.zeros_like(params[k], dtype=torch.float32) for k in GROUPS}
        self.exp_avg = {k: torch.zeros_like(params[k], dtype=torch.float32) for k in GROUPS}
        self.exp_avg_sq = {k: torch.zeros_like(params[k], dtype=torch.float32) for k in GROUPS}
        lr = dict(DEFAULT_LRS, **(lrs or {}))
        self.lrs = torch.tensor([lr[k] for k in GROUPS], dtype=torch.float32, device=dev)
        self.step_count = torch.zeros(1, dtype=torch.int64, device=dev)
        self.bias = torch.zeros(2, dtype=torch.float32, device=dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=dev)
        self.dL = torch.empty(3 * self.frame.total_pixels, dtype=torch.float32, device=dev)
        self.scratch_bytes = N.fgs4d_loss_scratch_size(self.frame.c_views, self.frame.nv)
        self.scratch = torch.empty(self.scratch_bytes, dtype=torch.uint8, device=dev)
        self._groups = []
        for i, k in enumerate(GROUPS):
            p = params[k]
            if p.dtype != torch.float32 or not p.is_contiguous():
                raise ValueError(f"master parameter {k} must be contiguous float32")
            bf = self.shs_bf16.data_ptr() if (k == "shs" and self.shs_bf16 is not None) else None
            self._groups.append(N.AdamGroup(p.data_ptr(), self.exp_avg[k].data_ptr(), self.exp_avg_sq[k].data_ptr(),
                                            self.grads[k].data_ptr(), bf, p.numel(), i))
        self.graph = None

    def step(self, stream=None):
        """Enqueues one full training step on the current stream."""
        fr = self.frame
        s = R._stream(stream)
        fr.forward(self.render_params, stream, check=False)
        N.fgs4d_loss_l1_dssim(fr.c_views, fr.nv, fr.image.data_ptr(), self.targets.data_ptr(), self.lam,
                              self.loss.data_ptr(), self.dL.data_ptr(), self.scratch.data_ptr(), self.scratch_bytes,
                              s)
        fr.backward(self.render_params, self.dL, self.grads, stream)
        N.fgs4d_adam_step(self._groups, self.lrs.data_ptr(), self.betas[0], self.betas[1], self.eps,
                          self.step_count.data_ptr(), self.bias.data_ptr(), s)

    def capture(self):
        """Records one step as a CUDA graph (the caller has run warm-up steps)."""
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.step()
        return self.graph

    def replay(self):
        self.graph.replay()
