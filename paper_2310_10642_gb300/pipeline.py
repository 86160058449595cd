"""Forward + backward over host-resident batches with the copies overlapped.

``HostPipeline`` runs ``Frame`` (or ``SplitFrame``) steps (slice/project,
bin/sort, render, backward) whose inputs (parameters, dL/dimage) come from pinned host memory
and whose outputs (image, gradients) go back to pinned host memory.  While
step k computes on the current stream, the inputs of step k + 1 are copied
in and the outputs of step k - 1 copied out on two copy streams, through two
device buffer sets; CUDA events keep each buffer from being overwritten while
a copy or a step still uses it.  With ``graphs`` (the default) the compute of
each buffer set is captured as a CUDA graph after its first eager step and
replayed from then on, so a step costs one launch on the host.  Argument
marshalling and stream ordering only: every step of the method runs in the
library's kernels.
"""
from __future__ import annotations

import torch

from . import render as R


class HostPipeline:
    def __init__(self, frame: "R.Frame", params_like: dict, device="cuda", graphs: bool = True):
        """params_like: device parameters whose shapes and dtypes the host
        inputs have (sh_degree, n_freq and period are taken from it)."""
        self.frame = frame
        self.graphs = bool(graphs)
        self.stream = torch.cuda.current_stream()
        self.s_in, self.s_out = torch.cuda.Stream(), torch.cuda.Stream()
        npix = frame.total_pixels
        self.slots = []
        for _ in range(2):
            dp = {k: torch.empty_like(params_like[k]) for k in R.PARAM_KEYS}
            dp.update({k: params_like[k] for k in ("sh_degree", "n_freq", "period") if k in params_like})
            if "rotation" in params_like:
                dp["rotation"] = params_like["rotation"]
            sl = dict(p=dp, dL=torch.empty(3 * npix, device=device), img=torch.empty(3 * npix, device=device),
                      g={k: torch.empty(params_like[k].shape, device=device) for k in R.PARAM_KEYS},
                      ev_in=torch.cuda.Event(), ev_used=torch.cuda.Event(), ev_out=torch.cuda.Event(),
                      graph=None, eager_steps=0)
            for ev in ("ev_in", "ev_used", "ev_out"):  # start recorded: the first waits do not block
                sl[ev].record(self.stream)
            self.slots.append(sl)

    def _copy_in(self, sl, host_params: dict, host_dL: torch.Tensor):
        with torch.cuda.stream(self.s_in):
            self.s_in.wait_event(sl["ev_used"])  # the step that last read this slot is done
            for k in R.PARAM_KEYS:
                sl["p"][k].copy_(host_params[k], non_blocking=True)
            sl["dL"].copy_(host_dL, non_blocking=True)
            sl["ev_in"].record(self.s_in)

    def _step(self, sl):
        fr = self.frame
        fr.step(sl["p"], sl["dL"], sl["g"])
        sl["img"].copy_(fr.image, non_blocking=True)

    def _compute(self, sl):
        st = self.stream
        st.wait_event(sl["ev_in"])
        st.wait_event(sl["ev_out"])  # the outputs of this slot have left the device
        if self.graphs and sl["graph"] is None and sl["eager_steps"] > 0:
            # every buffer the step touches is fixed per slot, so the step is captured once
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._step(sl)
            sl["graph"] = g
        if sl["graph"] is not None:
            sl["graph"].replay()
        else:
            self._step(sl)
            sl["eager_steps"] += 1
        sl["ev_used"].record(st)

    def _copy_out(self, sl, host_image: torch.Tensor, host_grads: dict):
        with torch.cuda.stream(self.s_out):
            self.s_out.wait_event(sl["ev_used"])
            host_image.copy_(sl["img"], non_blocking=True)
            for k in R.PARAM_KEYS:
                host_grads[k].copy_(sl["g"][k], non_blocking=True)
            sl["ev_out"].record(self.s_out)

    def run(self, inputs: list, outputs: list):
        """inputs[k] = (host_params, host_dL); outputs[k] = (host_image,
        host_grads), all pinned.  Enqueues len(inputs) steps; the current
        stream waits for the last copy out (synchronise it before reading)."""
        if len(outputs) != len(inputs):
            raise ValueError("one output set per input set")
        steps = len(inputs)
        self.s_in.wait_stream(self.stream)
        if steps:
            self._copy_in(self.slots[0], *inputs[0])
        for k in range(steps):
            if k + 1 < steps:
                self._copy_in(self.slots[(k + 1) % 2], *inputs[k + 1])
            self._compute(self.slots[k % 2])
            self._copy_out(self.slots[k % 2], *outputs[k])
        self.stream.wait_stream(self.s_out)
