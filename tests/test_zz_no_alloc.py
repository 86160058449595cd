"""fgs4d_render_backward_noalloc: the backward pass for callers that cannot
allocate device memory when they run it (code whose stream is being captured
into a CUDA graph, loops that reserve all memory at start-up, plugins of an
engine that owns the allocator).  It keeps its per-splat scratch in the
library's static device array instead of the caller's state.

Checked here through the C ABI: on two calls in a row (the second must not
see the first one's scratch), its gradients equal those of
fgs4d_render_backward within the gradient tolerance of the parity tests; a
problem larger than the array is refused on the host.  This file is
collected last so that a stop-at-first-failure run has already run every
other test; it also runs alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2310_10642_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_10642_gb300 import native
    native.build()
    native.lib()
    return native


def _grads_struct(N, grads):
    return N.GaussianGrads(*(grads[k].data_ptr() for k in ("mu", "log_s", "ql", "qr", "logit", "shs")), None)


def test_noalloc_backward_matches_regular_backward(N):
    from paper_2310_10642_gb300 import render as R
    G = I.gaussians(3000, 11, 3, 2)
    views = [I.view((0.3, 0.2, 4.0), 77, 53, 0.31, bg=(0.1, 0.3, 0.2)),
             I.view((-2.0, 1.0, 3.3), 40, 96, 0.55),
             I.view((1.5, -0.5, -3.6), 130, 31, 0.8)]
    p = R.params_to_device(G)
    fr = R.Frame(3000, views)
    fr.forward(p)
    dL = torch.randn(3 * fr.total_pixels, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    ref = {k: v.clone() for k, v in fr.backward(p, dL).items()}
    g = R.gaussians_struct(p)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = {k: torch.full(p[k].shape, float("nan"), device="cuda") for k in R.PARAM_KEYS}
        N.fgs4d_render_backward_noalloc(g, fr.c_views, fr.nv, fr.c_opts, fr.state.data_ptr(), fr.state_bytes,
                                        fr.final_T.data_ptr(), fr.n_last.data_ptr(), dL.data_ptr(),
                                        _grads_struct(N, out), stream)
        torch.cuda.synchronize()
        for k in R.PARAM_KEYS:
            a, b = out[k].double().cpu().numpy(), ref[k].double().cpu().numpy()
            assert np.all(np.isfinite(a)), (call, k)
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            assert rel <= GRAD_TOL, f"call {call}, {k}: relative difference {rel:.3e}"


def test_noalloc_backward_rejects_problems_beyond_the_array(N):
    n = N.NOALLOC_MAX_SPLATS // 2 + 1
    views = N.make_views([I.view((0, 0, 4), 16, 16, 0.5), I.view((0, 0, 4), 16, 16, 0.5)])
    opts = N.fgs4d_default_options()
    fake = 1 << 20  # 16-byte aligned stand-in pointers: the size check runs first, nothing is launched
    g = N.Gaussians(fake, fake, fake, fake, fake, fake, n, 1, 1, 1.0, 0)
    gr = N.GaussianGrads(fake, fake, fake, fake, fake, fake, None)
    code = N.lib().fgs4d_render_backward_noalloc(g, views, 2, opts, fake, 1 << 30, fake, fake, fake, gr, None)
    assert code == 2  # FGS4D_ERR_CAPACITY
