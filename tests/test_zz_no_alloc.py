"""fgs4d_render_backward_noalloc: the backward pass for callers that cannot
allocate device memory when they run it (render loops that reserve all device
memory at start-up and may not allocate afterwards, plugins hosted by an
engine that owns the allocator).  It keeps its per-splat scratch in the
library's static device array instead of the caller's state.

Checked here through the C ABI: on two calls in a row (the second must not
see the first one's scratch), its gradients equal those of
fgs4d_render_backward within the gradient tolerance of the parity tests, for
FP32 and BF16 coefficients, the 4D and the spatial-only rotation, and with
the densification sums requested; exactly FGS4D_NOALLOC_MAX_SPLATS splats
pass the size check and one more splat is refused on the host.  This file is
collected last so that a stop-at-first-failure run has already run every
other test; it also runs alone in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2310_10642_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3
KEYS = ("mu", "log_s", "ql", "qr", "logit", "shs", "mean2d_abs", "mu_t_abs")


@pytest.fixture(scope="module")
def N():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_10642_gb300 import native
    native.build()
    native.lib()
    return native


def _grads_struct(N, grads):
    return N.GaussianGrads(*(grads[k].data_ptr() for k in KEYS))


@pytest.mark.parametrize("shs_dtype,rotation", [("f32", "4d"), ("bf16", "4d"), ("f32", "spatial")])
def test_noalloc_backward_matches_regular_backward(N, shs_dtype, rotation):
    from paper_2310_10642_gb300 import render as R
    G = I.gaussians(3000, 11, 3, 2)
    if rotation == "spatial":
        G["rotation"] = N.ROT_SPATIAL
    views = [I.view((0.3, 0.2, 4.0), 77, 53, 0.31, bg=(0.1, 0.3, 0.2)),
             I.view((-2.0, 1.0, 3.3), 40, 96, 0.55),
             I.view((1.5, -0.5, -3.6), 130, 31, 0.8)]
    p = R.params_to_device(G, shs_dtype=torch.bfloat16 if shs_dtype == "bf16" else torch.float32)
    fr = R.Frame(3000, views, dict(record_fp16=int(shs_dtype == "bf16")))
    fr.forward(p)
    dL = torch.randn(3 * fr.total_pixels, device="cuda", generator=torch.Generator(device="cuda").manual_seed(3))
    ref = {k: v.clone() for k, v in fr.backward(p, dL, mean2d=True).items()}
    g = R.gaussians_struct(p)
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        out = {k: torch.full(ref[k].shape, float("nan"), device="cuda") for k in KEYS}
        N.fgs4d_render_backward_noalloc(g, fr.c_views, fr.nv, fr.c_opts, fr.state.data_ptr(), fr.state_bytes,
                                        fr.final_T.data_ptr(), fr.n_last.data_ptr(), dL.data_ptr(),
                                        _grads_struct(N, out), stream)
        torch.cuda.synchronize()
        for k in KEYS:
            a, b = out[k].double().cpu().numpy(), ref[k].double().cpu().numpy()
            if rotation == "spatial" and k == "qr":
                assert np.all(a == 0.0) and np.all(b == 0.0), call  # q_right takes no part
                continue
            assert np.all(np.isfinite(a)), (call, k)
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            assert np.linalg.norm(b) > 0 and rel <= GRAD_TOL, f"call {call}, {k}: relative difference {rel:.3e}"


def _noalloc_code(N, n, n_views, opts):
    views = N.make_views([I.view((0, 0, 4), 16, 16, 0.5)] * n_views)
    fake = 1 << 20  # 16-byte aligned stand-in pointers: both cases return before anything is launched
    g = N.Gaussians(fake, fake, fake, fake, fake, fake, n, 1, 1, 1.0, 0, 0)
    gr = N.GaussianGrads(fake, fake, fake, fake, fake, fake, None, None)
    return N.lib().fgs4d_render_backward_noalloc(g, views, n_views, opts, fake, 1 << 30, fake, fake, fake, gr, None)


def test_noalloc_backward_size_limit(N):
    """n * n_views = FGS4D_NOALLOC_MAX_SPLATS passes the size check (the
    invalid tile size then stops the call before any launch); one splat more
    is refused with FGS4D_ERR_CAPACITY."""
    bad = N.fgs4d_default_options()
    bad.tile_size = 7
    assert _noalloc_code(N, N.NOALLOC_MAX_SPLATS // 2, 2, bad) == 1      # FGS4D_ERR_INVALID_ARG
    assert _noalloc_code(N, N.NOALLOC_MAX_SPLATS, 1, bad) == 1
    ok = N.fgs4d_default_options()
    assert _noalloc_code(N, N.NOALLOC_MAX_SPLATS // 2 + 1, 2, ok) == 2  # FGS4D_ERR_CAPACITY
    assert _noalloc_code(N, N.NOALLOC_MAX_SPLATS + 1, 1, ok) == 2
