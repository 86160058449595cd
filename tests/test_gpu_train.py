"""The training step on the GPU against the FP64 oracle: the L1 + D-SSIM loss
and its image gradient, Adam over parameter groups, and the whole step
captured as one CUDA graph."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import train_oracle as TO  # noqa: E402
from paper_2310_10642_gb300 import inputs as I  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2310_10642_gb300 import native
    native.build()
    native.lib()


def _views(sizes):
    return [I.view((0.0, 0.0, 4.0), w, h, 0.5) for w, h in sizes]


def _loss_gpu(views, ims, tgs, lam):
    from paper_2310_10642_gb300 import native as N
    cv = N.make_views(views)
    img = torch.cat([torch.as_tensor(a, dtype=torch.float32).reshape(-1) for a in ims]).cuda()
    tgt = torch.cat([torch.as_tensor(a, dtype=torch.float32).reshape(-1) for a in tgs]).cuda()
    nbytes = N.fgs4d_loss_scratch_size(cv, len(views))
    scratch = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    loss = torch.zeros(1, device="cuda")
    dL = torch.empty_like(img)
    N.fgs4d_loss_l1_dssim(cv, len(views), img.data_ptr(), tgt.data_ptr(), lam, loss.data_ptr(), dL.data_ptr(),
                          scratch.data_ptr(), nbytes, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    out, off = [], 0
    for a in ims:
        out.append(dL[off: off + a.size].view(a.shape).double().cpu().numpy())
        off += a.size
    return float(loss.item()), out


@pytest.mark.parametrize("lam", [0.2, 0.0, 1.0])
def test_loss_and_image_gradient_match_oracle(lam):
    sizes = [(77, 53), (40, 96), (130, 31), (16, 16), (1, 1)]
    views = _views(sizes)
    r = np.random.default_rng(7)
    ims = [r.uniform(size=(3, h, w)).astype(np.float32) for w, h in sizes]
    tgs = [np.clip(a + r.normal(scale=0.2, size=a.shape), 0, 1).astype(np.float32) for a in ims]
    loss, g = _loss_gpu(views, ims, tgs, lam)
    want, gw = TO.loss_l1_dssim([a.astype(np.float64) for a in ims], [a.astype(np.float64) for a in tgs], lam)
    count = sum(a.size for a in ims)
    print(f"[parity] loss lambda={lam}: gpu {loss:.9f} oracle {want:.9f}")
    assert abs(loss - want) <= 2e-6 * abs(want) + 1e-7
    for a, b, im, tg in zip(g, gw, ims, tgs):
        ok = np.abs(im.astype(np.float64) - tg) > 1e-6  # away from the L1 kink
        err = np.abs(a - b)[ok].max() * count
        print(f"[parity] dL/dimage (x count) max-abs error {err:.3e}")
        assert err <= 2e-4


def test_adam_matches_oracle_over_three_steps():
    """Groups of 1000 and 777 elements take the 16-byte path (777: and its
    one-element tail, with the BF16 copy), 33 elements mostly the tail, and a
    group starting one element into its arrays (not 16-byte aligned) the
    element-by-element path."""
    from paper_2310_10642_gb300 import native as N
    r = np.random.default_rng(9)
    sizes = [1000, 777, 33, 101]
    lrs_h = [1e-2, 3e-3, 1e-1, 5e-3]
    ng = len(sizes)
    p = [torch.tensor(r.normal(size=s + 1), dtype=torch.float32, device="cuda")[1:] if i == 3 else
         torch.tensor(r.normal(size=s), dtype=torch.float32, device="cuda") for i, s in enumerate(sizes)]
    m = [torch.zeros(s + 1, device="cuda")[1:] if i == 3 else torch.zeros_like(x)
         for i, (x, s) in enumerate(zip(p, sizes))]
    v = [torch.zeros(s + 1, device="cuda")[1:] if i == 3 else torch.zeros_like(x)
         for i, (x, s) in enumerate(zip(p, sizes))]
    gs = [torch.zeros(s + 1, device="cuda")[1:] if i == 3 else torch.zeros_like(x)
          for i, (x, s) in enumerate(zip(p, sizes))]
    assert p[3].data_ptr() % 16 != 0
    bf = torch.empty(sizes[1], dtype=torch.bfloat16, device="cuda")
    lrs = torch.tensor(lrs_h, device="cuda")
    step = torch.zeros(1, dtype=torch.int64, device="cuda")
    bias = torch.zeros(2, device="cuda")
    groups = [N.AdamGroup(p[i].data_ptr(), m[i].data_ptr(), v[i].data_ptr(), gs[i].data_ptr(),
                          bf.data_ptr() if i == 1 else None, sizes[i], i) for i in range(ng)]
    ref = [(x.double().cpu().numpy(), np.zeros(s), np.zeros(s)) for x, s in zip(p, sizes)]
    for t in range(1, 4):
        gh = [r.normal(size=s).astype(np.float32) for s in sizes]
        for i in range(ng):
            gs[i].copy_(torch.as_tensor(gh[i]))
        N.fgs4d_adam_step(groups, lrs.data_ptr(), 0.9, 0.999, 1e-8, step.data_ptr(), bias.data_ptr(),
                          torch.cuda.current_stream().cuda_stream)
        ref = [TO.adam_step(rp, rm, rv, gh[i].astype(np.float64), t, lrs_h[i], 0.9, 0.999, 1e-8)
               for i, (rp, rm, rv) in enumerate(ref)]
    torch.cuda.synchronize()
    assert int(step.item()) == 3
    for i in range(ng):
        assert np.abs(p[i].double().cpu().numpy() - ref[i][0]).max() < 1e-5
        assert np.abs(m[i].double().cpu().numpy() - ref[i][1]).max() < 1e-6
        assert np.abs(v[i].double().cpu().numpy() - ref[i][2]).max() < 1e-6
    assert torch.equal(bf, p[1].to(torch.bfloat16))


@pytest.mark.parametrize("mixed", [False, True])
def test_training_step_as_one_cuda_graph(mixed):
    """Forward, loss, adjoint and Adam recorded once; replays advance the
    device step counter, the first replay's loss equals an eager step's, and
    the loss falls over the replays."""
    from paper_2310_10642_gb300 import render as R
    from paper_2310_10642_gb300.train import TrainStep
    c = I.config(4, n=20000, scale=0.1)
    G, views = c["gaussians"], c["views"]
    assert len(views) == 8 and len({(v["width"], v["height"]) for v in views}) == 2

    def fresh():
        p = R.params_to_device(G)
        tg = torch.cat([torch.as_tensor(t, dtype=torch.float32).reshape(-1) for t in I.random_target(views, 5)])
        return p, tg.cuda()

    p, tg = fresh()
    eager = TrainStep(p, views, tg, dict(tile_size=32), mixed=mixed, eps=1e-8)
    eager.step()
    torch.cuda.synchronize()
    loss_eager = float(eager.loss.item())

    p, tg = fresh()
    ts = TrainStep(p, views, tg, dict(tile_size=32), mixed=mixed, eps=1e-8)
    ts.capture()
    losses = []
    for k in range(6):
        ts.replay()
        torch.cuda.synchronize()
        losses.append(float(ts.loss.item()))
    assert int(ts.step_count.item()) == 6
    assert ts.frame.counters().status == 0
    # the same steps with the views in two groups on two streams: same images, so the same
    # losses up to the order of FP32 sums in the gradients
    p, tg = fresh()
    ts2 = TrainStep(p, views, tg, dict(tile_size=32), mixed=mixed, eps=1e-8, groups=2)
    assert ts2.frame.groups == 2
    ts2.capture()
    losses2 = []
    for k in range(6):
        ts2.replay()
        torch.cuda.synchronize()
        losses2.append(float(ts2.loss.item()))
    assert losses2[0] == losses[0]
    assert np.allclose(losses2, losses, rtol=1e-5, atol=0.0), (losses2, losses)
    assert all(c_.status == 0 for c_ in ts2.frame.counters())
    assert losses[0] == loss_eager
    assert losses[-1] < losses[0]
    if mixed:
        assert torch.equal(ts.shs_bf16, ts.master["shs"].to(torch.bfloat16))
    print(f"[train] mixed={mixed} losses {losses}")
