"""GPU checks of the learned segment proposal (not in the paper): the tensor-core MLP
inference and the training kernels against the FP64 oracle MLP, the segment log against
quantities the plain march fixes, and the learned march against the plain march."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import gpu_render, gpu_trace, params_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    import torch

    import paper_1212_3333_gb300 as amr
    from paper_1212_3333_gb300 import proposal

    return torch, amr, proposal


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even to bfloat16, returned as float64."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _oracle_params(proposal, p):
    ws = proposal.split_params(p)
    return [bf16_round(w) if w.ndim == 2 else w.astype(np.float64) for w in ws]


def test_mlp_forward_matches_oracle(mods):
    torch, amr, proposal = mods
    rng = np.random.default_rng(0)
    p = proposal.init_params(3) + rng.normal(0, 0.05, size=9217).astype(np.float32)
    x = rng.uniform(0, 1, size=(1000, 12)).astype(np.float32)
    prop = proposal.Proposal(p)
    y = prop.predict(torch.as_tensor(x, device="cuda")).cpu().numpy().astype(np.float64)
    ref = oracle.mlp_forward(_oracle_params(proposal, p), bf16_round(x))
    rel = np.abs(y - ref) / np.maximum(ref, 1e-3)
    assert rel.max() <= 2e-2, rel.max()


def test_mlp_gradient_matches_oracle(mods):
    torch, amr, proposal = mods
    rng = np.random.default_rng(1)
    p = proposal.init_params(5) + rng.normal(0, 0.05, size=9217).astype(np.float32)
    x = rng.uniform(0, 1, size=(700, 12)).astype(np.float32)
    t = rng.uniform(0, 1, size=700).astype(np.float32) ** 4
    prop = proposal.Proposal(p)
    prop.loss_grad(torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda"))
    torch.cuda.synchronize()
    g = prop.grad.cpu().numpy().astype(np.float64)
    loss = float(prop.loss.item())
    ref_loss, ref_g = oracle.mlp_loss_grad(_oracle_params(proposal, p), bf16_round(x), t)
    ref = np.concatenate([q.ravel() for q in ref_g])
    cos = g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref))
    assert cos >= 0.999, cos
    assert abs(loss - ref_loss) <= 1e-3 * abs(ref_loss)
    for k, (a, b) in enumerate(zip(proposal.split_params(g), ref_g)):
        b = b.ravel()
        a = a.ravel()
        if np.linalg.norm(b) > 1e-9:
            assert a @ b / (np.linalg.norm(a) * np.linalg.norm(b)) >= 0.995, k


def test_adam_step_matches_formula(mods):
    torch, amr, proposal = mods
    rng = np.random.default_rng(2)
    p = rng.normal(size=9217).astype(np.float32)
    prop = proposal.Proposal(p)
    g = rng.normal(size=9217).astype(np.float32)
    prop.grad.copy_(torch.as_tensor(g, device="cuda"))
    m = np.zeros(9217)
    v = np.zeros(9217)
    w = p.astype(np.float64)
    for step in (1, 2):
        prop.adam(1e-2, 0.9, 0.999, 1e-8)
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g.astype(np.float64) ** 2
        w = w - 1e-2 * (m / (1 - 0.9 ** step)) / (np.sqrt(v / (1 - 0.999 ** step)) + 1e-8)
    torch.cuda.synchronize()
    np.testing.assert_allclose(prop.params.cpu().numpy(), w, rtol=1e-5, atol=1e-6)


def test_permuted_batches_read_the_permuted_rows(mods):
    torch, amr, proposal = mods
    rng = np.random.default_rng(3)
    N, a, b, first, n = 997, 389, 123, 200, 300
    x = rng.uniform(0, 1, size=(N, 12)).astype(np.float32)
    t = rng.uniform(0, 1, size=N).astype(np.float32)
    prop = proposal.Proposal(seed=4)
    xd, td = torch.as_tensor(x, device="cuda"), torch.as_tensor(t, device="cuda")
    prop.loss_grad(xd, td, first, n, a, b)
    torch.cuda.synchronize()
    g1, l1 = prop.grad.clone(), float(prop.loss.item())
    rows = (a * (first + np.arange(n)) + b) % N
    prop.loss_grad(torch.as_tensor(x[rows], device="cuda"), torch.as_tensor(t[rows], device="cuda"))
    torch.cuda.synchronize()
    assert abs(l1 - float(prop.loss.item())) <= 1e-5 * abs(l1)
    torch.testing.assert_close(g1, prop.grad, rtol=1e-4, atol=1e-7)


@pytest.fixture(scope="module")
def c1_learned(mods):
    torch, amr, proposal = mods
    w = synth.c1_workload()
    ctx = amr.from_hierarchy(w["hier"])
    ctx.amr_build_kdtree("ptr")
    return w, ctx


def test_segment_log_invariants(mods, c1_learned):
    torch, amr, proposal = mods
    w, ctx = c1_learned
    cam = synth.orbit_camera(11, 64, 48)
    tf = torch.as_tensor(w["tf"], device="cuda")
    p, _ = params_pair(amr, w["vmin"], w["vmax"], ert_eps=0.0)
    feats, tgts, seen = proposal.log_segments(ctx, [cam], tf, p, capacity=1 << 20, keep_prob=1.0)
    # every segment of every ray is recorded
    _, _, ln = gpu_trace(ctx, cam, max_len=512)
    assert seen == int(ln.sum()) == feats.shape[0]
    # the contributions of a ray's segments add up to its opacity
    img, _ = gpu_render(ctx, cam, w["tf"], p)
    assert abs(float(tgts.double().sum()) - img[..., 3].sum()) <= 1e-4 * img[..., 3].sum()
    # records follow pixel order, then segment order: each pixel's records are its segments,
    # contiguous, and their contributions add up to that pixel's opacity
    counts = np.maximum(ln, 0).astype(np.int64)
    starts = (np.cumsum(counts) - counts)[counts > 0]
    per_pixel = np.add.reduceat(tgts.double().cpu().numpy(), starts)
    np.testing.assert_allclose(per_pixel, img[..., 3].reshape(-1)[counts > 0], rtol=0, atol=2e-6)
    # and logging the same view again gives the same records in the same places
    feats2, tgts2, seen2 = proposal.log_segments(ctx, [cam], tf, p, capacity=1 << 20,
                                                 keep_prob=1.0)
    assert seen2 == seen and torch.equal(feats2, feats) and torch.equal(tgts2, tgts)
    f = feats.cpu().numpy()
    t = tgts.cpu().numpy()
    assert np.all((t >= 0) & (t <= 1))
    assert f[:, :6].min() >= -1e-5 and f[:, :6].max() <= 1 + 1e-5
    assert set(np.unique(f[:, 6])) <= {0.0, 1.0}
    assert np.all((f[:, 7:10] >= 0) & (f[:, 7:10] <= 1)) and np.all(f[:, 7] <= f[:, 8])
    assert np.all(np.abs(f[:, 10:12]) <= 1 + 1e-6)
    # subsampling keeps about the requested fraction
    _, _, seen_half = proposal.log_segments(ctx, [cam], tf, p, capacity=1 << 20, keep_prob=0.5)
    assert abs(seen_half - 0.5 * seen) <= 0.05 * seen


def test_learned_render_with_zero_threshold_is_the_plain_march(mods, c1_learned):
    torch, amr, proposal = mods
    w, ctx = c1_learned
    prop = proposal.Proposal(seed=7)
    prop.install(ctx)
    for shade in (0, 1):
        p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=shade)
        plain, n_plain = gpu_render(ctx, w["camera"], w["tf"], p)
        for mode in (1, 2):
            pl, _ = params_pair(amr, w["vmin"], w["vmax"], shade=shade, learned=mode, tau=0.0)
            img, n = gpu_render(ctx, w["camera"], w["tf"], pl)
            assert np.array_equal(img, plain) and n == n_plain
    # a threshold above every prediction skips everything (every segment asks the MLP)
    pl, _ = params_pair(amr, w["vmin"], w["vmax"], learned=1, tau=1.5, learned_min_samples=1)
    img, n = gpu_render(ctx, w["camera"], w["tf"], pl)
    assert n == 0 and np.all(img == 0)


@pytest.mark.parametrize("size", [(77, 53), (5, 9), (130, 31)])
def test_learned_ragged_images_and_bands(mods, c1_learned, size):
    # images whose sides are no multiple of the warp tile, and a band of rows: with tau = 0
    # the learned march gives the plain march's pixels and sample count there too
    torch, amr, proposal = mods
    w, ctx = c1_learned
    proposal.Proposal(seed=7).install(ctx)
    W, H = size
    cam = synth.orbit_camera(41, W, H)
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1)
    plain, n_plain = gpu_render(ctx, cam, w["tf"], p)
    pl, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, learned=2, tau=0.0)
    img, n = gpu_render(ctx, cam, w["tf"], pl)
    assert np.array_equal(img, plain) and n == n_plain
    if H > 6:
        pb, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, learned=2, tau=0.0, row0=3,
                            rows=H - 5)
        band, _ = gpu_render(ctx, cam, w["tf"], pb)
        assert np.array_equal(band, plain[3:H - 2])


def test_learned_proposal_trains_and_keeps_psnr(mods, c1_learned):
    torch, amr, proposal = mods
    w, ctx = c1_learned
    tf = torch.as_tensor(w["tf"], device="cuda")
    p, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1)
    cams = [synth.orbit_camera(1000 + s, 64, 64) for s in range(48)]
    feats, tgts, seen = proposal.log_segments(ctx, cams, tf, p, capacity=1 << 21, keep_prob=1.0)
    prop = proposal.Proposal(seed=0)

    def full_loss():  # mean cross-entropy over the whole log (the per-epoch figures that
        # train() returns are single minibatches, too noisy to compare)
        prop.loss_grad(feats, tgts)
        torch.cuda.synchronize()
        return float(prop.loss.item())

    before = full_loss()
    prop.train(feats, tgts, epochs=6, batch=4096, lr=3e-3)
    after = full_loss()
    assert after < before, (before, after)
    prop.install(ctx)
    cam = synth.orbit_camera(2000, 256, 256)
    plain, n_plain = gpu_render(ctx, cam, w["tf"], p)
    ps, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, skip=1)
    _, n_minmax = gpu_render(ctx, cam, w["tf"], ps)
    pl, _ = params_pair(amr, w["vmin"], w["vmax"], shade=1, skip=1, learned=1, tau=1e-4)
    img, n = gpu_render(ctx, cam, w["tf"], pl)
    mse = np.mean((img - plain) ** 2)
    psnr = 10 * np.log10(1.0 / mse) if mse > 0 else np.inf
    assert psnr >= 45.0, psnr
    assert n <= n_minmax <= n_plain


def test_coarse_factor_scales_the_sample_count(mods, c1_learned):
    torch, amr, proposal = mods
    from paper_1212_3333_gb300 import _lib

    w, ctx = c1_learned
    proposal.Proposal(seed=7).install(ctx)
    p, _ = params_pair(amr, w["vmin"], w["vmax"], ert_eps=0.0)
    plain, n_plain = gpu_render(ctx, w["camera"], w["tf"], p)
    counts = []
    for cf in (2, 4, 16):
        # tau above every prediction: every segment is sampled coarsely
        pl, _ = params_pair(amr, w["vmin"], w["vmax"], ert_eps=0.0, learned=2, tau=1.5,
                            coarse_factor=cf, learned_min_samples=1)
        img, n = gpu_render(ctx, w["camera"], w["tf"], pl)
        assert np.all(np.isfinite(img))
        counts.append(n)
    assert n_plain > counts[0] > counts[1] > counts[2] > 0
    assert counts[0] >= n_plain / 2 and counts[2] >= n_plain / 16
    for cf in (1, 65):
        pl, _ = params_pair(amr, w["vmin"], w["vmax"], learned=2, tau=0.5, coarse_factor=cf)
        with pytest.raises(amr.AmrError) as e:
            gpu_render(ctx, w["camera"], w["tf"], pl)
        assert e.value.status == _lib.AMR_ERR_ARG


def test_gradient_is_deterministic(mods):
    # the blocks' partial sums are added in a fixed order, so repeated calls on the same
    # inputs give the same gradient and loss bit for bit (no atomics in the reduction)
    torch, amr, proposal = mods
    rng = np.random.default_rng(12)
    x = torch.as_tensor(rng.uniform(0, 1, size=(60000, 12)).astype(np.float32), device="cuda")
    t = torch.as_tensor(rng.uniform(0, 1, size=60000).astype(np.float32), device="cuda")
    prop = proposal.Proposal(seed=5)
    out = []
    for _ in range(3):
        prop.loss_grad(x, t, 0, 60000, 7, 11)
        torch.cuda.synchronize()
        out.append((prop.grad.clone(), prop.loss.clone()))
    for g, l in out[1:]:
        assert torch.equal(g, out[0][0]) and torch.equal(l, out[0][1])
    assert float(out[0][1].item()) > 0.0


def test_checkpoint_resume_continues_training(mods, tmp_path):
    torch, amr, proposal = mods
    rng = np.random.default_rng(8)
    x = torch.as_tensor(rng.uniform(0, 1, size=(4096, 12)).astype(np.float32), device="cuda")
    t = torch.as_tensor(rng.uniform(0, 1, size=4096).astype(np.float32) ** 3, device="cuda")
    a = proposal.Proposal(seed=3)
    a.train(x, t, epochs=2, batch=1024, lr=1e-3)
    path = str(tmp_path / "ckpt.npz")
    a.save(path)
    b = proposal.Proposal.load(path)
    for p in (a, b):
        p.loss_grad(x, t, 0, 1024, 1, 0)
        p.adam(1e-3)
    torch.cuda.synchronize()
    assert a.step == b.step == 9
    # the gradient's partial sums are added in a fixed order: resuming is exact
    for u, w in ((a.params, b.params), (a.m, b.m), (a.v, b.v)):
        assert torch.equal(u, w)


def test_learned_min_samples_limits_the_proposal(mods, c1_learned):
    # segments shorter than learned_min_samples are sampled as the plain march samples
    # them: with tau above every prediction, only the longer segments are skipped
    torch, amr, proposal = mods
    from paper_1212_3333_gb300 import _lib

    w, ctx = c1_learned
    proposal.Proposal(seed=7).install(ctx)
    p, _ = params_pair(amr, w["vmin"], w["vmax"], ert_eps=0.0)
    _, n_plain = gpu_render(ctx, w["camera"], w["tf"], p)
    kept = []
    for m in (1, 4, 16, 1 << 22):
        pl, _ = params_pair(amr, w["vmin"], w["vmax"], ert_eps=0.0, learned=1, tau=1.5,
                            learned_min_samples=m)
        _, n = gpu_render(ctx, w["camera"], w["tf"], pl)
        kept.append(n)
    assert kept[0] == 0 and kept[0] < kept[1] < kept[2] <= kept[3] == n_plain
    for m in (0, (1 << 22) + 1):
        pl, _ = params_pair(amr, w["vmin"], w["vmax"], learned=1, learned_min_samples=m)
        with pytest.raises(amr.AmrError) as e:
            gpu_render(ctx, w["camera"], w["tf"], pl)
        assert e.value.status == _lib.AMR_ERR_ARG
