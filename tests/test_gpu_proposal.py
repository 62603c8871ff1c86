"""Learned proposal sampler (an addition to the method) on the GPU versus the oracle:
ray selection and the inverse-CDF sampler bit for bit given the same PDF, the network's PDF
within FP32 rounding, the rendering weights the forward pass writes, and the cross-entropy
gradient of the proposal network."""
import numpy as np
import pytest
import torch

import oracle as oc
import paper_2206_14735_gb300 as gs
import scenegen as sg
from gpu_common import Problem, prepare_parity_batch, upload_oracle_batch
from helpers import CUBE, sdf_parity_params

pytestmark = pytest.mark.gpu

CUBE_P = CUBE.with_(name="cube-prop", prop_samples=32, prop_guided=8)
SEED, STEP = 4, 7


def _q(seed=3, scale=0.3):
    return np.random.default_rng(seed).normal(0.0, scale, oc.PROP_PARAMS).astype(np.float32)


@pytest.fixture(scope="module")
def prob():
    p = Problem(CUBE_P, max_rays=4096)
    # the proposal network's own hidden units switch (q ~ N(0, 0.3)); the main decoder's masks
    # are not what these tests are about, so its parameters keep every unit clear of its kink
    theta = sg.sdf_params(CUBE_P, sg.cube_scene(), seed=21)
    theta[:p.n_grid] += np.random.default_rng(5).normal(0, 0.2, p.n_grid).astype(np.float32)  # coarse features vary
    return dict(p=p, theta=theta, q=_q())


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint32)


def _gpu_prop_sample(pr, R, P, pdf_in=None, with_net=True):
    p = pr["p"]
    b = gs.Batch.allocate(R, CUBE_P.prop_samples, P, weights=True)
    th = torch.from_numpy(pr["theta"]).cuda()
    q = torch.from_numpy(pr["q"]).cuda()
    pdf_out = torch.empty(max(R, 1), oc.PROP_BINS, device="cuda")
    pin = None if pdf_in is None else torch.from_numpy(np.ascontiguousarray(pdf_in, np.float32)).cuda()
    p.ctx.proposal_sample(p.dfr, SEED, STEP, b, theta=th if with_net else None, prop=q if with_net else None,
                          pdf_in=pin, pdf_out=pdf_out)
    torch.cuda.synchronize()
    return b, pdf_out[:R].cpu().numpy()


@pytest.mark.parametrize("R", [1000, 33, 1, 0])
def test_rays_and_inverse_cdf_bit_exact_given_the_pdf(prob, R):
    p = prob["p"]
    bt, sm = p.oracle_sample(SEED, STEP, R, 64)
    # the PDF both sides sample from: the oracle network's, rounded to binary32
    pdf = oc.prop_forward(p.cfg, prob["theta"], prob["q"], bt["o"], bt["r"]).astype(np.float32)
    b, used = _gpu_prop_sample(prob, R, 64, pdf_in=pdf, with_net=False)
    assert np.array_equal(b.pix.cpu().numpy(), bt["pix"])
    for gk, ok in (("origin", "o"), ("dir", "r"), ("rgb", "rgb"), ("depth", "D")):
        assert np.array_equal(_bits(getattr(b, gk).cpu().numpy()), _bits(bt[ok])), gk
    assert np.array_equal(_bits(used), _bits(pdf))
    ref = oc.prop_sample(p.cfg, bt["D"], pdf, CUBE_P.prop_samples, CUBE_P.prop_guided, SEED, STEP)
    assert np.array_equal(_bits(b.t.cpu().numpy()), _bits(ref["t"]))
    assert np.array_equal(b.cls.cpu().numpy(), ref["cls"])
    assert list(b.counts.cpu().numpy()[:3]) == list(ref["counts"][:3])
    # smoothness points are the plain sampler's
    assert np.array_equal(_bits(b.xs[:64].cpu().numpy()), _bits(sm["xs"]))


def test_network_pdf_parity(prob):
    p = prob["p"]
    bt, _ = p.oracle_sample(SEED, STEP, 2000, 0)
    _, pdf = _gpu_prop_sample(prob, 2000, 0)
    ref = oc.prop_forward(p.cfg, prob["theta"], prob["q"], bt["o"], bt["r"])
    np.testing.assert_allclose(pdf, ref, rtol=2e-5, atol=1e-7)
    np.testing.assert_allclose(pdf.sum(1), 1.0, atol=2e-6)


def test_forward_writes_rendering_weights(prob):
    """batch.w after gs_forward equals the oracle's w_i = T_i alpha_i on a parity batch."""
    p = prob["p"]
    theta = sdf_parity_params(CUBE, sg.cube_scene(), seed=21)
    bt, sm = p.oracle_sample(3, 5)
    bt_s, _, _ = prepare_parity_batch(p, theta, bt, sm)
    ref = oc.step(p.cfg, theta, bt_s, sm, want_grad=False, want_weights=True)
    b = upload_oracle_batch(bt_s, sm, sm["n_valid"][0])
    b.w = torch.zeros_like(b.t)
    loss = torch.empty(6, device="cuda")
    p.ctx.forward(torch.from_numpy(theta).cuda(), b, loss)
    torch.cuda.synchronize()
    # alpha = (Phi_i - Phi_i+1) / Phi_i loses relative precision in binary32 when the two
    # opacities are close, so the bound is relative as well as absolute
    np.testing.assert_allclose(b.w.cpu().numpy(), ref["w"], rtol=1e-4, atol=2e-6)


def test_cross_entropy_gradient_parity(prob):
    p = prob["p"]
    R = 3000
    bt, _ = p.oracle_sample(SEED, STEP, R, 0)
    pdf = oc.prop_forward(p.cfg, prob["theta"], prob["q"], bt["o"], bt["r"]).astype(np.float32)
    b, _ = _gpu_prop_sample(prob, R, 0, pdf_in=pdf, with_net=False)
    ref_s = oc.prop_sample(p.cfg, bt["D"], pdf, CUBE_P.prop_samples, CUBE_P.prop_guided, SEED, STEP)
    # target weights: peaked per ray, some rays below the 1e-3 threshold (skipped)
    rng = np.random.default_rng(9)
    w = rng.dirichlet(np.full(CUBE_P.prop_samples, 0.2), R) * rng.uniform(0.2, 1.0, (R, 1))
    w[::17] *= 1e-4
    w = w.astype(np.float32)
    b.w.copy_(torch.from_numpy(w))
    grad = torch.zeros(oc.PROP_PARAMS, device="cuda")
    ce = torch.zeros(2, device="cuda")
    th = torch.from_numpy(prob["theta"]).cuda()
    q = torch.from_numpy(prob["q"]).cuda()
    p.ctx.proposal_backward(th, q, b, grad, ce)
    torch.cuda.synchronize()
    loss, g_ref, n_used = oc.prop_ce(p.cfg, prob["theta"], prob["q"], bt["o"], bt["r"], ref_s["t"], w)
    ce_h = ce.cpu().numpy()
    assert int(ce_h[1]) == n_used
    assert abs(ce_h[0] - loss) <= 1e-5 * abs(loss)
    g = grad.cpu().numpy().astype(np.float64)
    blocks = [("W1", 0, 352), ("b1", 352, 384), ("W2", 384, 1408), ("b2", 1408, 1440), ("w3", 1440, 1472)]
    for name, a, e in blocks:
        scale = np.abs(g_ref[a:e]).max()
        assert np.abs(g[a:e] - g_ref[a:e]).max() <= 1e-4 * scale, name
    # d/d b3 = sum_b (p_b - hh_b) / n = 0 for every ray (both distributions sum to one)
    assert abs(g_ref[1472]) < 1e-12 and abs(g[1472]) < 1e-6


def test_proposal_entry_points_reject_bad_shapes(prob):
    p = prob["p"]
    b = gs.Batch.allocate(8, CUBE_P.n_samples, 0)  # plain N, not prop_samples
    with pytest.raises(gs.GoSurfError):
        p.ctx.proposal_sample(p.dfr, 1, 1, b, theta=torch.from_numpy(prob["theta"]).cuda(),
                              prop=torch.from_numpy(prob["q"]).cuda())
    bp = gs.Batch.allocate(8, CUBE_P.prop_samples, 0)
    with pytest.raises(gs.GoSurfError):
        p.ctx.sample_rays(p.dfr, 1, 1, bp)  # the plain sampler writes n_strat + n_guided samples
    with pytest.raises(gs.GoSurfError):  # no weights to learn from
        p.ctx.proposal_backward(torch.from_numpy(prob["theta"]).cuda(), torch.from_numpy(prob["q"]).cuda(), bp,
                                torch.zeros(oc.PROP_PARAMS, device="cuda"))


def test_bf16_trainer_reads_the_bf16_copy_and_trains():
    """The BF16 proposal form: every main-model call of the trainer (fused step, held-out
    renders, Adam) takes the bfloat16 grid copy, which Adam keeps equal to the RNE copy of
    theta; the proposal's cross entropy falls and the main loss stays finite."""
    from paper_2206_14735_gb300.proposal import ProposalTrainer
    w = CUBE_P.with_(name="cube-prop-bf16", precision="bf16", prop_guided=24, rays=512, n_smooth=64)
    p = Problem(w)
    theta = torch.from_numpy(sg.init_params(w)).cuda()
    grad, m, v = torch.zeros_like(theta), torch.zeros_like(theta), torch.zeros_like(theta)
    mirror = theta[:p.n_grid].to(torch.bfloat16).view(torch.int16).contiguous()
    tr = ProposalTrainer(p.ctx, w, p.dfr, seed=5, eval_every=10, mirror=mirror)
    loss = torch.empty(6, device="cuda")
    ce = []
    for k in range(60):
        tr.step(k, theta, grad, m, v, loss)
        if k in (0, 59):
            ce.append(float(tr.ce[0].item()))
    torch.cuda.synchronize()
    p.ctx.sync_status()
    assert np.all(np.isfinite(loss.cpu().numpy()))
    assert ce[1] < ce[0]
    assert len(tr.controller.history) == 6
    want = theta[:p.n_grid].to(torch.bfloat16).view(torch.int16)
    assert torch.equal(mirror, want)
    # without the copy the BF16 context refuses the render call
    with pytest.raises(gs.GoSurfError, match="theta_bf16"):
        p.ctx.forward_backward(theta, tr.batch_plain, None, loss, grad)


def _depth_l1_dropped(ctx, w, dfr, gt, theta, q=None, R=8192, seed=991):
    """Rendered depth of R fresh rays (the proposal's samples when q is given, the plain
    sampler's otherwise) against the noise-free depth, on the rays whose observed depth is
    missing (dropped in a blob) but whose pixel sees a surface."""
    if q is None:
        b = gs.Batch.allocate(R, w.n_strat + w.n_guided, 0)
        ctx.sample_rays(dfr, seed, 0, b)
    else:
        b = gs.Batch.allocate(R, w.prop_samples, 0)
        ctx.proposal_sample(dfr, seed, 0, b, theta=theta, prop=q)
    loss = torch.empty(6, device="cuda")
    dh = torch.empty(R, device="cuda")
    ctx.forward(theta, b, loss, d_hat=dh)
    torch.cuda.synchronize()
    pix = b.pix.cpu().numpy()
    g = gt.reshape(-1)[pix].astype(np.float64)
    D = b.depth.cpu().numpy()
    drop = (g > 0) & (D <= 0)
    return float(np.abs(dh.cpu().numpy().astype(np.float64) - g)[drop].mean()), int(drop.sum())


def test_trained_proposal_beats_the_plain_sampler_where_depth_is_missing():
    """What the learned proposal gains over the method without it.  A blob-dropout scene (30 %
    of the depth pixels zeroed in discs); both forms take 32 samples per ray and are trained
    for the same number of steps from the same initial parameters: the plain form with 24
    stratified + 8 depth-guided samples, the proposal form with 24 proposal + 8 guided samples
    (the plain 32 as its fallback, the controller deciding).  Where the observed depth is
    missing the plain sampler has no guided samples, only 32 strata over [near, far]; the
    proposal, trained on the model's own rendering weights, puts its samples near the surface,
    so its rendered depth there must come out closer to the true depth."""
    from paper_2206_14735_gb300.proposal import ProposalTrainer
    w = CUBE.with_(name="cube-blob-prop", frames=8, rays=2048, n_strat=24, n_guided=8, blob_frac=0.3,
                   prop_samples=32, prop_guided=8, n_smooth=1024)
    fr = sg.make_frames(w, with_gt=True)
    dfr = gs.DeviceFrames(fr.rgb, fr.depth, fr.c2w, fr.fx, fr.fy, fr.cx, fr.cy)
    steps = 1500
    theta0 = torch.from_numpy(sg.init_params(w)).cuda()
    res = {}
    for form in ("plain", "proposal"):
        ctx = gs.Context(w, max_rays=8192)
        theta = theta0.clone()
        grad, m, v = torch.zeros_like(theta), torch.zeros_like(theta), torch.zeros_like(theta)
        loss = torch.empty(6, device="cuda")
        if form == "plain":
            b = gs.Batch.allocate(w.rays, w.n_samples, w.n_smooth)
            for k in range(steps):
                ctx.sample_rays(dfr, 5, k, b)
                ctx.forward_backward(theta, b, None, loss, grad)
                ctx.adam_step(theta, grad, m, v, k + 1, w.lr_grid, w.lr_mlp, w.betas[0], w.betas[1], w.adam_eps)
            res[form] = _depth_l1_dropped(ctx, w, dfr, fr.gt_depth, theta)
        else:
            tr = ProposalTrainer(ctx, w, dfr, seed=5, holdout=512)
            for k in range(steps):
                tr.step(k, theta, grad, m, v, loss)
            res[form] = _depth_l1_dropped(ctx, w, dfr, fr.gt_depth, theta, q=tr.q)
            res["proposal_steps"] = sum(1 for h in tr.controller.history if h[2]) * tr.eval_every
            res["ce"] = float(tr.ce[0].item())
        ctx.sync_status()
        ctx.close()
    print(f"\ndepth L1 on rays with missing depth after {steps} steps at 32 samples per ray: "
          f"plain {res['plain'][0]:.4f} m ({res['plain'][1]} rays), proposal {res['proposal'][0]:.4f} m "
          f"({res['proposal'][1]} rays); about {res['proposal_steps']} steps on the proposal; CE {res['ce']:.3f}")
    assert res["plain"][1] > 200 and res["proposal"][1] > 200
    assert res["proposal"][0] < 0.8 * res["plain"][0], res


# ---- the BF16 form: the network's layers on the tensor core (bfloat16 operands) ----------
CUBE_PB = CUBE_P.with_(name="cube-prop-bf16", precision="bf16")


def _bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).float().numpy()


def _q_bf16(q):
    """The proposal parameters with the matrices the tensor core reads (W1, W2) rounded to
    bfloat16, as the oracle's reference for the BF16 form (reading R44)."""
    qq = q.copy()
    qq[0:352] = _bf16(qq[0:352])
    qq[384:1408] = _bf16(qq[384:1408])
    return qq


@pytest.fixture(scope="module")
def prob_bf16(prob):
    p = Problem(CUBE_PB, max_rays=4096)
    return dict(p=p, theta=prob["theta"], q=_q_bf16(prob["q"]))


def test_bf16_network_pdf_and_draws(prob_bf16):
    """PDF of the tensor-core network against the oracle's on the bfloat16-rounded weights:
    what remains is the bfloat16 rounding of the inputs and of the first hidden layer (about
    2^-9 relative each, through the logits into the softmax); measured 7.5e-3 of a bin's
    probability at most (p > 1e-3) and 2.7e-4 absolute, bounded at 1.5e-2 of each bin's
    probability plus 3e-4; the draws from the kernel's own PDF are the oracle's to the bit."""
    pr = prob_bf16
    p = pr["p"]
    R = 2000
    bt, _ = p.oracle_sample(SEED, STEP, R, 0)
    b, pdf = _gpu_prop_sample(pr, R, 0)
    ref = oc.prop_forward(p.cfg, pr["theta"], pr["q"], bt["o"], bt["r"])
    err = np.abs(pdf - ref)
    print(f"\nBF16 proposal PDF vs oracle: max abs {err.max():.2e}, max rel (p > 1e-3) "
          f"{(err / np.maximum(ref, 1e-3)).max():.2e}, mean abs {err.mean():.2e}")
    assert np.all(err <= 1.5e-2 * ref + 3e-4)
    np.testing.assert_allclose(pdf.sum(1), 1.0, atol=2e-6)
    ref_s = oc.prop_sample(p.cfg, bt["D"], pdf, CUBE_PB.prop_samples, CUBE_PB.prop_guided, SEED, STEP)
    assert np.array_equal(_bits(b.t.cpu().numpy()), _bits(ref_s["t"]))
    assert np.array_equal(b.cls.cpu().numpy(), ref_s["cls"])


def test_bf16_cross_entropy_gradient(prob_bf16):
    """Cross-entropy gradient of the tensor-core network against the oracle's on the
    bfloat16-rounded weights, per parameter block.  The bfloat16 rounding of the inputs, the
    first hidden layer and the second layer's adjoint (2^-9 relative each) gave max-norm
    errors of 1.2e-2 (W1), 1.7e-2 (b1: a sum of adjoints that cancel), 6e-3 (W2, b2) and
    7e-4 (w3, whose adjoint is the FP32 softmax residual); the bounds are about twice those.
    The cross entropy itself came within 7e-6 relative (bound 3e-5: a mean over all bins
    whose rounding errors partly cancel, so more headroom)."""
    pr = prob_bf16
    p = pr["p"]
    R = 3000
    bt, _ = p.oracle_sample(SEED, STEP, R, 0)
    pdf = oc.prop_forward(p.cfg, pr["theta"], pr["q"], bt["o"], bt["r"]).astype(np.float32)
    b, _ = _gpu_prop_sample(pr, R, 0, pdf_in=pdf, with_net=False)
    ref_s = oc.prop_sample(p.cfg, bt["D"], pdf, CUBE_PB.prop_samples, CUBE_PB.prop_guided, SEED, STEP)
    rng = np.random.default_rng(9)
    w = rng.dirichlet(np.full(CUBE_PB.prop_samples, 0.2), R) * rng.uniform(0.2, 1.0, (R, 1))
    w[::17] *= 1e-4
    w = w.astype(np.float32)
    b.w.copy_(torch.from_numpy(w))
    grad = torch.zeros(oc.PROP_PARAMS, device="cuda")
    ce = torch.zeros(2, device="cuda")
    p.ctx.proposal_backward(torch.from_numpy(pr["theta"]).cuda(), torch.from_numpy(pr["q"]).cuda(), b, grad, ce)
    torch.cuda.synchronize()
    p.ctx.sync_status()
    loss, g_ref, n_used = oc.prop_ce(p.cfg, pr["theta"], pr["q"], bt["o"], bt["r"], ref_s["t"], w)
    ce_h = ce.cpu().numpy()
    assert int(ce_h[1]) == n_used
    g = grad.cpu().numpy().astype(np.float64)
    errs = {}
    for name, a, e in [("W1", 0, 352), ("b1", 352, 384), ("W2", 384, 1408), ("b2", 1408, 1440), ("w3", 1440, 1472)]:
        errs[name] = float(np.abs(g[a:e] - g_ref[a:e]).max() / np.abs(g_ref[a:e]).max())
    print(f"\nBF16 proposal CE {ce_h[0]:.6f} vs {loss:.6f} (rel {abs(ce_h[0] - loss) / loss:.2e}); "
          f"gradient max-norm errors {errs}")
    assert abs(ce_h[0] - loss) <= 3e-5 * abs(loss)
    for name, bound in (("W1", 2.5e-2), ("b1", 3.5e-2), ("W2", 1.2e-2), ("b2", 1.2e-2), ("w3", 1.5e-3)):
        assert errs[name] <= bound, (name, errs)
