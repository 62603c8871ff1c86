"""Differentiation form: stored decoder activations versus recomputation in the backward pass.

With store_activations the forward pass writes every sample's decoder inputs and
activations and the backward pass reads them instead of gathering and decoding again.
Both forms compute the same arithmetic, so their gradients agree to summation order, and
both agree with the FP64 oracle within the parity tolerances.
"""
import numpy as np
import pytest
import torch

import paper_2206_14735_gb300 as gs
import scenegen as sg
from gpu_common import LOSS_RTOL, Problem, assert_grad_close, prepare_parity_batch, upload_oracle_batch
from helpers import CUBE, sdf_parity_params

pytestmark = pytest.mark.gpu

SEED, STEP = 3, 5


@pytest.fixture(scope="module")
def case():
    p = Problem(CUBE)
    theta = sdf_parity_params(CUBE, sg.cube_scene(), seed=21)
    bt, sm = p.oracle_sample(SEED, STEP)
    bt_s, ref, _ = prepare_parity_batch(p, theta, bt, sm, max_drop=0.05, min_switch=0.25, label="store cube")
    batch = upload_oracle_batch(bt_s, sm, sm["n_valid"][0])
    store_ctx = gs.Context(CUBE, store_activations=True)
    return dict(p=p, theta=theta, ref=ref, batch=batch, store_ctx=store_ctx)


def _split(ctx, th, batch, dloss=None):
    loss = torch.empty(6, device="cuda")
    grad = torch.zeros_like(th)
    ctx.forward(th, batch, loss)
    ctx.backward(th, batch, dloss, grad)
    torch.cuda.synchronize()
    return loss.cpu().numpy().astype(np.float64), grad.cpu().numpy()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-30)


def test_store_split_matches_recompute_and_oracle(case):
    th = torch.from_numpy(case["theta"]).cuda()
    l_s, g_s = _split(case["store_ctx"], th, case["batch"])
    l_r, g_r = _split(case["p"].ctx, th, case["batch"])
    np.testing.assert_allclose(l_s, l_r, rtol=1e-6)  # the same forward kernel; only summation order differs
    assert _rel(g_s, g_r) < 1e-5
    for k in range(6):
        assert abs(l_s[k] - case["ref"]["loss"][k]) <= LOSS_RTOL * abs(case["ref"]["loss"][k])
    assert_grad_close(case["p"], g_s, case["ref"]["grad"])


def test_store_fused_matches_oracle(case):
    th = torch.from_numpy(case["theta"]).cuda()
    loss = torch.empty(6, device="cuda")
    grad = torch.zeros_like(th)
    case["store_ctx"].forward_backward(th, case["batch"], None, loss, grad)
    torch.cuda.synchronize()
    got = loss.cpu().numpy().astype(np.float64)
    for k in range(6):
        assert abs(got[k] - case["ref"]["loss"][k]) <= LOSS_RTOL * abs(case["ref"]["loss"][k])
    assert_grad_close(case["p"], grad.cpu().numpy(), case["ref"]["grad"])


def test_store_autograd_function(case):
    th = torch.from_numpy(case["theta"]).cuda().requires_grad_(True)
    losses = gs.GoSurfStep.apply(th, case["store_ctx"], case["batch"])
    losses[5].backward()
    assert_grad_close(case["p"], th.grad.cpu().numpy(), case["ref"]["grad"])


def test_store_backward_needs_a_matching_forward(case):
    th = torch.from_numpy(case["theta"]).cuda()
    ctx = gs.Context(CUBE, store_activations=True)
    grad = torch.zeros_like(th)
    with pytest.raises(gs.GoSurfError):
        ctx.backward(th, case["batch"], None, grad)  # nothing stored yet
    loss = torch.empty(6, device="cuda")
    ctx.forward(th, case["batch"], loss)
    other = gs.Batch.allocate(case["batch"].R, case["batch"].N, case["batch"].P)
    with pytest.raises(gs.GoSurfError):
        ctx.backward(th, other, None, grad)  # another batch's activations are not there
    ctx.backward(th, case["batch"], None, grad)
    torch.cuda.synchronize()
    ctx.close()


def test_store_sampled_batch_room_scale():
    """A sampled room batch at full size: store and recompute agree (no oracle at this size)."""
    w = sg.WORKLOADS["room-diff-65536x96"]
    frames = sg.make_frames(w, n_frames=8)
    dfr = gs.DeviceFrames(frames.rgb, frames.depth, frames.c2w, frames.fx, frames.fy, frames.cx, frames.cy)
    theta = torch.from_numpy(sg.init_params(w, seed=1).astype(np.float32)).cuda()
    res = []
    for store in (False, True):
        ctx = gs.Context(w, store_activations=store)
        b = gs.Batch.allocate(w.rays, w.n_samples, w.n_smooth)
        ctx.sample_rays(dfr, 7, 0, b)
        res.append(_split(ctx, theta, b))
        ctx.close()
    np.testing.assert_allclose(res[0][0], res[1][0], rtol=1e-6)
    assert _rel(res[1][1], res[0][1]) < 1e-5
