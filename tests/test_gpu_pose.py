"""Camera-pose refinement on the GPU (gs_pose_apply, the dL/dz export of the backward pass,
gs_pose_backward) against the FP64 oracle, and pose recovery from perturbed poses."""
import numpy as np
import pytest
import torch

import oracle as oc
import paper_2206_14735_gb300 as gs
import scenegen as sg
from gpu_common import Problem, prepare_parity_batch, upload_oracle_batch
from helpers import CUBE, sdf_parity_params

pytestmark = pytest.mark.gpu
W3 = CUBE.with_(name="cube-3frames", frames=3)


@pytest.fixture(scope="module")
def posed():
    p = Problem(W3)
    rng = np.random.default_rng(5)
    xi = np.c_[rng.normal(0, 0.01, (3, 3)), rng.normal(0, 0.01, (3, 3))]
    c2w = oc.pose_apply(p.frames.c2w, xi)
    F = oc.OcFramesHolder(p.frames, c2w=c2w)
    theta = sdf_parity_params(W3, sg.cube_scene(), seed=21)
    return p, xi, c2w, F, theta


def test_pose_apply_matches_oracle(posed):
    p, xi, c2w, F, theta = posed
    out = torch.empty((3, 3, 4), device="cuda")
    p.ctx.pose_apply(torch.from_numpy(p.frames.c2w).cuda(), torch.from_numpy(xi.astype(np.float32)).cuda(), out)
    np.testing.assert_allclose(out.cpu().numpy(), c2w, atol=2e-6)


def test_dz_export_and_pose_gradient_match_oracle(posed):
    p, xi, c2w, F, theta = posed
    bt = oc.sample_rays(p.cfg, F, 9, 2, W3.rays)
    sm = oc.sample_smooth(p.cfg, F, 9, 2, W3.n_smooth)
    bt_s, ref, _ = prepare_parity_batch(p, theta, bt, sm)
    ref_dz = oc.step_dz(p.cfg, theta, bt_s, sm)["dz"]
    g_ref = oc.pose_grad(p.cfg, F, theta, c2w, xi, bt_s, ref_dz)
    batch = upload_oracle_batch(bt_s, sm, sm["n_valid"][0])
    batch.dz = torch.zeros(batch.R, batch.N, 16, device="cuda")
    th = torch.from_numpy(theta).cuda()
    loss = torch.empty(6, device="cuda")
    grad = torch.zeros_like(th)
    p.ctx.forward_backward(th, batch, None, loss, grad)
    dz = batch.dz.cpu().numpy().astype(np.float64)
    # per sample (no summation over samples as in the parameter gradients): the FP32-grade
    # tensor-core adjoint chain, a few 1e-5 of the largest element; 1e-3 allowed
    scale = np.abs(ref_dz).max()
    assert np.abs(dz - ref_dz).max() <= 1e-3 * scale, np.abs(dz - ref_dz).max() / scale
    c2w_dev = torch.from_numpy(c2w.astype(np.float32)).cuda()
    dfr = p.dfr.with_poses(c2w_dev)
    pg = torch.zeros(3, 6, device="cuda")
    p.ctx.pose_backward(th, dfr, torch.from_numpy(xi.astype(np.float32)).cuda(), batch, pg)
    torch.cuda.synchronize()
    p.ctx.sync_status()
    g = pg.cpu().numpy().astype(np.float64)
    assert np.abs(g_ref).max() > 1e-3
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max(), (g, g_ref)


@pytest.mark.parametrize("records", [False, True])
def test_eikonal_pose_gradient_matches_oracle(posed, records):
    """The Eikonal term's pose gradient (x-Hessian of phi through the free-space samples'
    positions) against the oracle's, on hidden units that switch from sample to sample; rays
    holding a free-space sample within binary32 rounding of a ReLU kink are left out (the
    term jumps there).  With records, d phi / d z comes from the batch's deferred Eikonal
    records, which an Eikonal call on the batch writes first."""
    from gpu_common import drop_kink_rays
    p, xi, c2w, F, theta = posed
    bt = oc.sample_rays(p.cfg, F, 9, 2, W3.rays)
    bt, dropped = drop_kink_rays(p, theta, bt)
    assert dropped <= 0.05 * W3.rays
    assert int(bt["counts"][2]) > 1000
    for dscale in (1.0, -0.75):
        g_ref = oc.eikonal_pose_grad(p.cfg, F, theta, c2w, xi, bt, dscale)
        batch = upload_oracle_batch(bt, None, 0)
        if records:
            batch.eik = torch.full((5, batch.R, batch.N, 4), float("nan"), device="cuda")
            p.ctx.eikonal(torch.from_numpy(theta).cuda(), batch, loss=torch.empty(1, device="cuda"))
        dfr = p.dfr.with_poses(torch.from_numpy(c2w.astype(np.float32)).cuda())
        pg = torch.zeros(3, 6, device="cuda")
        dl = None if dscale == 1.0 else torch.tensor([dscale], dtype=torch.float32, device="cuda")
        p.ctx.eikonal_pose_backward(torch.from_numpy(theta).cuda(), dfr, torch.from_numpy(xi.astype(np.float32)).cuda(),
                                    batch, pg, dloss=dl)
        torch.cuda.synchronize()
        p.ctx.sync_status()
        g = pg.cpu().numpy().astype(np.float64)
        assert np.abs(g_ref).max() > 1e-4
        assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max(), (g, g_ref)


def test_pose_backward_empty_batch(posed):
    p, xi, c2w, F, theta = posed
    b = gs.Batch.allocate(0, W3.n_samples, 0, dz=True)
    pg = torch.zeros(3, 6, device="cuda")
    p.ctx.pose_backward(torch.from_numpy(theta).cuda(), p.dfr, torch.zeros(3, 6, device="cuda"), b, pg)
    torch.cuda.synchronize()
    assert not torch.any(pg)


def test_pose_refinement_reduces_the_pose_error():
    """Frames rendered from the true poses; the optimisation starts from poses off by about
    1.5 degrees and 3 cm, with the scene's SDF baked into the finest level as the model (held
    fixed, sharpness s = 2000 so that the rendered depth sits at the zero crossing).  Adam on
    (dt, nu) at the paper's learning rate 5e-4, driven by the depth and truncated-SDF terms,
    halves the depth loss and moves the poses towards the true ones; what remains is of the
    order of the model's own error (an 8 cm trilinear SDF, samples 1-6 cm apart)."""
    import math
    w = W3.with_(rays=2048, n_smooth=0)
    p = Problem(w)
    th = sdf_parity_params(w, sg.cube_scene(), seed=21, mix=0.0, phi_shift=0.0)
    th[-1] = math.log(2000.0)
    theta = torch.from_numpy(th).cuda()
    rng = np.random.default_rng(11)
    true_xi = np.c_[rng.normal(0, 0.02, (3, 3)), rng.normal(0, 0.015, (3, 3))]
    # c2w0 = the true poses with the correction taken out: xi = true_xi gives them back
    true_c2w = p.frames.c2w.astype(np.float64)
    R_off = oc.pose_apply(np.tile(np.c_[np.eye(3), np.zeros(3)][None], (3, 1, 1)).astype(np.float32),
                          np.c_[np.zeros((3, 3)), true_xi[:, 3:]])[:, :, :3]
    c2w0 = np.empty((3, 3, 4), np.float32)
    for f in range(3):
        c2w0[f, :, :3] = true_c2w[f, :, :3] @ R_off[f].T
        c2w0[f, :, 3] = true_c2w[f, :, 3] - true_xi[f, :3]
    c2w0_dev = torch.from_numpy(c2w0).cuda()
    xi = torch.zeros(4 * 5, device="cuda")  # 3 x 6 used, padded to a multiple of 4 for Adam
    m, v, gxi = torch.zeros_like(xi), torch.zeros_like(xi), torch.zeros_like(xi)
    c2w = torch.empty((3, 3, 4), device="cuda")
    batch = gs.Batch.allocate(w.rays, w.n_samples, 0, dz=True)
    loss = torch.empty(6, device="cuda")
    gth = torch.zeros_like(theta)
    dl = torch.tensor([0.0, 1.0, 1.0, 0.0, 0.0, 0.0], device="cuda")  # depth and truncated SDF
    first = None
    for k in range(700):
        x6 = xi[:18].view(3, 6)
        p.ctx.pose_apply(c2w0_dev, x6, c2w)
        dfr = p.dfr.with_poses(c2w)
        p.ctx.sample_rays(dfr, 4, k, batch)
        p.ctx.forward_backward(theta, batch, dl, loss, gth)
        if first is None:
            first = float(loss[1].item())
        p.ctx.pose_backward(theta, dfr, x6, batch, gxi[:18].view(3, 6))
        p.ctx.adam_step(xi, gxi, m, v, k + 1, 0.0, 5e-4, n_grid=0)
    torch.cuda.synchronize()
    p.ctx.sync_status()
    e = np.abs(xi[:18].view(3, 6).cpu().numpy() - true_xi)
    e0 = np.abs(true_xi)
    last = float(loss[1].item())
    assert last < 0.5 * first, (first, last)
    assert e[:, :3].max() < 0.75 * e0[:, :3].max(), (e[:, :3].max(), e0[:, :3].max())
    assert e[:, 3:].max() < e0[:, 3:].max(), (e[:, 3:].max(), e0[:, 3:].max())
