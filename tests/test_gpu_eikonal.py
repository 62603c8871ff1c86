"""Eikonal term (gs_eikonal, Sec. 3.3 Eq. eikonal_loss on S_fs) against the FP64 oracle:
loss and parameter gradient on sampled batches of the cube workload (several tiles and
ragged tails), the degenerate cases, the room workload at its full batch and grid, and the
deferred form (grid part added by the render call's scatter from per-sample records)."""
import numpy as np
import pytest
import torch

import oracle as oc
import scenegen as sg
from gpu_common import (LOSS_RTOL, Problem, assert_grad_close, drop_kink_rays, prepare_parity_batch,
                        switching_fraction, upload_oracle_batch)
from helpers import CUBE, sdf_parity_params

pytestmark = pytest.mark.gpu
SEED = 2024
NO_COLOUR = ("W3", "b3", "W4", "b4", "kappa")


def _gpu(p, theta, batch, want_grad=True, dloss=None, want_loss=True):
    th = torch.from_numpy(theta).cuda()
    loss = torch.full((1,), float("nan"), device="cuda") if want_loss else None
    grad = torch.zeros_like(th) if want_grad else None
    dl = None if dloss is None else torch.tensor([dloss], dtype=torch.float32, device="cuda")
    p.ctx.eikonal(th, batch, loss=loss, grad=grad, dloss=dl)
    torch.cuda.synchronize()
    return (float(loss.item()) if want_loss else None), (grad.cpu().numpy() if want_grad else None)


def _loss_tol(ref_loss, gnorm):
    """|Delta L_eik| allowed for a binary32 evaluation of grad_x phi.

    Each |g| carries a relative error of at most about 1e-5 (a 48-term FP32 dot product of
    trilinear derivatives with the decoder sensitivities, then a square root), so
    |Delta (1 - |g|)^2| <= 2 |1 - |g|| 1e-5 |g| + (1e-5 |g|)^2 per sample; the mean of that,
    plus 1e-6 relative for the FP32 per-lane partial sums."""
    n = gnorm[gnorm >= 0]
    if len(n) == 0:
        return 0.0
    e = 1e-5 * n
    return float(np.mean(2 * np.abs(1 - n) * e + e * e)) + 1e-6 * ref_loss


@pytest.fixture(scope="module")
def cube():
    p = Problem(CUBE)
    theta = sdf_parity_params(CUBE, sg.cube_scene(), seed=21)
    return p, theta


def _parity_rays(p, theta, bt, max_drop, label):
    """grad_x phi jumps where a hidden unit switches, and with it L_eik: rays holding a
    free-space sample within binary32 rounding of a kink are left out (printed, bounded)."""
    assert len(bt["D"]) < 64 or switching_fraction(p, theta, bt) >= 0.25
    sub, dropped = drop_kink_rays(p, theta, bt)
    print(f"eikonal batch {label}: {dropped} of {len(bt['D'])} rays left out")
    assert dropped <= max_drop * max(len(bt["D"]), 1)
    return sub


@pytest.mark.parametrize("R", [CUBE.rays, 333, 7, 1])
def test_eikonal_parity_cube(cube, R):
    p, theta = cube
    bt, _ = p.oracle_sample(SEED, 3, R=R, P=0)
    bt = _parity_rays(p, theta, bt, 0.04 if R > 100 else 1.0, f"cube R={R}")
    batch = upload_oracle_batch(bt, None, 0)
    ref_l, ref_g, n_fs, gnorm = oc.eikonal(p.cfg, theta, bt)
    assert n_fs == int(bt["counts"][2])
    got_l, got_g = _gpu(p, theta, batch)
    assert abs(got_l - ref_l) <= _loss_tol(ref_l, gnorm), (got_l, ref_l, n_fs)
    assert_grad_close(p, got_g, ref_g, skip=NO_COLOUR)
    n_grid = p.n_grid
    assert not np.any(got_g[n_grid + 512:n_grid + 544])  # b1: the mask carries no gradient
    assert not np.any(got_g[n_grid + 576:])              # W2 rows 1.., b2, colour decoder, kappa: unreachable
    if R == CUBE.rays:
        assert n_fs > 1000


def test_eikonal_loss_only_seed_and_repeated_calls(cube):
    """Loss-only calls give the same loss (the last-CTA reduction resets its counter); the
    gradient is linear in the upstream seed."""
    p, theta = cube
    bt, _ = p.oracle_sample(SEED, 4, R=CUBE.rays, P=0)
    batch = upload_oracle_batch(bt, None, 0)
    l1, g1 = _gpu(p, theta, batch)
    for _ in range(3):
        l2, _ = _gpu(p, theta, batch, want_grad=False)
        assert abs(l2 - l1) <= 1e-6 * l1
    _, g3 = _gpu(p, theta, batch, dloss=-2.5, want_loss=False)
    scale = np.abs(g1).max()
    assert np.abs(g3 + 2.5 * g1).max() <= 1e-5 * 2.5 * scale


def test_eikonal_without_free_space_samples(cube):
    p, theta = cube
    bt, _ = p.oracle_sample(SEED, 5, R=64, P=0)
    bt["cls"][:] = oc.CLS_TR
    bt["counts"] = np.array([bt["counts"][0], bt["cls"].size, 0, 0], np.int64)
    batch = upload_oracle_batch(bt, None, 0)
    got_l, got_g = _gpu(p, theta, batch)
    assert got_l == 0.0 and not np.any(got_g)


def test_eikonal_empty_batch(cube):
    p, theta = cube
    bt, _ = p.oracle_sample(SEED, 6, R=0, P=0)
    batch = upload_oracle_batch(bt, None, 0)
    got_l, got_g = _gpu(p, theta, batch)
    assert got_l == 0.0 and not np.any(got_g)


def test_eikonal_room_scale_parity():
    """The room workload at its full batch (8192 rays x 96 samples) and full grid (75.7 M
    parameters) on the first 40 frames of its trajectory."""
    w = sg.WORKLOADS["room-8192x96"]
    p = Problem(w, n_frames=40)
    bt, _ = p.oracle_sample(SEED, 11, P=0)
    theta = sdf_parity_params(w, sg.room_scene(), seed=31)
    bt = _parity_rays(p, theta, bt, 0.1, "room")
    batch = upload_oracle_batch(bt, None, 0)
    ref_l, ref_g, n_fs, gnorm = oc.eikonal(p.cfg, theta, bt)
    assert n_fs > 100000
    got_l, got_g = _gpu(p, theta, batch)
    assert abs(got_l - ref_l) <= _loss_tol(ref_l, gnorm), (got_l, ref_l)
    assert_grad_close(p, got_g, ref_g, skip=NO_COLOUR)


# ---- deferred grid term: gs_eikonal writes per-sample records, the render call scatters them ----
def _with_records(b):
    b.eik = torch.full((5, b.R, b.N, 4), float("nan"), device="cuda")  # every record the render reads is written
    return b


def test_deferred_grid_term_matches_oracle(cube):
    """With batch->eik, the Eikonal call writes each free-space sample's (p_l / v_l, a) and the
    fused forward/backward adds p_l (1/v_l)(a . dw_c/df) to the corner vectors it reduces: the
    two calls' gradient is the oracle's render gradient plus its Eikonal gradient, and the
    losses are the oracle's."""
    p, theta = cube
    bt, sm = p.oracle_sample(SEED, 8)
    bt = _parity_rays(p, theta, bt, 0.04, "cube, deferred")
    bt_s, ref, _ = prepare_parity_batch(p, theta, bt, sm, max_drop=0.05, label="cube, deferred")
    ref_l, ref_g, n_fs, gnorm = oc.eikonal(p.cfg, theta, bt_s)
    assert n_fs > 1000
    batch = _with_records(upload_oracle_batch(bt_s, sm, sm["n_valid"][0]))
    th = torch.from_numpy(theta).cuda()
    grad = torch.zeros_like(th)
    eik = torch.full((1,), float("nan"), device="cuda")
    loss = torch.empty(6, device="cuda")
    p.ctx.eikonal(th, batch, loss=eik, grad=grad)
    p.ctx.forward_backward(th, batch, None, loss, grad)
    torch.cuda.synchronize()
    p.ctx.sync_status()
    assert abs(eik.item() - ref_l) <= _loss_tol(ref_l, gnorm)
    got = loss.cpu().numpy().astype(np.float64)
    for k in range(6):
        assert abs(got[k] - ref["loss"][k]) <= LOSS_RTOL * abs(ref["loss"][k]), (k, got, ref["loss"])
    assert_grad_close(p, grad.cpu().numpy(), ref["grad"] + ref_g)
    # the records hold every free-space sample (NaN fill elsewhere is never read)
    fs = torch.from_numpy(bt_s["cls"] == oc.CLS_FS).cuda()
    assert torch.isfinite(batch.eik[:, fs]).all()


def test_deferred_equals_direct_and_loss_only_records_are_zero(cube):
    """The deferred form's gradient equals the direct form's (Eikonal call scattering its own
    grid part) on a sampled batch; a loss-only Eikonal call with records writes zero adjoints,
    so the render call after it gives the render gradient alone."""
    p, theta = cube
    batch = p.gpu_sample(SEED, 9)
    th = torch.from_numpy(theta).cuda()
    loss = torch.empty(6, device="cuda")
    g_direct = torch.zeros_like(th)
    p.ctx.forward_backward(th, batch, None, loss, g_direct)
    p.ctx.eikonal(th, batch, grad=g_direct)
    g_render = torch.zeros_like(th)
    p.ctx.forward_backward(th, batch, None, loss, g_render)
    _with_records(batch)
    g_def = torch.zeros_like(th)
    p.ctx.eikonal(th, batch, grad=g_def)
    p.ctx.forward_backward(th, batch, None, loss, g_def)
    eik = torch.empty(1, device="cuda")
    g_lo = torch.zeros_like(th)
    p.ctx.eikonal(th, batch, loss=eik)  # loss only: zero adjoints in the records
    p.ctx.forward_backward(th, batch, None, loss, g_lo)
    torch.cuda.synchronize()
    p.ctx.sync_status()
    assert_grad_close(p, g_def.cpu().numpy(), g_direct.cpu().numpy())
    assert_grad_close(p, g_lo.cpu().numpy(), g_render.cpu().numpy())
    fs = batch.cls == oc.CLS_FS
    assert fs.any() and torch.count_nonzero(batch.eik[4][fs]).item() == 0


def test_deferred_room_scale():
    """The room workload's batch (the benchmark's form): deferred and direct agree."""
    w = sg.WORKLOADS["room-8192x96"]
    p = Problem(w, n_frames=40)
    theta = sdf_parity_params(w, sg.room_scene(), seed=31)
    batch = p.gpu_sample(SEED, 12)
    th = torch.from_numpy(theta).cuda()
    loss = torch.empty(6, device="cuda")
    g_direct = torch.zeros_like(th)
    p.ctx.forward_backward(th, batch, None, loss, g_direct)
    p.ctx.eikonal(th, batch, grad=g_direct)
    _with_records(batch)
    g_def = torch.zeros_like(th)
    p.ctx.eikonal(th, batch, grad=g_def)
    p.ctx.forward_backward(th, batch, None, loss, g_def)
    torch.cuda.synchronize()
    p.ctx.sync_status()
    assert_grad_close(p, g_def.cpu().numpy(), g_direct.cpu().numpy())


def test_deferred_in_the_bf16_form():
    """The BF16 form's render kernel adds the records as the FP32 form's does: its gradient
    with records equals its gradient without them plus the direct Eikonal gradient."""
    w = CUBE.with_(name="cube-bf16", precision="bf16")
    p = Problem(w)
    theta = sdf_parity_params(CUBE, sg.cube_scene(), seed=21)
    th = torch.from_numpy(theta).cuda()
    mirror = th[:p.n_grid].to(torch.bfloat16).view(torch.int16).contiguous()
    batch = p.gpu_sample(SEED, 10)
    loss = torch.empty(6, device="cuda")
    g_direct = torch.zeros_like(th)
    p.ctx.forward_backward(th, batch, None, loss, g_direct, theta_bf16=mirror)
    p.ctx.eikonal(th, batch, grad=g_direct)
    _with_records(batch)
    g_def = torch.zeros_like(th)
    p.ctx.eikonal(th, batch, grad=g_def)
    p.ctx.forward_backward(th, batch, None, loss, g_def, theta_bf16=mirror)
    torch.cuda.synchronize()
    p.ctx.sync_status()
    assert_grad_close(p, g_def.cpu().numpy(), g_direct.cpu().numpy())
