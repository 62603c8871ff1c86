"""gs_forward_backward_noalloc: the allocation-free variant of the fused forward/backward,
for callers that may not allocate device memory (code inside a framework that owns every
device allocation, or a loop that cannot take cudaMalloc's implicit synchronisation).

It is called through the C ABI and must give what gs_forward_backward gives, within the
parity tolerances, on two calls in a row (the static scratch array keeps the previous
call's contents, which must not leak into the next result).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2206_14735_gb300 as gs
import scenegen as sg
from gpu_common import LOSS_RTOL, Problem, assert_grad_close
from helpers import CUBE, sdf_parity_params
from paper_2206_14735_gb300 import _lib

pytestmark = pytest.mark.gpu


def _noalloc(cfg, theta, b, dl, loss, grad):
    L = _lib.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return L.gs_forward_backward_noalloc(ctypes.byref(cfg), ctypes.c_void_p(theta.data_ptr()), ctypes.byref(b),
                                         ctypes.c_void_p(0 if dl is None else dl.data_ptr()),
                                         ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(grad.data_ptr()), stream)


# rays and smoothness points; rays only (no smoothness rows to combine); smoothness points only
# (the rows start after the render CTAs' rows)
@pytest.mark.parametrize("R,P", [(None, None), (None, 0), (0, None)])
def test_noalloc_matches_forward_backward_twice(R, P):
    p = Problem(CUBE)
    batch = p.gpu_sample(7, 3, R=R, P=P)
    theta = torch.from_numpy(sdf_parity_params(CUBE, sg.cube_scene(), seed=21)).cuda()
    # existing entry point (context workspace)
    loss_ref = torch.empty(6, device="cuda")
    grad_ref = torch.zeros_like(theta)
    p.ctx.forward_backward(theta, batch, None, loss_ref, grad_ref)
    torch.cuda.synchronize()
    L = _lib.lib()
    cfg = gs.make_config(CUBE)
    b = batch.struct()
    dl = torch.tensor([0.0, 0.0, 0.0, 0.0, 0.0, 1.0], device="cuda")
    for call in range(2):
        loss = torch.full((6,), float("nan"), device="cuda")
        grad = torch.zeros_like(theta)
        st = _noalloc(cfg, theta, b, dl if call else None, loss, grad)
        assert st == 0, L.gs_last_error(None)
        torch.cuda.synchronize()
        got, ref = loss.cpu().numpy().astype(np.float64), loss_ref.cpu().numpy().astype(np.float64)
        # every entry finite: the call's status word (cleared at its start) reports no failure
        assert np.isfinite(got).all(), got
        np.testing.assert_array_less(np.abs(got - ref), LOSS_RTOL * np.abs(ref) + 1e-12)
        assert_grad_close(p, grad.cpu().numpy(), grad_ref.cpu().numpy())


def test_noalloc_rejects_bad_arguments():
    L = _lib.lib()
    cfg = gs.make_config(CUBE)
    assert L.gs_forward_backward_noalloc(None, None, None, None, None, None, None) == 1
    theta = torch.zeros(CUBE.layout()[2], device="cuda")
    th = ctypes.c_void_p(theta.data_ptr())
    assert L.gs_forward_backward_noalloc(ctypes.byref(cfg), th, None, None, None, None, None) == 1

    def code(**change):
        bad = gs.make_config(CUBE)
        for k, v in change.items():
            if k == "voxel1":
                bad.voxel[1] = v
            elif k == "dims0":
                bad.dims[0][0] = v
            elif k == "dims1_huge":
                bad.dims[1][0], bad.dims[1][1], bad.dims[1][2] = 2048, 2048, 512
            else:
                setattr(bad, k, v)
        return L.gs_forward_backward_noalloc(ctypes.byref(bad), th, None, None, None, None, None)

    # the rules gs_create applies, with its status codes
    assert code(voxel1=-1.0) == 1
    assert code(dims0=1) == 1
    assert code(dims1_huge=True) == 6  # 2^31 vertices on level 1: the run keys are 32-bit
    assert code(near_m=5.0, far_m=1.0) == 1
    assert code(trunc=0.0) == 1
    assert code(guide_half=-0.1) == 1
    assert code(n_strat=0) == 1
    assert code(n_strat=150, n_guided=20) == 6
    assert code(max_rays=-1) == 1
    # forms this entry point does not run
    assert code(precision=gs.GS_PREC_BF16) == 6
    assert code(arch=gs.GS_ARCH_PAPER) == 6


def test_noalloc_adds_deferred_eikonal_records():
    """gs_forward_backward_noalloc reads batch->eik as gs_forward_backward does: after one
    Eikonal call writes the records, both entry points give the same gradient."""
    p = Problem(CUBE)
    batch = p.gpu_sample(7, 4)
    theta = torch.from_numpy(sdf_parity_params(CUBE, sg.cube_scene(), seed=21)).cuda()
    batch.eik = torch.full((5, batch.R, batch.N, 4), float("nan"), device="cuda")
    g_eik = torch.zeros_like(theta)
    p.ctx.eikonal(theta, batch, grad=g_eik)  # decoder part into g_eik, grid part into the records
    loss_ref = torch.empty(6, device="cuda")
    grad_ref = g_eik.clone()
    p.ctx.forward_backward(theta, batch, None, loss_ref, grad_ref)
    torch.cuda.synchronize()
    p.ctx.sync_status()
    loss = torch.empty(6, device="cuda")
    grad = g_eik.clone()
    st = _noalloc(gs.make_config(CUBE), theta, batch.struct(), None, loss, grad)
    assert st == 0, _lib.lib().gs_last_error(None)
    torch.cuda.synchronize()
    assert np.isfinite(loss.cpu().numpy()).all()
    assert_grad_close(p, grad.cpu().numpy(), grad_ref.cpu().numpy())
    # without the records the grid part is missing: the records do reach the scatter
    batch.eik = None
    grad_plain = g_eik.clone()
    assert _noalloc(gs.make_config(CUBE), theta, batch.struct(), None, loss, grad_plain) == 0
    torch.cuda.synchronize()
    n = p.n_grid
    assert np.abs(grad_plain.cpu().numpy()[:n] - grad.cpu().numpy()[:n]).max() > 0
