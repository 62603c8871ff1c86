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


def test_noalloc_matches_forward_backward_twice():
    p = Problem(CUBE)
    batch = p.gpu_sample(7, 3)
    theta = torch.from_numpy(sdf_parity_params(CUBE, sg.cube_scene(), seed=21)).cuda()
    # existing entry point (context workspace)
    loss_ref = torch.empty(6, device="cuda")
    grad_ref = torch.zeros_like(theta)
    p.ctx.forward_backward(theta, batch, None, loss_ref, grad_ref)
    torch.cuda.synchronize()
    L = _lib.lib()
    cfg = gs.make_config(CUBE)
    b = batch.struct()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    dl = torch.tensor([0.0, 0.0, 0.0, 0.0, 0.0, 1.0], device="cuda")
    for call in range(2):
        loss = torch.full((6,), float("nan"), device="cuda")
        grad = torch.zeros_like(theta)
        st = L.gs_forward_backward_noalloc(ctypes.byref(cfg), ctypes.c_void_p(theta.data_ptr()), ctypes.byref(b),
                                           ctypes.c_void_p(dl.data_ptr() if call else 0),
                                           ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(grad.data_ptr()), stream)
        assert st == 0, L.gs_last_error(None)
        torch.cuda.synchronize()
        got, ref = loss.cpu().numpy().astype(np.float64), loss_ref.cpu().numpy().astype(np.float64)
        np.testing.assert_array_less(np.abs(got - ref), LOSS_RTOL * np.abs(ref) + 1e-12)
        assert_grad_close(p, grad.cpu().numpy(), grad_ref.cpu().numpy())


def test_noalloc_rejects_bad_arguments():
    L = _lib.lib()
    cfg = gs.make_config(CUBE)
    assert L.gs_forward_backward_noalloc(None, None, None, None, None, None, None) == 1
    bad = gs.make_config(CUBE)
    bad.voxel[1] = -1.0
    assert L.gs_forward_backward_noalloc(ctypes.byref(bad), None, None, None, None, None, None) == 1
    theta = torch.zeros(CUBE.layout()[2], device="cuda")
    assert L.gs_forward_backward_noalloc(ctypes.byref(cfg), ctypes.c_void_p(theta.data_ptr()), None, None, None,
                                         None, None) == 1
