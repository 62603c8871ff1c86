"""SDF query and its reverse mode (the double backward of grad_x phi) versus the FP64 oracle:
gs_query_sdf_backward through the C ABI and the SdfGrad autograd Function."""
import numpy as np
import pytest
import torch

import oracle as oc
import paper_2206_14735_gb300 as gs
import scenegen as sg
from gpu_common import Problem, assert_grad_close, far_from_kinks
from helpers import CUBE, sdf_parity_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    p = Problem(CUBE)
    theta = sdf_parity_params(CUBE, sg.cube_scene(), seed=21)
    _, sm = p.oracle_sample(3, 5, R=16, P=3000)
    x = sm["xs"][sm["valid"] > 0]  # points near the observed surface, as the smoothness term draws them
    rng = np.random.default_rng(7)
    x = np.concatenate([x, rng.uniform(-1.5, 1.5, (1000, 3)).astype(np.float32)])  # and anywhere, outside too
    # the hidden units switch between points; grad_x phi (and its reverse mode) jumps at a
    # kink, so points within binary32 rounding of one are left out
    ok = far_from_kinks(p, theta, x)
    print(f"sdfgrad points: {int((~ok).sum())} of {len(x)} left out")
    assert ok.mean() > 0.99
    return dict(p=p, theta=theta, x=x[ok], rng=rng)


def _run(p, theta, x, dsdf, dgrad):
    th = torch.from_numpy(theta).cuda()
    grad = torch.zeros_like(th)
    xd = torch.from_numpy(x).cuda()
    ds = None if dsdf is None else torch.from_numpy(dsdf.astype(np.float32)).cuda()
    dg = None if dgrad is None else torch.from_numpy(dgrad.astype(np.float32)).cuda()
    p.ctx.query_sdf_backward(th, xd, ds, dg, grad)
    torch.cuda.synchronize()
    return grad.cpu().numpy()


@pytest.mark.parametrize("seeds", ["both", "sdf", "grad"])
def test_query_sdf_backward_parity(case, seeds):
    x, rng = case["x"], case["rng"]
    ds = rng.normal(size=len(x)).astype(np.float32) if seeds in ("both", "sdf") else None
    dg = rng.normal(size=(len(x), 3)).astype(np.float32) if seeds in ("both", "grad") else None
    got = _run(case["p"], case["theta"], x, ds, dg)
    ref = oc.query_sdf_backward(case["p"].cfg, case["theta"], x, ds, dg)
    assert_grad_close(case["p"], got, ref, skip=("W3", "b3", "W4", "b4", "kappa"))
    _, n_grid, _ = CUBE.layout()
    assert not np.any(got[n_grid + 512 + 32 + 512 + 16:])  # no colour-decoder or kappa gradient


def test_query_sdf_backward_empty_and_ragged(case):
    for P in (0, 1, 63, 65):
        x = case["x"][:P]
        ds = np.ones(P, np.float32)
        dg = np.ones((P, 3), np.float32)
        got = _run(case["p"], case["theta"], x, ds, dg)
        if P == 0:
            assert not np.any(got)
            continue
        ref = oc.query_sdf_backward(case["p"].cfg, case["theta"], x, ds, dg)
        assert_grad_close(case["p"], got, ref, skip=("W3", "b3", "W4", "b4", "kappa"))


def test_sdfgrad_autograd_linear_seeds(case):
    """Loss linear in (phi, grad phi): the upstream seeds are known exactly."""
    x, rng = case["x"], case["rng"]
    A = rng.normal(size=len(x)).astype(np.float32)
    B = rng.normal(size=(len(x), 3)).astype(np.float32)
    th = torch.from_numpy(case["theta"]).cuda().requires_grad_(True)
    sdf, g = gs.SdfGrad.apply(th, case["p"].ctx, torch.from_numpy(x).cuda())
    ((sdf * torch.from_numpy(A).cuda()).sum() + (g * torch.from_numpy(B).cuda()).sum()).backward()
    ref = oc.query_sdf_backward(case["p"].cfg, case["theta"], x, A, B)
    assert_grad_close(case["p"], th.grad.cpu().numpy(), ref, skip=("W3", "b3", "W4", "b4", "kappa"))


def test_sdfgrad_autograd_eikonal(case):
    """An eikonal term mean((|grad phi| - 1)^2): the autograd seeds equal the closed form
    2 (|g| - 1) g / (|g| P) and the gradient matches the oracle's for those seeds."""
    x = case["x"]
    th = torch.from_numpy(case["theta"]).cuda().requires_grad_(True)
    _, g = gs.SdfGrad.apply(th, case["p"].ctx, torch.from_numpy(x).cuda())
    ((g.norm(dim=1) - 1.0) ** 2).mean().backward()
    _, g_ref = oc.query_sdf(case["p"].cfg, case["theta"], x)
    n = np.linalg.norm(g_ref, axis=1, keepdims=True)
    # grad phi vanishes outside the grid box (clamped cells); the norm's subgradient there is 0
    seeds = np.where(n > 0, 2.0 * (n - 1.0) * g_ref / (np.maximum(n, 1e-30) * len(x)), 0.0)
    ref = oc.query_sdf_backward(case["p"].cfg, case["theta"], x, None, seeds)
    assert_grad_close(case["p"], th.grad.cpu().numpy(), ref, tol=1e-3, elem_rtol=1e-2,
                      skip=("W3", "b3", "W4", "b4", "kappa"))
