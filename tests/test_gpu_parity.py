"""CUDA path (through the C ABI) versus the FP64 oracle on identical seeded inputs.

Discrete outputs (pixel ids, sample depths, classes, counts, smoothness points, voxel
cells) must match bit for bit.  Floating-point outputs must agree within the stated
tolerances: loss terms to 1e-5 relative; each gradient tensor to 1e-4 of its largest
entry (and 1e-3 relative element-wise where an entry exceeds 1% of that maximum).
"""
import math

import numpy as np
import pytest
import torch

import oracle as oc
import paper_2206_14735_gb300 as gs
import scenegen as sg
from gpu_common import (GRAD_TOL, LOSS_RTOL, Problem, assert_grad_close, corner_case, far_from_kinks,
                        prepare_parity_batch, sample_positions, upload_oracle_batch)
from helpers import CUBE, sdf_parity_params

pytestmark = pytest.mark.gpu

SEED, STEP = 3, 5


@pytest.fixture(scope="module")
def cube():
    return Problem(CUBE)


def _bits(a):
    a = np.ascontiguousarray(a)
    return a.view(np.uint32) if a.dtype == np.float32 else a


def _check_sampler(p: Problem, R, P, seed=SEED, step=STEP):
    b = p.gpu_sample(seed, step, R, P)
    bt, sm = p.oracle_sample(seed, step, R, P)
    assert np.array_equal(b.pix.cpu().numpy(), bt["pix"])
    for gk, ok in (("origin", "o"), ("dir", "r"), ("rgb", "rgb"), ("depth", "D"), ("t", "t")):
        assert np.array_equal(_bits(getattr(b, gk).cpu().numpy()), _bits(bt[ok])), gk
    assert np.array_equal(b.cls.cpu().numpy(), bt["cls"])
    c = b.counts.cpu().numpy()
    assert list(c[:3]) == list(bt["counts"][:3])
    if P > 0:
        assert np.array_equal(b.valid[:P].cpu().numpy(), sm["valid"])
        assert np.array_equal(_bits(b.xs[:P].cpu().numpy()), _bits(sm["xs"]))
        assert np.array_equal(_bits(b.eps[:P].cpu().numpy()), _bits(sm["eps"]))
        assert c[3] == sm["n_valid"][0]
    return b, bt, sm


def test_sampler_bit_exact(cube):
    _check_sampler(cube, CUBE.rays, CUBE.n_smooth)


def test_sampler_bit_exact_ragged_sizes(cube):
    # batch sizes that are not multiples of the block size, a single ray, an empty batch
    for R, P in ((1000, 77), (1, 1), (0, 0), (33, 0)):
        _check_sampler(cube, R, P, seed=9, step=R)


def test_voxel_index_bit_exact(cube):
    rng = np.random.default_rng(0)
    x = rng.uniform(-1.6, 1.6, (20000, 3)).astype(np.float32)
    # points exactly on vertices and cell faces, and on the box faces
    v = np.float32(CUBE.voxels[3])
    idx = rng.integers(0, 33, (2000, 3)).astype(np.float32)
    x = np.concatenate([x, (np.float32(-1.28) + idx * v).astype(np.float32),
                        np.float32([[1.28, 1.28, 1.28], [-1.28, -1.28, -1.28], [1.2799999, 0, 0]])])
    bt, _ = cube.oracle_sample(SEED, STEP)
    x = np.concatenate([x, sample_positions(bt).reshape(-1, 3)])
    want = oc.voxel_index(cube.cfg, x)
    xd = torch.from_numpy(x).cuda()
    out = torch.empty(len(x), 4, dtype=torch.int64, device="cuda")
    cube.ctx.voxel_index(xd, out)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), want)


@pytest.fixture(scope="module")
def cube_case(cube):
    theta = sdf_parity_params(CUBE, sg.cube_scene(), seed=21)
    bt, sm = cube.oracle_sample(SEED, STEP)
    # hidden units switch within the batch; rays with a unit, an alpha, an SDF sign or a
    # free-space maximum within binary32 rounding of its tie are left out
    bt_s, ref, n_dropped = prepare_parity_batch(cube, theta, bt, sm, max_drop=0.05, min_switch=0.25, label="cube")
    assert ref["margins"][5] > 1e-5, ref["margins"]  # per-ray depth signs clear of their kink
    batch = upload_oracle_batch(bt_s, sm, sm["n_valid"][0])
    return dict(theta=theta, bt=bt_s, sm=sm, ref=ref, batch=batch)


def test_forward_loss_parity(cube, cube_case):
    th = torch.from_numpy(cube_case["theta"]).cuda()
    b = cube_case["batch"]
    loss = torch.empty(6, device="cuda")
    rgb_hat = torch.empty(b.R, 3, device="cuda")
    d_hat = torch.empty(b.R, device="cuda")
    wsum = torch.empty(b.R, device="cuda")
    cube.ctx.forward(th, b, loss, rgb_hat, d_hat, wsum)
    torch.cuda.synchronize()
    ref = cube_case["ref"]
    got = loss.cpu().numpy().astype(np.float64)
    for k in range(6):
        assert abs(got[k] - ref["loss"][k]) <= LOSS_RTOL * abs(ref["loss"][k]), (k, got, ref["loss"])
    np.testing.assert_allclose(rgb_hat.cpu().numpy(), ref["rgb_hat"], atol=2e-6)
    np.testing.assert_allclose(d_hat.cpu().numpy(), ref["d_hat"], atol=2e-5)
    np.testing.assert_allclose(wsum.cpu().numpy(), ref["wsum"], atol=2e-6)
    assert wsum.max().item() <= 1.0 + 1e-6


def test_backward_gradient_parity(cube, cube_case):
    th = torch.from_numpy(cube_case["theta"]).cuda()
    grad = torch.zeros_like(th)
    cube.ctx.backward(th, cube_case["batch"], None, grad)
    torch.cuda.synchronize()
    rep = assert_grad_close(cube, grad.cpu().numpy(), cube_case["ref"]["grad"])
    assert max(e for e, _ in rep.values()) < GRAD_TOL


def test_forward_backward_fused_equals_split(cube, cube_case):
    th = torch.from_numpy(cube_case["theta"]).cuda()
    b = cube_case["batch"]
    loss = torch.empty(6, device="cuda")
    grad = torch.zeros_like(th)
    cube.ctx.forward_backward(th, b, None, loss, grad)
    torch.cuda.synchronize()
    ref = cube_case["ref"]
    got = loss.cpu().numpy().astype(np.float64)
    for k in range(6):
        assert abs(got[k] - ref["loss"][k]) <= LOSS_RTOL * abs(ref["loss"][k])
    assert_grad_close(cube, grad.cpu().numpy(), ref["grad"])


def test_backward_per_term_seeds(cube, cube_case):
    """Upstream derivative per loss term (the autograd contract)."""
    dl = np.array([0.3, -1.1, 0.7, 2.0, 5.0, 0.25])
    ref = oc.step(cube.cfg, cube_case["theta"], cube_case["bt"], cube_case["sm"], dloss=dl)
    th = torch.from_numpy(cube_case["theta"]).cuda()
    grad = torch.zeros_like(th)
    cube.ctx.backward(th, cube_case["batch"], torch.tensor(dl, dtype=torch.float32, device="cuda"), grad)
    torch.cuda.synchronize()
    assert_grad_close(cube, grad.cpu().numpy(), ref["grad"])


def test_autograd_function_matches_oracle(cube, cube_case):
    th = torch.from_numpy(cube_case["theta"]).cuda().requires_grad_(True)
    losses = gs.GoSurfStep.apply(th, cube.ctx, cube_case["batch"])
    (losses[5] + 0.5 * losses[4]).backward()
    dl = np.array([0, 0, 0, 0, 0.5, 1.0])
    ref = oc.step(cube.cfg, cube_case["theta"], cube_case["bt"], cube_case["sm"], dloss=dl)
    assert_grad_close(cube, th.grad.cpu().numpy(), ref["grad"])


def test_smoothness_term_alone(cube, cube_case):
    """Only the second-order path: dloss selects L_smooth."""
    dl = np.array([0, 0, 0, 0, 1.0, 0])
    ref = oc.step(cube.cfg, cube_case["theta"], cube_case["bt"], cube_case["sm"], dloss=dl)
    th = torch.from_numpy(cube_case["theta"]).cuda()
    grad = torch.zeros_like(th)
    cube.ctx.backward(th, cube_case["batch"], torch.tensor(dl, dtype=torch.float32, device="cuda"), grad)
    torch.cuda.synchronize()
    g = grad.cpu().numpy()
    assert np.abs(g[:cube.n_grid]).max() > 0
    # decoder entries the smoothness term cannot reach stay exactly zero
    parts = cube.split_grad(g)
    for k in ("b1", "b2", "W3", "b3", "W4", "b4", "kappa"):
        assert np.abs(parts[k]).max() == 0, k
    assert_grad_close(cube, g, ref["grad"], skip=("b1", "b2", "W3", "b3", "W4", "b4", "kappa"))


def test_query_sdf_parity(cube, cube_case):
    rng = np.random.default_rng(1)
    x = rng.uniform(-1.5, 1.5, (5000, 3)).astype(np.float32)
    sdf_ref, g_ref = oc.query_sdf(cube.cfg, cube_case["theta"], x)
    th = torch.from_numpy(cube_case["theta"]).cuda()
    sdf = torch.empty(len(x), device="cuda")
    grad = torch.empty(len(x), 3, device="cuda")
    cube.ctx.query_sdf(th, torch.from_numpy(x).cuda(), sdf, grad)
    torch.cuda.synchronize()
    np.testing.assert_allclose(sdf.cpu().numpy(), sdf_ref, atol=2e-6)
    # grad_x phi jumps where a hidden unit switches: points within binary32 rounding of a
    # kink are not compared
    ok = far_from_kinks(cube, cube_case["theta"], x)
    assert ok.mean() > 0.99
    np.testing.assert_allclose(grad.cpu().numpy()[ok], g_ref[ok], atol=2e-4 * np.abs(g_ref).max())


def test_adam_parity(cube):
    rng = np.random.default_rng(2)
    n, n_grid = cube.n_tot, cube.n_grid
    p0 = rng.normal(size=n).astype(np.float32)
    m0 = (rng.normal(size=n) * 1e-2).astype(np.float32)
    v0 = (rng.uniform(size=n) * 1e-3).astype(np.float32)
    g0 = rng.normal(size=n).astype(np.float32)
    P, G, M, V = (torch.from_numpy(a.copy()).cuda() for a in (p0, g0, m0, v0))
    bf = torch.empty(n_grid, dtype=torch.int16, device="cuda")
    cube.ctx.adam_step(P, G, M, V, 7, 1e-2, 1e-3, theta_bf16=bf)
    torch.cuda.synchronize()
    p, g, m, v = (a.astype(np.float64) for a in (p0, g0, m0, v0))
    f32 = lambda x: float(np.float32(x))  # the kernel receives binary32 hyper-parameters
    oc.adam(p, g, m, v, n_grid, 7, f32(1e-2), f32(1e-3), f32(0.9), f32(0.999), f32(1e-8))
    # binary32 rounding bounds: a few ulps of the operands of each update
    u32 = 2.0 ** -24
    np.testing.assert_array_less(np.abs(M.cpu().numpy() - m), 4 * u32 * (0.9 * np.abs(m0) + 0.1 * np.abs(g0)) + 1e-30)
    np.testing.assert_array_less(np.abs(V.cpu().numpy() - v), 4 * u32 * (0.999 * v0 + 0.001 * g0 * g0) + 1e-30)
    lr = np.where(np.arange(n) < n_grid, 1e-2, 1e-3)
    upd = np.abs(p - p0.astype(np.float64))
    np.testing.assert_array_less(np.abs(P.cpu().numpy() - p), 4 * u32 * np.abs(p0) + 1e-5 * upd + 1e-7 * lr)
    assert G.abs().max().item() == 0.0
    # the bfloat16 copy is the round-to-nearest-even image of the updated grid
    want = torch.from_numpy(P.cpu().numpy()[:n_grid]).to(torch.bfloat16).view(torch.int16)
    assert torch.equal(bf.cpu(), want)


def test_edge_cases_empty_and_ragged(cube):
    theta = torch.from_numpy(sdf_parity_params(CUBE, sg.cube_scene(), seed=21)).cuda()
    loss = torch.empty(6, device="cuda")
    # empty batch: all losses 0, gradient untouched
    b0 = cube.gpu_sample(1, 1, 0, 0)
    grad = torch.zeros_like(theta)
    cube.ctx.forward_backward(theta, b0, None, loss, grad)
    torch.cuda.synchronize()
    assert loss.abs().max().item() == 0.0 and grad.abs().max().item() == 0.0
    # rays without smoothness points and vice versa
    b1 = cube.gpu_sample(1, 2, 37, 0)
    cube.ctx.forward(theta, b1, loss)
    torch.cuda.synchronize()
    assert loss[4].item() == 0.0 and loss[0].item() > 0
    b2 = cube.gpu_sample(1, 3, 0, 50)
    cube.ctx.forward(theta, b2, loss)
    torch.cuda.synchronize()
    assert loss[0].item() == 0.0 and loss[4].item() > 0


def test_ragged_samples_per_ray():
    """N = 33 (one full chunk of 32 plus one) and rays that leave the grid box."""
    w = CUBE.with_(name="cube-ragged", n_strat=21, n_guided=12, far=6.0, rays=333, n_smooth=100)
    p = Problem(w)
    theta = sdf_parity_params(w, sg.cube_scene(), seed=22)
    b_gpu, bt, sm = _check_sampler(p, w.rays, w.n_smooth, seed=4, step=1)
    bt_s, ref, _ = prepare_parity_batch(p, theta, bt, sm, max_drop=0.06, min_switch=0.25, label="ragged N=33")
    batch = upload_oracle_batch(bt_s, sm, sm["n_valid"][0])
    th = torch.from_numpy(theta).cuda()
    loss = torch.empty(6, device="cuda")
    grad = torch.zeros_like(th)
    p.ctx.forward_backward(th, batch, None, loss, grad)
    torch.cuda.synchronize()
    got = loss.cpu().numpy().astype(np.float64)
    for k in range(6):
        assert abs(got[k] - ref["loss"][k]) <= LOSS_RTOL * abs(ref["loss"][k]), (k, got, ref["loss"])
    assert_grad_close(p, grad.cpu().numpy(), ref["grad"])


@pytest.mark.parametrize("n_frames", [40])
def test_room_scale_parity(n_frames):
    """The room workload at its full batch (8192 rays x 96 samples, 4096 smoothness points)
    and full grid (75.7 M parameters) on the first frames of its trajectory."""
    w = sg.WORKLOADS["room-8192x96"]
    p = Problem(w, n_frames=n_frames)
    _check_sampler(p, w.rays, w.n_smooth, seed=SEED, step=11)
    bt, sm = p.oracle_sample(SEED, 11)
    theta = sdf_parity_params(w, sg.room_scene(), seed=31)
    # 96 samples per ray, so more rays hold a sample within binary32 rounding of a tie
    bt_s, ref, n_dropped = prepare_parity_batch(p, theta, bt, sm, max_drop=0.15, min_switch=0.25, label="room")
    assert ref["margins"][5] > 1e-5
    batch = upload_oracle_batch(bt_s, sm, sm["n_valid"][0])
    th = torch.from_numpy(theta).cuda()
    loss = torch.empty(6, device="cuda")
    grad = torch.zeros_like(th)
    p.ctx.forward_backward(th, batch, None, loss, grad)
    torch.cuda.synchronize()
    got = loss.cpu().numpy().astype(np.float64)
    for k in range(6):
        assert abs(got[k] - ref["loss"][k]) <= LOSS_RTOL * abs(ref["loss"][k]), (k, got, ref["loss"])
    assert_grad_close(p, grad.cpu().numpy(), ref["grad"])


@pytest.mark.parametrize("corner", ["max", "min"])
def test_samples_at_the_grid_corners(corner):
    """Samples crossing a corner of the grid: the finest level's tile::gather4 rows reach the
    first or last (y, z) lines and columns; loss and every gradient tensor against the FP64
    oracle."""
    p = Problem(CUBE, max_rays=256)
    theta, bt_s, ref = corner_case(p, sdf_parity_params(CUBE, sg.cube_scene(), seed=21), "b2", corner, SEED, STEP)
    batch = upload_oracle_batch(bt_s, None, 0)
    th = torch.from_numpy(theta).cuda()
    loss = torch.empty(6, device="cuda")
    grad = torch.zeros_like(th)
    p.ctx.forward_backward(th, batch, None, loss, grad)
    torch.cuda.synchronize()
    got = loss.cpu().numpy().astype(np.float64)
    for k in range(6):
        assert abs(got[k] - ref["loss"][k]) <= LOSS_RTOL * abs(ref["loss"][k]) + 1e-12, (k, got, ref["loss"])
    assert_grad_close(p, grad.cpu().numpy(), ref["grad"])
