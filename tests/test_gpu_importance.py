"""Hierarchical importance sampler (gs_sample_importance, Sec. 3.2) and the render kernel at
its 132 samples per ray (5 chunks of 32) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle as oc
import paper_2206_14735_gb300 as gs
import scenegen as sg
from gpu_common import (LOSS_RTOL, Problem, assert_grad_close, prepare_parity_batch, upload_oracle_batch)
from helpers import CUBE, sdf_parity_params

pytestmark = pytest.mark.gpu
IMP = dict(imp_coarse=96, imp_steps=3, imp_per_step=12)
W = CUBE.with_(name="cube-imp", **IMP)
SEED = 77


@pytest.fixture(scope="module")
def prob():
    p = Problem(W)
    theta = sdf_parity_params(W, sg.cube_scene(), seed=21)
    return p, theta


def _gpu_sample(p, theta, R, step, P=0):
    b = gs.Batch.allocate(R, W.n_samples, P)
    th = torch.from_numpy(theta).cuda()
    p.ctx.sample_importance(p.dfr, th, SEED, step, b)
    torch.cuda.synchronize()
    p.ctx.sync_status()
    return {k: getattr(b, a).cpu().numpy() for k, a in
            (("pix", "pix"), ("o", "origin"), ("r", "dir"), ("rgb", "rgb"), ("D", "depth"), ("t", "t"), ("cls", "cls"),
             ("counts", "counts"))}


def _compare_samples(got, ref, coarse, n_coarse):
    for k in ("pix", "o", "r", "rgb", "D"):
        assert np.array_equal(got[k], ref[k]), k
    tg, tr = got["t"].astype(np.float64), ref["t"].astype(np.float64)
    assert np.all(np.diff(tg, axis=1) >= 0)
    # the coarse strata do not depend on phi: the same binary32 values on both sides
    for i in range(len(tg)):
        assert np.isin(coarse[i], got["t"][i]).all(), i
    _check_depth_deviation(tg - tr, W.far - W.near, n_coarse)
    flip = got["cls"] != ref["cls"]
    assert flip.mean() <= 1e-3


def _check_depth_deviation(diff, span, n_coarse):
    """The importance depths follow the weights, computed here from FP32 phi with FP32 running
    sums and in the oracle in FP64.  Where the weight is large a draw moves by a few ulps.
    Where it falls among intervals that hold only the 1e-5 floor of mass, a difference in the
    running sum of the order of that floor moves it across one or more of those intervals.
    So: 90 % of the depths within 1e-5 of the range, at most 0.2 % of them moved by more than
    1 mm, and none by more than four coarse intervals."""
    d = np.abs(diff)
    stats = dict(q90=float(np.quantile(d, 0.9)), moved=float((d > 1e-3).mean()), max=float(d.max()),
                 interval=span / n_coarse)
    assert stats["q90"] <= 1e-5 * span, stats
    assert stats["moved"] <= 2e-3, stats
    assert stats["max"] <= 4 * span / n_coarse, stats


@pytest.mark.parametrize("R", [W.rays, 257, 1])
def test_importance_sampler_parity(prob, R):
    p, theta = prob
    got = _gpu_sample(p, theta, R, step=3)
    ref = oc.sample_importance(p.cfg, p.ofr, theta, SEED, 3, R, 96, 3, 12)
    coarse = oc.sample_importance(p.cfg, p.ofr, theta, SEED, 3, R, 96, 0, 12)["t"]
    _compare_samples(got, ref, coarse, 96)
    assert abs(int(got["counts"][0]) - int(ref["counts"][0])) == 0
    assert abs(int(got["counts"][1]) - int(ref["counts"][1])) <= 2 + R // 100
    assert abs(int(got["counts"][2]) - int(ref["counts"][2])) <= 2 + R // 100


def test_importance_samples_concentrate_where_the_weight_is(prob):
    """The importance depths cluster around the rendered depth: with the scene's SDF baked
    into the grid, the median distance of the added samples to the observed surface is far
    below that of the coarse samples."""
    p, theta = prob
    got = _gpu_sample(p, theta, W.rays, step=4)
    ref = oc.sample_importance(p.cfg, p.ofr, theta, SEED, 4, W.rays, 96, 0, 12)  # the coarse depths alone
    D = got["D"]
    hit = D > 0
    added, coarse = [], []
    for i in np.nonzero(hit)[0]:
        rest = list(got["t"][i])
        for v in ref["t"][i]:
            rest.remove(v)
        added += list(np.abs(np.array(rest) - D[i]))
        coarse += list(np.abs(ref["t"][i] - D[i]))
    assert np.median(added) < 0.1 * np.median(coarse), (np.median(added), np.median(coarse))


@pytest.mark.parametrize("store", [False, True])
def test_render_parity_at_132_samples(prob, store):
    """The fused render kernel on importance batches (5 chunks of 32 samples, 2 tile groups
    per CTA): losses and gradients against the oracle's step on the oracle's own batch."""
    p, theta = prob
    ctx = gs.Context(W, store_activations=store) if store else p.ctx
    bt = oc.sample_importance(p.cfg, p.ofr, theta, SEED, 5, 600, 96, 3, 12)
    _, sm = p.oracle_sample(SEED, 5, R=4, P=W.n_smooth)
    bt_s, ref, dropped = prepare_parity_batch(p, theta, bt, sm)
    batch = upload_oracle_batch(bt_s, sm, sm["n_valid"][0])
    th = torch.from_numpy(theta).cuda()
    loss = torch.empty(6, device="cuda")
    grad = torch.zeros_like(th)
    ctx.forward_backward(th, batch, None, loss, grad)
    torch.cuda.synchronize()
    ctx.sync_status()
    got = loss.cpu().numpy().astype(np.float64)
    for k in range(6):
        assert abs(got[k] - ref["loss"][k]) <= LOSS_RTOL * abs(ref["loss"][k]), (k, got, ref["loss"])
    assert_grad_close(p, grad.cpu().numpy(), ref["grad"])


def test_importance_sampler_room_scale():
    """The room workload's importance configuration at its full batch (8192 rays x 132)."""
    w = sg.WORKLOADS["room-imp-8192x132"]
    p = Problem(w, n_frames=40)
    theta = sdf_parity_params(w, sg.room_scene(), seed=31)
    b = gs.Batch.allocate(w.rays, w.n_samples, 0)
    p.ctx.sample_importance(p.dfr, torch.from_numpy(theta).cuda(), SEED, 11, b)
    torch.cuda.synchronize()
    got = {k: getattr(b, a).cpu().numpy() for k, a in (("pix", "pix"), ("o", "origin"), ("r", "dir"), ("rgb", "rgb"),
                                                        ("D", "depth"), ("t", "t"), ("cls", "cls"))}
    ref = oc.sample_importance(p.cfg, p.ofr, theta, SEED, 11, w.rays, 96, 3, 12)
    for k in ("pix", "o", "r", "rgb", "D"):
        assert np.array_equal(got[k], ref[k]), k
    _check_depth_deviation(got["t"].astype(np.float64) - ref["t"], w.far - w.near, 96)
    assert (got["cls"] != ref["cls"]).mean() <= 1e-3


def test_importance_sampler_ragged_configuration():
    """N_c not a multiple of 32 and M not 12 (40 coarse samples in two rounds, the second with
    8 busy rows per ray; 2 steps of 20): the tensor-core rounds with idle rows against the
    oracle."""
    w2 = CUBE.with_(name="cube-imp-ragged", imp_coarse=40, imp_steps=2, imp_per_step=20)
    p = Problem(w2)
    theta = sdf_parity_params(w2, sg.cube_scene(), seed=21)
    R = 333
    b = gs.Batch.allocate(R, w2.n_samples, 0)
    assert w2.n_samples == 80
    p.ctx.sample_importance(p.dfr, torch.from_numpy(theta).cuda(), SEED, 5, b)
    torch.cuda.synchronize()
    p.ctx.sync_status()
    got = {k: getattr(b, a).cpu().numpy() for k, a in
           (("pix", "pix"), ("o", "origin"), ("r", "dir"), ("rgb", "rgb"), ("D", "depth"), ("t", "t"), ("cls", "cls"))}
    ref = oc.sample_importance(p.cfg, p.ofr, theta, SEED, 5, R, 40, 2, 20)
    coarse = oc.sample_importance(p.cfg, p.ofr, theta, SEED, 5, R, 40, 0, 20)["t"]
    for k in ("pix", "o", "r", "rgb", "D"):
        assert np.array_equal(got[k], ref[k]), k
    assert np.all(np.diff(got["t"].astype(np.float64), axis=1) >= 0)
    for i in range(R):
        assert np.isin(coarse[i], got["t"][i]).all(), i
    _check_depth_deviation(got["t"].astype(np.float64) - ref["t"].astype(np.float64), w2.far - w2.near, 40)
    assert (got["cls"] != ref["cls"]).mean() <= 1e-3
