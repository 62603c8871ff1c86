"""Pins of the learned proposal sampler in the oracle (a sample-count reduction that is not
part of the paper): central differences of its cross-entropy loss, closed forms of the
softmax / cross entropy, and properties of the inverse-CDF sampler that any correct
implementation has (a uniform PDF gives stratified samples; one draw per CDF stratum)."""
import math

import numpy as np
import pytest

import oracle as oc
import scenegen as sg
from helpers import CUBE, TINY

NB = oc.PROP_BINS


def _rays(w, R, seed=3):
    cfg = oc.make_config(w)
    fr = oc.OcFramesHolder(sg.make_frames(w))
    bt = oc.sample_rays(cfg, fr, seed, 0, R)
    return cfg, bt


def _random_q(seed=1, scale=0.3):
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, oc.PROP_PARAMS)


def _mixture_cdf(cfg, p):
    """pp = 0.95 p + 0.05/32 and its running sums (FP64) for the CDF checks."""
    pp = 0.95 * np.asarray(p, np.float64) + 0.05 / NB
    return pp, np.cumsum(pp, axis=-1)


def test_softmax_rows_sum_to_one():
    cfg, bt = _rays(CUBE, 64)
    th = sg.parity_params(CUBE, seed=2, grid_std=0.3).astype(np.float64)
    p = oc.prop_forward(cfg, th, _random_q(), bt["o"], bt["r"])
    assert p.shape == (64, NB)
    assert np.all(p > 0)
    np.testing.assert_allclose(p.sum(1), 1.0, rtol=0, atol=1e-12)


def test_uniform_logits_give_log32_and_zero_gradient():
    """All weights zero: every logit equals b3, p = 1/32, and the cross entropy against any
    normalised histogram is log 32 with dL/dl_b = 1/32 - hh_b summing to zero, so b3 gets
    no gradient (nor does anything else: every activation is zero)."""
    cfg, bt = _rays(CUBE, 32)
    th = sg.parity_params(CUBE, seed=2).astype(np.float64)
    q = np.zeros(oc.PROP_PARAMS)
    q[-1] = 0.7
    rng = np.random.default_rng(4)
    w = rng.uniform(0, 1, bt["t"].shape) / bt["t"].shape[1]
    ce, g, n = oc.prop_ce(cfg, th, q, bt["o"], bt["r"], bt["t"], w)
    assert n == 32
    assert abs(ce - math.log(NB)) < 1e-12
    assert np.abs(g).max() < 1e-12


def test_one_hot_target_cross_entropy_closed_form():
    """All of a ray's weight in one bin: the loss is -log p_b of that bin."""
    cfg, bt = _rays(CUBE, 16)
    th = sg.parity_params(CUBE, seed=2, grid_std=0.3).astype(np.float64)
    q = _random_q(5)
    R, N = bt["t"].shape
    width = (np.float32(cfg.far_m) - np.float32(cfg.near_m)) / np.float32(NB)
    t = np.empty((R, N), np.float32)
    bins = np.arange(R) % NB
    for i in range(R):  # every sample of ray i in the middle of bin bins[i]
        t[i] = np.float32(cfg.near_m) + (np.float32(bins[i]) + np.float32(0.5)) * width
    w = np.full((R, N), 1.0 / N)
    ce, _, n = oc.prop_ce(cfg, th, q, bt["o"], bt["r"], t, w)
    p = oc.prop_forward(cfg, th, q, bt["o"], bt["r"])
    assert n == R
    assert abs(ce - np.mean(-np.log(p[np.arange(R), bins]))) < 1e-12


def test_rays_with_little_weight_are_skipped():
    cfg, bt = _rays(CUBE, 8)
    th = sg.parity_params(CUBE, seed=2).astype(np.float64)
    w = np.zeros(bt["t"].shape)
    w[:3] = 0.5 / bt["t"].shape[1]       # sum 0.5: used
    w[3:5] = 0.9e-3 / bt["t"].shape[1]   # below 1e-3: skipped
    _, _, n = oc.prop_ce(cfg, th, _random_q(), bt["o"], bt["r"], bt["t"], w)
    assert n == 3


@pytest.mark.parametrize("h,tol", [(1e-6, 1e-6), (1e-3, 1e-4)])
def test_cross_entropy_gradient_matches_central_differences(h, tol):
    cfg, bt = _rays(TINY, 6)
    th = sg.parity_params(TINY, seed=12, grid_std=0.2).astype(np.float64)
    q = _random_q(7, 0.4)
    R, N = bt["t"].shape
    rng = np.random.default_rng(8)
    w = rng.dirichlet(np.full(N, 0.3), R) * rng.uniform(0.5, 1.0, (R, 1))
    _, g, _ = oc.prop_ce(cfg, th, q, bt["o"], bt["r"], bt["t"], w)
    fd = np.empty(oc.PROP_PARAMS)
    for i in range(oc.PROP_PARAMS):
        qp, qm = q.copy(), q.copy()
        qp[i] += h
        qm[i] -= h
        fd[i] = (oc.prop_ce(cfg, th, qp, bt["o"], bt["r"], bt["t"], w, want_grad=False)[0]
                 - oc.prop_ce(cfg, th, qm, bt["o"], bt["r"], bt["t"], w, want_grad=False)[0]) / (2 * h)
    err = np.abs(fd - g) / np.abs(g).max()
    if h < 1e-5:
        assert err.max() < tol, err.max()
    else:  # a ReLU unit may switch inside [q - h, q + h]
        assert np.median(err) < tol and np.mean(err < tol) > 0.9, err.max()


def test_uniform_pdf_reproduces_stratified_samples():
    cfg, _ = _rays(CUBE, 1)
    R, N, seed, step = 40, 32, 11, 3
    D = np.zeros(R, np.float32)  # no depth: all N samples come from the proposal
    p = np.full((R, NB), 1.0 / NB, np.float32)
    out = oc.prop_sample(cfg, D, p, N, 8, seed, step)
    near, far = float(np.float32(cfg.near_m)), float(np.float32(cfg.far_m))
    for i in range(R):
        xi = np.array([(oc.draw(seed, 2, step, i, 1 + k) >> 40) * 2.0 ** -24 for k in range(N)])
        want = near + (np.arange(N) + xi) / N * (far - near)
        np.testing.assert_allclose(out["t"][i], want, rtol=0, atol=2e-5)
    assert not np.any(out["cls"])
    assert list(out["counts"][:3]) == [0, 0, 0]


def test_one_draw_per_cdf_stratum_and_guided_band():
    """For any PDF, sample k of the K proposal draws sits where the mixture CDF reaches
    [k/K, (k+1)/K) of its total; with D > 0 the guided samples lie in [D - g, D + g]."""
    cfg, _ = _rays(CUBE, 1)
    rng = np.random.default_rng(12)
    R, N, Ng = 64, 32, 8
    p = rng.dirichlet(np.full(NB, 0.2), R).astype(np.float32)
    D = np.where(np.arange(R) % 2 == 0, rng.uniform(0.5, 3.5, R), 0.0).astype(np.float32)
    out = oc.prop_sample(cfg, D, p, N, Ng, 5, 9)
    pp, C = _mixture_cdf(cfg, p)
    near = float(np.float32(cfg.near_m))
    width = float((np.float32(cfg.far_m) - np.float32(cfg.near_m)) / np.float32(NB))
    g = float(np.float32(cfg.guide_half))
    for i in range(R):
        t = out["t"][i].astype(np.float64)
        assert np.all(np.diff(t) >= 0)
        if D[i] > 0:
            band = (t >= D[i] - g - 1e-6) & (t <= D[i] + g + 1e-6)
            assert band.sum() >= Ng
        K = N - (Ng if D[i] > 0 else 0)
        # the CDF value of every sample; the K proposal draws are one per stratum
        b = np.clip(np.floor((t - near) / width).astype(int), 0, NB - 1)
        F = (np.where(b > 0, C[i][np.maximum(b - 1, 0)], 0.0) + pp[i][b] * (t - (near + b * width)) / width) / C[i][-1]
        strata = np.floor(F * K + 1e-4).astype(int)
        if D[i] > 0:
            continue  # guided samples interleave; the strata check applies to proposal-only rays
        assert sorted(np.clip(strata, 0, K - 1).tolist()) == list(range(K)), (i, strata)
    # classes follow the plain sampler's rule
    b_ = (D[:, None] - out["t"]).astype(np.float32)
    tr = np.float32(cfg.trunc)
    want = np.where(D[:, None] > 0, np.where(np.abs(b_) <= tr, 1, np.where(b_ > tr, 2, 0)), 0)
    assert np.array_equal(out["cls"], want)


def test_concentrated_pdf_puts_most_draws_in_its_bin():
    cfg, _ = _rays(CUBE, 1)
    R, N = 16, 32
    p = np.zeros((R, NB), np.float32)
    p[np.arange(R), np.arange(R) + 4] = 1.0
    out = oc.prop_sample(cfg, np.zeros(R, np.float32), p, N, 8, 2, 2)
    near = np.float32(cfg.near_m)
    width = (np.float32(cfg.far_m) - near) / np.float32(NB)
    for i in range(R):
        b = np.clip(np.floor((out["t"][i] - near) / width), 0, NB - 1).astype(int)
        inside = int((b == i + 4).sum())
        expect = (0.95 + 0.05 / NB) * N
        assert abs(inside - expect) <= 1.0 + 1e-9, (i, inside, expect)
