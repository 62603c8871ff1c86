"""Pins of the oracle's Eikonal term (Sec. 3.3 Eq. eikonal_loss, batch normalisation of
Sec. 3.4) against closed forms, an invariant and central finite differences of its own
loss value."""
import math

import numpy as np
import pytest

import oracle as oc
import scenegen as sg
from helpers import CUBE, TINY, hand_batch, passthrough_decoder, set_level_field, zero_params


def _inside_batch(seed=0, R=12, N=20):
    """Rays whose samples all stay inside the cube workload's grid box (no clamped axis),
    with a mix of free-space, near-surface and unsupervised samples."""
    rng = np.random.default_rng(seed)
    o = rng.uniform(-0.5, 0.5, (R, 3))
    r = rng.normal(size=(R, 3))
    r /= np.linalg.norm(r, axis=1, keepdims=True)
    t = np.sort(rng.uniform(0.0, 0.6, (R, N)), axis=1)
    D = rng.uniform(0.25, 0.55, R)
    D[-1] = 0.0  # a ray without depth: no sample of it is supervised
    return hand_batch(o, r, t, D, trunc=0.1)


@pytest.mark.parametrize("n", [(0.3, -0.7, 0.2), (1.1, 0.9, -0.8), (0.6, 0.0, 0.8)])
def test_affine_field_closed_form(n):
    """phi = z_9 (pass-through decoder) on the affine field n . x + 10 of level 2: grad_x phi
    = n at every interior point, so L_eik = (1 - |n|)^2 for any set of free-space samples.
    Only the active pass-through unit (z_9 > 0 everywhere) gets decoder gradient:
    dL/dW2[0][0] = dL/dW1[0][9] = -2 (1 - |n|) |n|; every other decoder entry is 0.  The
    grid gradient lives on feature 1 of level 2 and sums to 0 over the vertices (the corner
    weights' x-derivatives sum to zero in every cell)."""
    n = np.asarray(n, np.float64)
    th = zero_params(CUBE).astype(np.float64)
    set_level_field(CUBE, th, 2, 1, lambda X: X @ n + 10.0)
    passthrough_decoder(CUBE, th, 9)
    cfg = oc.make_config(CUBE)
    bt = _inside_batch()
    n_fs = int((bt["cls"] == oc.CLS_FS).sum())
    assert 0 < n_fs < bt["cls"].size
    loss, g, nf, gnorm = oc.eikonal(cfg, th, bt, dscale=1.0)
    nn = np.linalg.norm(n)
    assert nf == n_fs
    assert abs(loss - (1 - nn) ** 2) < 1e-12
    fs = bt["cls"] == oc.CLS_FS
    np.testing.assert_allclose(gnorm[fs], nn, rtol=1e-12)
    assert np.all(gnorm[~fs] == -1)
    offs, n_grid, n_tot = CUBE.layout()
    m = sg.mlp_views(g, n_grid)
    want = -2 * (1 - nn) * nn
    assert abs(m["W2"][0, 0] - want) < 1e-12 and abs(m["W1"][0, 9] - want) < 1e-12
    dec = g[n_grid:].copy()
    mv = sg.mlp_views(np.r_[np.zeros(n_grid), dec], n_grid)
    mv["W2"][0, 0] = 0.0
    mv["W1"][0, 9] = 0.0
    assert np.abs(mv["W2"]).max() < 1e-12 and np.abs(mv["W1"]).max() < 1e-12
    assert not np.any(mv["b1"]) and not np.any(mv["b2"]) and not np.any(mv["W3"]) and not np.any(mv["kappa"])
    n2 = int(np.prod(CUBE.dims[2])) * 4
    lvl = g[offs[2]:offs[2] + n2].reshape(-1, 4)
    other = np.r_[g[:offs[2]], g[offs[2] + n2:n_grid], lvl[:, [0, 2, 3]].ravel()]
    assert not np.any(other)
    if abs(1 - nn) > 1e-9:
        assert np.abs(lvl[:, 1]).max() > 0
    assert abs(lvl[:, 1].sum()) < 1e-9 * max(np.abs(lvl[:, 1]).max(), 1e-30) * n_fs


def test_unit_gradient_field_has_zero_loss_and_gradient():
    th = zero_params(CUBE).astype(np.float64)
    u = np.array([0.48, -0.6, 0.64])  # |u| = 1
    set_level_field(CUBE, th, 3, 0, lambda X: X @ u + 10.0)
    passthrough_decoder(CUBE, th, 12)
    cfg = oc.make_config(CUBE)
    loss, g, _, _ = oc.eikonal(cfg, th, _inside_batch(1))
    assert loss < 1e-24 and np.abs(g).max() < 1e-11


def test_empty_free_space_set():
    th = sg.parity_params(TINY, seed=3).astype(np.float64)
    cfg = oc.make_config(TINY)
    bt = _inside_batch(2)
    bt["cls"][:] = oc.CLS_TR
    loss, g, nf, gnorm = oc.eikonal(cfg, th, bt)
    assert nf == 0 and loss == 0.0 and not np.any(g) and np.all(gnorm == -1)


def test_batch_mean_invariant_under_repetition_and_linear_in_seed():
    """L_eik is a mean over S_fs: the batch repeated twice gives the same loss and the same
    gradient; the gradient is linear in the upstream seed."""
    th = sg.parity_params(TINY, seed=5, grid_std=0.2).astype(np.float64)
    cfg = oc.make_config(TINY)
    bt = _inside_batch(3, R=8, N=16)
    l1, g1, n1, _ = oc.eikonal(cfg, th, bt)
    bt2 = {k: np.concatenate([v, v]) for k, v in bt.items()}
    l2, g2, n2, _ = oc.eikonal(cfg, th, bt2)
    assert n2 == 2 * n1 and abs(l2 - l1) < 1e-13 * max(1.0, l1)
    np.testing.assert_allclose(g2, g1, rtol=1e-10, atol=1e-15)
    _, g3, _, _ = oc.eikonal(cfg, th, bt, dscale=-2.5)
    np.testing.assert_allclose(g3, -2.5 * g1, rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("h,tol", [(1e-6, 1e-6), (1e-3, 1e-4)])
def test_gradient_matches_central_differences(h, tol):
    """dL_eik/dtheta (grid through d z/d x, decoders through d phi/d z) against central
    differences of the oracle's own L_eik, on the sampled tiny problem."""
    fr = sg.make_frames(TINY)
    cfg = oc.make_config(TINY)
    F = oc.OcFramesHolder(fr)
    bt = oc.sample_rays(cfg, F, 3, 0, TINY.rays)
    assert (bt["cls"] == oc.CLS_FS).sum() >= 10
    th = sg.parity_params(TINY, seed=12, grid_std=0.2).astype(np.float64)
    th[-1] = math.log(8.0)
    _, n_grid, n_tot = TINY.layout()
    loss, g, _, _ = oc.eikonal(cfg, th, bt)
    assert loss > 1e-3
    touched = np.nonzero(g[:n_grid])[0]
    assert len(touched) > 100
    dec = np.nonzero(g[n_grid:])[0] + n_grid
    assert len(dec) > 100  # W1 and row 0 of W2
    idx = np.r_[touched[::2], dec]
    fd = np.empty(len(idx))
    for j, i in enumerate(idx):
        xp, xm = th.copy(), th.copy()
        xp[i] += h
        xm[i] -= h
        fd[j] = (oc.eikonal(cfg, xp, bt, want_grad=False)[0] - oc.eikonal(cfg, xm, bt, want_grad=False)[0]) / (2 * h)
    err = np.abs(fd - g[idx]) / np.abs(g[idx]).max()
    # at h = 1e-3 a ReLU unit of some point may switch inside [theta - h, theta + h]
    assert (np.median(err) < tol and np.mean(err < tol) > 0.98) if h > 1e-5 else err.max() < tol, err.max()
    # entries the term cannot reach: kappa, b1, b2, the colour decoder
    offs = dict(zip([nm for nm, _ in sg.MLP_SHAPES], np.cumsum([0] + [int(np.prod(s)) for _, s in sg.MLP_SHAPES])))
    assert not np.any(g[n_grid + offs["W3"]:])
    assert not np.any(g[n_grid + offs["b1"]:n_grid + offs["W2"]])
    assert not np.any(g[n_grid + offs["b2"]:n_grid + offs["W3"]])
