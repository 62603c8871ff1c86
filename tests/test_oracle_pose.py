"""Pins of the oracle's camera-pose refinement (Sec. 3.4: the poses are parameters; Sec. 4:
translation t in R^3 and nu in so(3)): the rotation map against closed forms, and the pose
gradient of the per-ray losses against central differences of the oracle's own loss with
the rays re-formed from the perturbed poses."""
import math

import numpy as np
import pytest

import oracle as oc
import scenegen as sg
from helpers import TINY, passthrough_decoder, set_level_field, zero_params

W3 = TINY.with_(name="tiny-3frames", frames=3, rays=48)


def test_rotation_map_closed_forms():
    c2w0 = np.tile(np.c_[np.eye(3), np.zeros(3)][None], (3, 1, 1)).astype(np.float32)
    a = 0.7
    xi = np.array([[0, 0, 0, 0, 0, a], [0.1, -0.2, 0.3, a, 0, 0], [0, 0, 0, 1e-6, -2e-6, 3e-6]])
    c2w = oc.pose_apply(c2w0, xi)
    Rz = np.array([[math.cos(a), -math.sin(a), 0], [math.sin(a), math.cos(a), 0], [0, 0, 1]])
    Rx = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    np.testing.assert_allclose(c2w[0, :, :3], Rz, atol=1e-15)
    np.testing.assert_allclose(c2w[1, :, :3], Rx, atol=1e-15)
    np.testing.assert_allclose(c2w[1, :, 3], [0.1, -0.2, 0.3], atol=1e-15)
    # near zero: I + [nu]_x to first order, orthonormal
    nu = xi[2, 3:]
    K = np.array([[0, -nu[2], nu[1]], [nu[2], 0, -nu[0]], [-nu[1], nu[0], 0]])
    np.testing.assert_allclose(c2w[2, :, :3], np.eye(3) + K + K @ K / 2, atol=1e-15)
    rng = np.random.default_rng(0)
    for _ in range(5):
        v = rng.normal(size=3)
        R = oc.pose_apply(c2w0[:1], np.r_[0, 0, 0, v][None])[0, :, :3]
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
        Rinv = oc.pose_apply(c2w0[:1], np.r_[0, 0, 0, -v][None])[0, :, :3]
        np.testing.assert_allclose(R @ Rinv, np.eye(3), atol=1e-14)
        np.testing.assert_allclose(R @ v, v, atol=1e-14)  # the axis is fixed


@pytest.fixture(scope="module")
def posed():
    """Three frames with pose corrections; an affine SDF (trilinear is exact: no kinks at cell
    faces) through the pass-through decoder, so that the rendering losses are smooth in the
    sample positions and central differences converge."""
    fr = sg.make_frames(W3)
    cfg = oc.make_config(W3)
    rng = np.random.default_rng(7)
    xi = np.c_[rng.normal(0, 0.02, (3, 3)), rng.normal(0, 0.02, (3, 3))]
    c2w = oc.pose_apply(fr.c2w, xi)
    F = oc.OcFramesHolder(fr, c2w=c2w)
    bt = oc.sample_rays(cfg, F, 3, 0, W3.rays)
    th = zero_params(W3).astype(np.float64)
    set_level_field(W3, th, 3, 0, lambda X: X @ np.array([0.3, -0.4, 0.85]) + 0.1)
    set_level_field(W3, th, 2, 1, lambda X: X @ np.array([0.5, 0.2, -0.1]))
    passthrough_decoder(W3, th, 12, kappa=math.log(6.0))
    return fr, cfg, xi, c2w, F, bt, th


DLOSS = np.array([1.0, 1.0, 0.0, 0.0, 0.0, 0.0])  # L_rgb + L_d (the truncated-SDF terms have kinks)


def _loss_at(fr, cfg, th, bt, xi):
    c2w = oc.pose_apply(fr.c2w, xi)
    o, r = oc.rays_of_pixels(oc.OcFramesHolder(fr, c2w=c2w), bt["pix"])
    b = dict(bt, o=o, r=r)
    return float(np.dot(oc.step(cfg, th, b, None, want_grad=False)["loss"], DLOSS))


def test_rays_of_pixels_are_the_samplers(posed):
    fr, cfg, xi, c2w, F, bt, th = posed
    o, r = oc.rays_of_pixels(F, bt["pix"])
    assert np.array_equal(o, bt["o"]) and np.array_equal(r, bt["r"])
    assert len(np.unique(bt["pix"] // (W3.height * W3.width))) == 3  # rays of every frame


def test_pose_gradient_matches_central_differences(posed):
    fr, cfg, xi, c2w, F, bt, th = posed
    out = oc.step_dz(cfg, th, bt, None, dloss=DLOSS)
    g = oc.pose_grad(cfg, F, th, c2w, xi, bt, out["dz"])
    assert np.abs(g[:, :3]).max() > 1e-2 and np.abs(g[:, 3:]).max() > 1e-2
    fd = np.zeros_like(g)
    h = 3e-4
    for f in range(3):
        for c in range(6):
            xp, xm = xi.copy(), xi.copy()
            xp[f, c] += h
            xm[f, c] -= h
            fd[f, c] = (_loss_at(fr, cfg, th, bt, xp) - _loss_at(fr, cfg, th, bt, xm)) / (2 * h)
    err = np.abs(fd - g).max() / np.abs(g).max()
    assert err < 5e-4, (err, g, fd)


def test_pose_gradient_of_a_frame_without_rays_is_zero(posed):
    fr, cfg, xi, c2w, F, bt, th = posed
    keep = bt["pix"] // (W3.height * W3.width) != 1
    sub = {k: (v[keep] if k != "counts" else v) for k, v in bt.items()}
    sub["counts"] = np.array([(sub["D"] > 0).sum(), (sub["cls"] == 1).sum(), (sub["cls"] == 2).sum(), 0])
    out = oc.step_dz(cfg, th, sub, None, dloss=DLOSS)
    g = oc.pose_grad(cfg, F, th, c2w, xi, sub, out["dz"])
    assert not np.any(g[1]) and np.abs(g[0]).max() > 0 and np.abs(g[2]).max() > 0
