"""Pins of the oracle's camera-pose gradient of the Eikonal term (Sec. 3.3 Eq. eikonal_loss;
Sec. 3.4 puts the poses among the optimised parameters; the x-Hessian of the trilinear
interpolation from Supp. Sec. 1): the free-space samples move with the pose, and with them
grad_x phi, through the x-Hessian of phi.

A multilinear field (products of coordinates, which trilinear interpolation reproduces
exactly, so phi is smooth across cell faces) through the pass-through decoder gives a
constant, known x-Hessian; the gradient is checked against central differences of the
oracle's own L_eik with the rays re-formed from the perturbed poses, an affine field (zero
Hessian) gives a zero pose gradient, and planted mistakes in a copy of the oracle fail."""
import math

import numpy as np
import pytest

import oracle as oc
import scenegen as sg
from helpers import TINY, passthrough_decoder, set_level_field, zero_params

W3 = TINY.with_(name="tiny-3frames-eik", frames=3, rays=256)
W3P = W3.with_(name="tiny-3frames-eik-paper", arch="paper")


def _multilinear(X):
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    return 0.3 * x * y + 0.2 * y * z - 0.25 * x * z + 0.5 * x - 0.4 * y + 0.85 * z + 0.1


def _posed(w, field, paper=False):
    fr = sg.make_frames(w)
    cfg = oc.make_config(w)
    rng = np.random.default_rng(7)
    xi = np.c_[rng.normal(0, 0.02, (3, 3)), rng.normal(0, 0.02, (3, 3))]
    c2w = oc.pose_apply(fr.c2w, xi)
    F = oc.OcFramesHolder(fr, c2w=c2w)
    bt = oc.sample_rays(cfg, F, 3, 0, w.rays)
    th = np.zeros(w.layout()[2], np.float64)
    set_level_field(w, th, 3, 0, field)
    if paper:
        from test_oracle_paper import passthrough_paper
        passthrough_paper(w, th, zindex=12, kappa=math.log(6.0))
    else:
        passthrough_decoder(w, th, 12, kappa=math.log(6.0))
    return fr, cfg, xi, c2w, F, bt, th


def _eik_at(fr, cfg, th, bt, xi):
    c2w = oc.pose_apply(fr.c2w, xi)
    o, r = oc.rays_of_pixels(oc.OcFramesHolder(fr, c2w=c2w), bt["pix"])
    return oc.eikonal(cfg, th, dict(bt, o=o, r=r), want_grad=False)[0]


def _fd(fr, cfg, th, bt, xi, h=3e-4):
    fd = np.zeros((3, 6))
    for f in range(3):
        for c in range(6):
            xp, xm = xi.copy(), xi.copy()
            xp[f, c] += h
            xm[f, c] -= h
            fd[f, c] = (_eik_at(fr, cfg, th, bt, xp) - _eik_at(fr, cfg, th, bt, xm)) / (2 * h)
    return fd


def _check(fr, cfg, xi, c2w, F, bt, th, dscale=1.0):
    """Raises AssertionError unless the pose gradient equals central differences."""
    n_fs = int((bt["cls"] == oc.CLS_FS).sum())
    assert n_fs > 100
    g = oc.eikonal_pose_grad(cfg, F, th, c2w, xi, bt, dscale)
    fd = dscale * _fd(fr, cfg, th, bt, xi)
    assert np.abs(fd).max() > 1e-3  # the term reaches every frame's pose
    err = np.abs(fd - g).max() / np.abs(fd).max()
    assert err < 5e-4, (err, g, fd)


@pytest.fixture(scope="module")
def posed():
    return _posed(W3, _multilinear)


def test_eikonal_pose_gradient_matches_central_differences(posed):
    _check(*posed)


def test_eikonal_pose_gradient_is_linear_in_the_seed(posed):
    fr, cfg, xi, c2w, F, bt, th = posed
    g1 = oc.eikonal_pose_grad(cfg, F, th, c2w, xi, bt, 1.0)
    g2 = oc.eikonal_pose_grad(cfg, F, th, c2w, xi, bt, -2.5)
    np.testing.assert_allclose(g2, -2.5 * g1, rtol=1e-12, atol=1e-15)


def test_affine_field_has_no_eikonal_pose_gradient():
    """grad_x phi is constant on an affine field (zero Hessian): L_eik does not change with
    the poses, and neither do its sample positions' gradients."""
    fr, cfg, xi, c2w, F, bt, th = _posed(W3, lambda X: X @ np.array([0.3, -0.4, 0.85]) + 0.1)
    g = oc.eikonal_pose_grad(cfg, F, th, c2w, xi, bt)
    assert np.abs(g).max() < 1e-12


def test_paper_architecture_eikonal_pose_gradient():
    """The same with the paper's two-hidden-layer geometry decoder carrying phi = z[12]."""
    _check(*_posed(W3P, _multilinear, paper=True))


PLANTED = {
    # the Hessian in metres needs 1 / v^2 (cell coordinates to metres, twice)
    "one_over_v": [("const double iv2 = cells[l].inv_v * cells[l].inv_v;", "const double iv2 = cells[l].inv_v;")],
    # the rotation's moment weighs each sample's position gradient by its depth
    "no_depth": [("        gr[a] += (double)t[s] * v;", "        gr[a] += v;")],
    # the Eikonal adjoint's sign
    "sign": [("const double kk = dscale * (-2.0 / (double)n_fs) * (1.0 - nrm) / nrm;",
              "const double kk = dscale * (2.0 / (double)n_fs) * (1.0 - nrm) / nrm;")],
}


@pytest.mark.parametrize("mistake", sorted(PLANTED))
def test_eikonal_pose_pins_catch_planted_mistakes(posed, mistake):
    so = oc.build_variant(PLANTED[mistake], mistake)
    with oc.using_variant(so):
        with pytest.raises(AssertionError):
            _check(*posed)
