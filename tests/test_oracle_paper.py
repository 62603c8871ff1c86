"""Pins of the oracle's paper architecture (Sec. 3.1 Eq. SDF_MLP, Eq. COLOR_MLP and the
architecture details: colour grid W_beta with h_c = 6 at the finest level, a colour decoder
fed W_beta(x) and the viewing direction, two hidden layers of 32 in both decoders).

Closed forms with pass-through decoders (weights that make phi or a colour channel equal one
feature exactly), exact reproduction of affine colour fields by the trilinear colour gather,
the unit viewing direction, and central finite differences of the oracle's own forward pass
for every parameter (geometry grid, colour grid, both decoders, kappa), including the
second-order path of the smoothness term.
"""
import math

import numpy as np
import pytest

import oracle as oc
import scenegen as sg
from helpers import CUBE, TINY, hand_batch, set_level_field

CUBE_P = sg.WORKLOADS["cube-paper-1024x64"]
TINY_P = TINY.with_(name="tiny-16-paper", arch="paper")
B = 3.0  # bias that keeps a pass-through unit on for |value| < B


def _views(w, th):
    return sg.mlp_views(th, w.layout()[1], sg.PAPER_MLP_SHAPES)


def passthrough_paper(w, th, zindex=None, cindex=None, kappa=math.log(20.0)):
    """Decoders with phi = z[zindex] and every colour channel = sigmoid(u[cindex]) exactly
    (u = [W_beta(x), d]): relu(v + B) - relu(B - v) = 2v carried through both hidden layers."""
    _, n_grid, _ = w.layout()
    th[n_grid:] = 0.0
    m = _views(w, th)
    if zindex is not None:
        m["gW1"][0, zindex], m["gW1"][1, zindex] = 1.0, -1.0
        m["gb1"][0] = m["gb1"][1] = B
        m["gW2"][0, 0], m["gW2"][0, 1] = 0.5, -0.5  # = v, unit 0 of layer 2 then holds v + B
        m["gb2"][0] = B
        m["gw3"][0, 0] = 1.0
        m["gb3"][0] = -B
    if cindex is not None:
        m["cW1"][0, cindex], m["cW1"][1, cindex] = 1.0, -1.0
        m["cb1"][0] = m["cb1"][1] = B
        m["cW2"][0, 0], m["cW2"][0, 1] = 0.5, -0.5
        m["cb2"][0] = B
        m["cW3"][:, 0] = 1.0
        m["cb3"][:] = -B
    m["kappa"][0] = kappa
    return th


def test_layout_matches_the_oracle_count():
    cfg = oc.make_config(CUBE_P)
    offs, n_grid, n_tot = CUBE_P.layout()
    assert oc.paper_param_count(cfg) == (n_tot, n_grid)
    nx, ny, nz = CUBE_P.dims[3]
    assert CUBE_P.colour_floats() >= nx * ny * nz * 6 and CUBE_P.colour_floats() % 4 == 0
    # 16*32+32 + 32*32+32 + 32+1 + 9*32+32 + 32*32+32 + 3*32+3 + 1
    assert sg.PAPER_MLP_PARAMS == 3109


def _plane_batch(shift, R=8, N=40):
    rng = np.random.default_rng(6)
    o = np.c_[np.full(R, -1.0), rng.uniform(-0.5, 0.5, (R, 2))]
    r = np.tile([1.0, 0.0, 0.0], (R, 1))
    t = np.sort(rng.uniform(0.3, 1.8, (R, N)), axis=1)
    return hand_batch(o, r, t, np.full(R, 1.5))


@pytest.mark.parametrize("shift", [0.0, 0.03, -0.03])
def test_plane_sdf_losses_through_two_hidden_layers(shift):
    """phi = b + shift through the 2-hidden-layer geometry decoder: L_sdf = |shift| on S_tr,
    L_fs = max(0, shift) on S_fs (as for the workload's decoders)."""
    th = np.zeros(CUBE_P.layout()[2], np.float32)
    set_level_field(CUBE_P, th, 3, 2, lambda X: (0.5 - X[..., 0]) + shift)
    passthrough_paper(CUBE_P, th, zindex=14)
    bt = _plane_batch(shift)
    out = oc.step(oc.make_config(CUBE_P), th, bt, None, want_grad=False)
    assert abs(out["loss"][2] - abs(shift)) < 2e-6
    assert abs(out["loss"][3] - max(0.0, shift)) < 2e-6


def _colour_case(field, cindex, rays):
    """Plane geometry (phi = 0.5 - x) and a colour feature set by `field` at the colour-grid
    vertices; the colour decoder passes u[cindex] through a sigmoid."""
    th = np.zeros(CUBE_P.layout()[2], np.float32)
    set_level_field(CUBE_P, th, 3, 2, lambda X: 0.5 - X[..., 0])
    passthrough_paper(CUBE_P, th, zindex=14, cindex=cindex)
    if field is not None:
        sg.colour_view(CUBE_P, th)[..., cindex] = field(sg.vertex_positions(CUBE_P, 3))
    o, r, t = rays
    bt = hand_batch(o, r, t, np.full(len(o), 1.5))
    out = oc.step(oc.make_config(CUBE_P), th, bt, None, want_grad=False, want_weights=True)
    return bt, out


def _rays(R=6, N=48, seed=9, spread=0.3):
    rng = np.random.default_rng(seed)
    o = np.c_[np.full(R, -1.0), rng.uniform(-0.4, 0.4, (R, 2))]
    r = np.c_[np.ones(R), rng.uniform(-spread, spread, (R, 2))]
    t = np.sort(rng.uniform(0.3, 2.2, (R, N)), axis=1)
    return o, r, t


def test_colour_grid_reproduces_affine_fields():
    """An affine colour feature is reproduced exactly by the trilinear colour gather, so the
    rendered colour is sum_k w_k sigmoid(a . x_k + a0) with the oracle's own weights w_k
    (pinned by the compositing tests) and x_k = o + t_k r in binary32."""
    a, a0 = np.array([0.7, -1.3, 0.4]), 0.2
    for cindex in (0, 3, 5):
        bt, out = _colour_case(lambda X: X @ a + a0, cindex, _rays())
        x = (bt["o"][:, None, :] + (bt["t"][..., None] * bt["r"][:, None, :]).astype(np.float32)).astype(np.float64)
        want = (out["w"] * (1.0 / (1.0 + np.exp(-(x @ a + a0))))).sum(1)
        for j in range(3):
            np.testing.assert_allclose(out["rgb_hat"][:, j], want, rtol=0, atol=1e-6)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_colour_reads_the_unit_viewing_direction(axis):
    """With the colour decoder passing d[axis] through (u = [W_beta, d], d = r / |r|), every
    sample of a ray has colour sigmoid(r[axis] / |r|): c_hat = wsum sigmoid(r[axis] / |r|)."""
    bt, out = _colour_case(None, 6 + axis, _rays(spread=0.6))
    r = bt["r"].astype(np.float64)
    d = r[:, axis] / np.linalg.norm(r, axis=1)
    want = out["wsum"] / (1.0 + np.exp(-d))
    for j in range(3):
        np.testing.assert_allclose(out["rgb_hat"][:, j], want, rtol=0, atol=1e-12)


def test_smoothness_bilinear_closed_form_two_hidden_layers():
    """phi = x y (in the trilinear span): grad phi = (y, x, 0), so the smoothness term is
    mean(eps_x^2 + eps_y^2) through the two-hidden-layer decoder's d phi / d z."""
    th = np.zeros(CUBE_P.layout()[2], np.float32)
    set_level_field(CUBE_P, th, 3, 0, lambda X: X[..., 0] * X[..., 1])
    passthrough_paper(CUBE_P, th, zindex=12)
    rng = np.random.default_rng(8)
    P = 64
    xs = rng.uniform(-0.9, 0.9, (P, 3)).astype(np.float32)
    v = rng.normal(size=(P, 3))
    eps = (0.004 * v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    sm = dict(xs=xs, eps=eps, valid=np.ones(P, np.uint8))
    bt = _plane_batch(0.0, R=1, N=4)
    out = oc.step(oc.make_config(CUBE_P), th, bt, sm, want_grad=False)
    e = eps.astype(np.float64)
    want = (e[:, 0] ** 2 + e[:, 1] ** 2).mean()
    assert abs(out["loss"][4] - want) < 1e-5 * want


def test_second_layer_is_not_transposed():
    """A decoder whose second layer is not symmetric: phi = relu(z0 + B) - relu(z1 + B) routed
    through gW2[0] = (1, -1) only; swapping to gW2^T would route unit 1 through row 1 (zero).
    With z0 = 0.3 and z1 = 0.1 everywhere: phi = 0.2, so the constant-phi free-space loss is
    max(0, exp(-5 * 0.2) - 1, 0.2 - b) = max(0, 0.2 - b) on S_fs and the sdf loss on S_tr is
    |0.2 - b|."""
    th = np.zeros(CUBE_P.layout()[2], np.float32)
    set_level_field(CUBE_P, th, 0, 0, lambda X: np.full(X.shape[:-1], 0.3))
    set_level_field(CUBE_P, th, 0, 1, lambda X: np.full(X.shape[:-1], 0.1))
    _, n_grid, _ = CUBE_P.layout()
    m = _views(CUBE_P, th)
    m["gW1"][0, 0], m["gW1"][1, 1] = 1.0, 1.0
    m["gb1"][0] = m["gb1"][1] = B
    m["gW2"][0, 0], m["gW2"][0, 1] = 1.0, -1.0
    m["gb2"][0] = B
    m["gw3"][0, 0], m["gb3"][0] = 1.0, -B
    m["kappa"][0] = math.log(20.0)
    bt = _plane_batch(0.0)
    out = oc.step(oc.make_config(CUBE_P), th, bt, None, want_grad=False)
    b = (bt["D"][:, None].astype(np.float64) - bt["t"].astype(np.float64))
    tr = bt["cls"] == 1
    assert abs(out["loss"][2] - np.abs(0.2 - b[tr]).mean()) < 1e-6
    fs = bt["cls"] == 2
    assert abs(out["loss"][3] - np.maximum(0.0, 0.2 - b[fs]).mean()) < 1e-6
    assert out["loss"][3] > 0


# ----------------------------------------------------------------------------------------
# gradients: central differences of the oracle's forward pass
# ----------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tiny_paper():
    fr = sg.make_frames(TINY_P)
    cfg = oc.make_config(TINY_P)
    F = oc.OcFramesHolder(fr)
    bt = oc.sample_rays(cfg, F, 3, 0, TINY_P.rays)
    sm = oc.sample_smooth(cfg, F, 3, 0, TINY_P.n_smooth)
    th = sg.paper_sdf_params(TINY_P, sg.cube_scene(), seed=12, grid_std=0.1).astype(np.float64)
    th[-1] = math.log(8.0)
    return cfg, bt, sm, th


def _fd(cfg, bt, sm, th, dloss, h, idx):
    def total(x):
        lo = oc.step(cfg, x, bt, sm, want_grad=False)["loss"]
        return lo[5] if dloss is None else float(np.dot(lo, dloss))

    fd = np.zeros(len(idx))
    for j, i in enumerate(idx):
        x = th.copy()
        x[i] += h
        fp = total(x)
        x[i] -= 2 * h
        fd[j] = (fp - total(x)) / (2 * h)
    return fd


def _check(tiny, dloss, h=1e-6, tol=1e-6, stride=1):
    cfg, bt, sm, th = tiny
    offs, n_grid, n_tot = TINY_P.layout()
    out = oc.step(cfg, th, bt, sm, dloss=dloss, want_margins=True)
    assert out["margins"][0] > 1e-2, out["margins"]  # every hidden unit clear of its kink
    g = out["grad"]
    touched = np.nonzero(g[:n_grid])[0]
    col = touched[touched >= TINY_P.colour_offset()]
    idx = np.r_[touched[::stride], np.arange(n_grid, n_tot, stride)]
    fd = _fd(cfg, bt, sm, th, dloss, h, idx)
    err = np.abs(fd - g[idx]).max() / np.abs(g[idx]).max()
    assert err < tol, err
    return g, col


def test_paper_gradients_match_central_differences(tiny_paper):
    g, col = _check(tiny_paper, None)
    assert len(col) > 20  # the colour grid receives gradient


def test_paper_gradients_match_central_differences_per_term_seeds(tiny_paper):
    _check(tiny_paper, np.array([0.3, -1.1, 0.7, 2.0, 5.0, 0.25]), stride=2)


def test_paper_smoothness_second_order_gradient_alone(tiny_paper):
    """The smoothness term alone: d/dtheta and d/domega through grad_x phi of the
    two-hidden-layer decoder; the colour parameters get none of it."""
    cfg, bt, sm, th = tiny_paper
    offs, n_grid, n_tot = TINY_P.layout()
    g, _ = _check(tiny_paper, np.array([0, 0, 0, 0, 1.0, 0]))
    m = sg.mlp_views(g, n_grid, sg.PAPER_MLP_SHAPES)
    assert np.abs(m["gW1"]).max() > 0 and np.abs(m["gW2"]).max() > 0 and np.abs(m["gw3"]).max() > 0
    for k in ("gb1", "gb2", "gb3", "cW1", "cb1", "cW2", "cb2", "cW3", "cb3"):
        assert np.abs(m[k]).max() == 0, k
    assert np.abs(g[TINY_P.colour_offset():n_grid]).max() == 0


def test_paper_gradients_h1e3(tiny_paper):
    """The h = 1e-3 central-difference check."""
    _check(tiny_paper, None, h=1e-3, tol=1e-4, stride=3)


# ----------------------------------------------------------------------------------------
# the SDF query, its reverse mode, the Eikonal term, the importance sampler and mesh
# extraction with the paper's architecture
# ----------------------------------------------------------------------------------------
def _affine_passthrough(w, n, c0=0.1):
    th = np.zeros(w.layout()[2], np.float32)
    set_level_field(w, th, 3, 0, lambda X: X @ np.asarray(n) + c0)
    return passthrough_paper(w, th, zindex=12)


def test_paper_query_affine_field_closed_form():
    """phi = n . x + c through the two-hidden-layer decoder: the query returns it and its
    gradient n exactly (inside the grid box)."""
    n = np.array([0.3, -0.6, 0.2])
    th = _affine_passthrough(CUBE_P, n)
    x = np.random.default_rng(3).uniform(-1.2, 1.2, (200, 3)).astype(np.float32)
    phi, g = oc.query_sdf(oc.make_config(CUBE_P), th, x)
    np.testing.assert_allclose(phi, x.astype(np.float64) @ n + 0.1, atol=2e-6)
    np.testing.assert_allclose(g, np.tile(n, (len(x), 1)), atol=2e-6)


def test_paper_query_gradient_matches_central_differences_in_x(tiny_paper):
    """grad_x phi against central differences of phi along each axis, for points whose two
    probes stay in the same cell of every level (phi is multilinear per cell and the
    decoder is linear on its piece, so the difference quotient is exact up to rounding)."""
    cfg, _, _, th = tiny_paper
    rng = np.random.default_rng(4)
    x = rng.uniform(-1.1, 1.1, (300, 3)).astype(np.float32)
    phi, g = oc.query_sdf(cfg, th, x)
    h = np.float32(1e-3)
    checked = 0
    for a in range(3):
        xp, xm = x.copy(), x.copy()
        xp[:, a] += h
        xm[:, a] -= h
        same = np.all(oc.voxel_index(cfg, xp) == oc.voxel_index(cfg, xm), axis=1)
        fp, _ = oc.query_sdf(cfg, th, xp, want_grad=False)
        fm, _ = oc.query_sdf(cfg, th, xm, want_grad=False)
        fd = (fp - fm) / (xp[:, a].astype(np.float64) - xm[:, a].astype(np.float64))
        np.testing.assert_allclose(fd[same], g[same, a], rtol=1e-6, atol=1e-7)
        checked += same.sum()
    assert checked > 600


def test_paper_query_backward_matches_central_differences(tiny_paper):
    """d/dtheta of sum dsdf phi + dgrad . grad_x phi (both terms, and the second alone)."""
    cfg, _, _, th = tiny_paper
    offs, n_grid, n_tot = TINY_P.layout()
    rng = np.random.default_rng(5)
    x = rng.uniform(-1.0, 1.0, (40, 3)).astype(np.float32)
    dsdf, dgrad = rng.normal(size=40), rng.normal(size=(40, 3))
    for ds in (dsdf, None):
        g = oc.query_sdf_backward(cfg, th, x, ds, dgrad)

        def obj(t):
            p, gr = oc.query_sdf(cfg, t, x)
            return (0.0 if ds is None else float(p @ ds)) + float((gr * dgrad).sum())

        idx = np.r_[np.nonzero(g[:n_grid])[0][::5], np.arange(n_grid, n_tot, 3)]
        fd = []
        for i in idx:
            t = th.copy()
            t[i] += 1e-6
            fp = obj(t)
            t[i] -= 2e-6
            fd.append((fp - obj(t)) / 2e-6)
        fd = np.array(fd)
        assert np.abs(fd - g[idx]).max() <= 1e-6 * np.abs(g[idx]).max()
        m = sg.mlp_views(g, n_grid, sg.PAPER_MLP_SHAPES)
        assert all(np.abs(m[k]).max() == 0 for k in ("cW1", "cb1", "cW2", "cb2", "cW3", "cb3", "kappa"))
        assert np.abs(g[TINY_P.colour_offset():n_grid]).max() == 0


def test_paper_eikonal_affine_closed_form_and_central_differences(tiny_paper):
    """L_eik = (1 - |n|)^2 for phi = n . x + c; the gradient matches central differences."""
    n = np.array([0.3, -0.6, 0.2])
    th = _affine_passthrough(CUBE_P, n)
    bt = _plane_batch(0.0)
    le, _, nfs, gn = oc.eikonal(oc.make_config(CUBE_P), th, bt, want_grad=False)
    assert nfs > 0 and abs(le - (1 - np.linalg.norm(n)) ** 2) < 1e-7  # binary32 vertex values
    cfg, bt2, _, th2 = tiny_paper
    offs, n_grid, n_tot = TINY_P.layout()
    le, g, nfs, _ = oc.eikonal(cfg, th2, bt2)
    assert nfs > 10 and le > 0
    idx = np.r_[np.nonzero(g[:n_grid])[0][::3], np.arange(n_grid, n_tot, 2)]
    fd = []
    for i in idx:
        t = th2.copy()
        t[i] += 1e-6
        fp = oc.eikonal(cfg, t, bt2, want_grad=False)[0]
        t[i] -= 2e-6
        fd.append((fp - oc.eikonal(cfg, t, bt2, want_grad=False)[0]) / 2e-6)
    assert np.abs(np.array(fd) - g[idx]).max() <= 1e-6 * np.abs(g[idx]).max()


def _compact_twin(th_paper, w_paper, w_compact, kappa):
    """The workload's model with the same geometry grid and a pass-through decoder of z[12]."""
    from helpers import passthrough_decoder
    th = np.zeros(w_compact.layout()[2], np.float32)
    ng = w_compact.layout()[1]
    th[:ng] = th_paper[:ng]
    return passthrough_decoder(w_compact, th, 12, kappa=kappa)


def test_paper_importance_sampler_reduces_to_the_workload_model():
    """With phi = z[12] in both models (same geometry grid, same kappa) the importance
    sampler draws the same depths for the paper's architecture as for the workload's."""
    wp = CUBE_P.with_(imp_coarse=32, imp_steps=2, imp_per_step=8, rays=64)
    wc = CUBE.with_(imp_coarse=32, imp_steps=2, imp_per_step=8, rays=64)
    fr = sg.make_frames(wp)
    th_p = np.zeros(wp.layout()[2], np.float32)
    set_level_field(wp, th_p, 3, 0, lambda X: np.linalg.norm(X - [-0.4, 0, 0], axis=-1) - 0.5)
    passthrough_paper(wp, th_p, zindex=12, kappa=math.log(60.0))
    th_c = _compact_twin(th_p, wp, wc, math.log(60.0))
    outs = []
    for w, th in ((wp, th_p), (wc, th_c)):
        cfg = oc.make_config(w)
        outs.append(oc.sample_importance(cfg, oc.OcFramesHolder(fr), th, 3, 1, w.rays, 32, 2, 8))
    a, b = outs
    np.testing.assert_allclose(a["phi"], b["phi"], atol=1e-12)
    same = (a["t"] == b["t"]).mean()
    assert same > 0.999 and np.abs(a["t"] - b["t"]).max() < 1e-5


def test_paper_mesh_reduces_to_the_workload_model():
    """With phi = z[12] in both models the lattice values agree to rounding and the
    isosurface has the same triangles."""
    th_p = np.zeros(CUBE_P.layout()[2], np.float32)
    set_level_field(CUBE_P, th_p, 3, 0, lambda X: np.linalg.norm(X - [-0.4, 0, 0], axis=-1) - 0.5)
    passthrough_paper(CUBE_P, th_p, zindex=12)
    th_c = _compact_twin(th_p, CUBE_P, CUBE, math.log(20.0))
    lo, step, dims = (-1.0, -0.7, -0.7), 0.05, (25, 29, 29)
    tp, pp = oc.extract_mesh(oc.make_config(CUBE_P), th_p, lo, step, dims)
    tc, pc = oc.extract_mesh(oc.make_config(CUBE), th_c, lo, step, dims)
    np.testing.assert_allclose(pp, pc, atol=1e-12)
    assert len(tp) == len(tc) > 500


# ----------------------------------------------------------------------------------------
# camera-pose refinement with the paper's architecture: the poses reach the losses through
# the sample positions (geometry and colour grids) and through the viewing direction
# ----------------------------------------------------------------------------------------
W3P = TINY_P.with_(name="tiny-3frames-paper", frames=3, rays=48)
DLOSS_POSE = np.array([1.0, 1.0, 0.0, 0.0, 0.0, 0.0])  # L_rgb + L_d (the SDF terms have kinks)


@pytest.fixture(scope="module")
def posed_paper():
    """Three frames with pose corrections; affine geometry and colour fields (trilinear is
    exact) through pass-through decoders, the colour also reading the viewing direction, so
    that the losses are smooth in the poses."""
    fr = sg.make_frames(W3P)
    cfg = oc.make_config(W3P)
    rng = np.random.default_rng(7)
    xi = np.c_[rng.normal(0, 0.02, (3, 3)), rng.normal(0, 0.02, (3, 3))]
    c2w = oc.pose_apply(fr.c2w, xi)
    F = oc.OcFramesHolder(fr, c2w=c2w)
    bt = oc.sample_rays(cfg, F, 3, 0, W3P.rays)
    th = np.zeros(W3P.layout()[2], np.float32)
    set_level_field(W3P, th, 3, 0, lambda X: X @ np.array([0.3, -0.4, 0.85]) + 0.1)
    sg.colour_view(W3P, th)[..., 2] = sg.vertex_positions(W3P, 3) @ np.array([0.6, 0.3, -0.5])
    passthrough_paper(W3P, th, zindex=12, cindex=2, kappa=math.log(6.0))
    m = _views(W3P, th)
    m["cW1"][0, 7], m["cW1"][1, 7] = 1.0, -1.0  # colour = sigmoid(W_beta_2 + d_y)
    return fr, cfg, xi, c2w, F, bt, th.astype(np.float64)


def _pose_loss(fr, cfg, th, bt, xi):
    c2w = oc.pose_apply(fr.c2w, xi)
    o, r = oc.rays_of_pixels(oc.OcFramesHolder(fr, c2w=c2w), bt["pix"])
    return float(np.dot(oc.step(cfg, th, dict(bt, o=o, r=r), None, want_grad=False)["loss"], DLOSS_POSE))


def test_paper_pose_gradient_matches_central_differences(posed_paper):
    fr, cfg, xi, c2w, F, bt, th = posed_paper
    out = oc.step_dz(cfg, th, bt, None, dloss=DLOSS_POSE)
    assert out["dz"].shape[2] == 32 and np.abs(out["dz"][..., 22:25]).max() > 0
    g = oc.pose_grad(cfg, F, th, c2w, xi, bt, out["dz"])
    assert np.abs(g[:, :3]).max() > 1e-2 and np.abs(g[:, 3:]).max() > 1e-2
    fd = np.zeros_like(g)
    h = 3e-4
    for f in range(3):
        for c in range(6):
            xp, xm = xi.copy(), xi.copy()
            xp[f, c] += h
            xm[f, c] -= h
            fd[f, c] = (_pose_loss(fr, cfg, th, bt, xp) - _pose_loss(fr, cfg, th, bt, xm)) / (2 * h)
    err = np.abs(fd - g).max() / np.abs(g).max()
    assert err < 5e-4, (err, g, fd)
    # the viewing direction's share of the rotation gradient (dropping it would exceed the
    # central-difference tolerance above some 40 times)
    dz0 = out["dz"].copy()
    dz0[..., 22:25] = 0
    g0 = oc.pose_grad(cfg, F, th, c2w, xi, bt, dz0)
    assert np.abs(g0[:, 3:] - g[:, 3:]).max() > 0.02 * np.abs(g[:, 3:]).max()
    np.testing.assert_allclose(g0[:, :3], g[:, :3], rtol=1e-12, atol=1e-14)
