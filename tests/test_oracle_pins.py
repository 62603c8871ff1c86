"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: values evaluated by hand
from the supplement's printed formulas (tests/golden), closed forms, invariants, special
cases with known answers, an independently written renderer, or central finite
differences of the oracle's own forward pass.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as oc
import scenegen as sg
from helpers import CUBE, TINY, hand_batch, passthrough_decoder, set_level_field, zero_params

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GAMMA = 0x9E3779B97F4A7C15


# ----------------------------------------------------------------------------------------
# random numbers
# ----------------------------------------------------------------------------------------
def test_splitmix64_published_sequence():
    """SplitMix64 (Steele, Lea & Flood 2014) seeded with 1234567: first five outputs of the
    published reference generator."""
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
            16408922859458223821]
    got = [oc.sm64((1234567 + k * GAMMA) % 2 ** 64) for k in range(5)]
    assert got == want


def test_draw_key_chain_is_a_function_of_every_key():
    base = oc.draw(3, 0, 5, 7, 9)
    assert base == oc.draw(3, 0, 5, 7, 9)
    for k in range(5):
        key = [3, 0, 5, 7, 9]
        key[k] += 1
        assert oc.draw(*key) != base


# ----------------------------------------------------------------------------------------
# trilinear interpolation and its derivatives (Supp. Sec. 1)
# ----------------------------------------------------------------------------------------
def test_trilinear_matches_supplement_printed_values():
    g = json.load(open(os.path.join(GOLDEN, "supp_trilinear_cell.json")))
    w, J = oc.trilinear_coeffs(g["f"])
    np.testing.assert_allclose(w, g["w"], atol=1e-15)
    np.testing.assert_allclose(J[:, 0], g["J1"], atol=1e-15)
    np.testing.assert_allclose(J[:, 1], g["J2"], atol=1e-15)
    np.testing.assert_allclose(J[:, 2], g["J3"], atol=1e-15)
    h = oc.trilinear_hessian(g["theta"], g["f"])
    np.testing.assert_allclose(h, [g["h12"], g["h13"], g["h23"]], atol=1e-14)


def test_trilinear_jacobian_and_hessian_match_finite_differences():
    rng = np.random.default_rng(0)
    for _ in range(20):
        f = rng.uniform(0.05, 0.95, 3)
        th = rng.normal(size=8)
        w, J = oc.trilinear_coeffs(f)
        assert abs(w.sum() - 1) < 1e-14 and np.all(np.abs(J.sum(0)) < 1e-14)
        h = 1e-6
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            wp, Jp = oc.trilinear_coeffs(f + e)
            wm, Jm = oc.trilinear_coeffs(f - e)
            np.testing.assert_allclose((wp - wm) / (2 * h), J[:, a], atol=1e-9)
            # column a of the x-Hessian of theta^T w: d/dx_a (J^T theta)
            col = ((Jp - Jm) / (2 * h)).T @ th
            H = oc.trilinear_hessian(th, f)
            full = np.array([[0, H[0], H[1]], [H[0], 0, H[2]], [H[1], H[2], 0]])
            np.testing.assert_allclose(col, full[:, a], atol=1e-8)


def test_affine_field_reproduced_exactly_with_constant_gradient():
    """Trilinear interpolation reproduces any affine field a.x + b exactly, with
    grad_x = a, at every level (Supp. Eq. trilinear_interp is exact on affine data)."""
    rng = np.random.default_rng(1)
    cfg = oc.make_config(CUBE)
    for level in range(4):
        for feat in (0, 3):
            a = rng.normal(size=3)
            b = rng.normal()
            th = zero_params(CUBE)
            set_level_field(CUBE, th, level, feat, lambda X: X @ a + b)
            passthrough_decoder(CUBE, th, 4 * level + feat)
            x = rng.uniform(-1.2, 1.2, (64, 3)).astype(np.float32)
            th64 = th.astype(np.float64)
            # the vertex values themselves are float32-rounded; compare with the rounded field
            sdf, grad = oc.query_sdf(cfg, th64, x)
            want = x.astype(np.float64) @ a + b
            np.testing.assert_allclose(sdf, want, atol=2e-6)
            np.testing.assert_allclose(grad, np.broadcast_to(a, grad.shape), atol=2e-5)


def test_vertex_values_at_vertices_and_clamping_outside():
    rng = np.random.default_rng(2)
    cfg = oc.make_config(CUBE)
    th = zero_params(CUBE)
    level = 3
    vals = rng.normal(size=CUBE.dims[level][::-1]).astype(np.float32)
    set_level_field(CUBE, th, level, 1, lambda X: vals)
    passthrough_decoder(CUBE, th, 4 * level + 1)
    v = np.float32(CUBE.voxels[level])
    o = np.float32(CUBE.extent_min[0])
    idx = rng.integers(0, 33, (50, 3))
    x = (o + idx.astype(np.float32) * v).astype(np.float32)
    sdf, _ = oc.query_sdf(cfg, th.astype(np.float64), x)
    # binary32 vertex positions sit within ~2e-6 cells of the vertex, hence the tolerance
    np.testing.assert_allclose(sdf, vals[idx[:, 2], idx[:, 1], idx[:, 0]], atol=2e-5)
    # outside the box: value of the clamped point, zero derivative along clamped axes
    xin = np.array([[0.3, -0.2, 0.1]], np.float32)
    xout = np.array([[5.0, -0.2, 0.1]], np.float32)
    xface = np.array([[1.28, -0.2, 0.1]], np.float32)
    s_out, g_out = oc.query_sdf(cfg, th.astype(np.float64), xout)
    s_face, _ = oc.query_sdf(cfg, th.astype(np.float64), xface)
    assert abs(s_out[0] - s_face[0]) < 1e-12 and g_out[0, 0] == 0.0
    _, g_in = oc.query_sdf(cfg, th.astype(np.float64), xin)
    assert g_in[0, 0] != 0.0


def test_voxel_index_cell_contains_point():
    rng = np.random.default_rng(3)
    cfg = oc.make_config(CUBE)
    x = rng.uniform(-1.5, 1.5, (4000, 3)).astype(np.float32)
    idx = oc.voxel_index(cfg, x)
    for level in range(4):
        nx, ny, nz = CUBE.dims[level]
        ix = idx[:, level] % nx
        iy = (idx[:, level] // nx) % ny
        iz = idx[:, level] // (nx * ny)
        v = float(np.float32(CUBE.voxels[level]))
        for a, ia, n in ((0, ix, nx), (1, iy, ny), (2, iz, nz)):
            assert ia.min() >= 0 and ia.max() <= n - 2
            u = np.clip((x[:, a].astype(np.float64) + 1.28) / v, 0, n - 1)
            assert np.all(u >= ia - 1e-5) and np.all(u <= ia + 1 + 1e-5)


# ----------------------------------------------------------------------------------------
# ray batch sampling (Sec. 3.4) and sample placement
# ----------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cube_inputs():
    fr = sg.make_frames(CUBE)
    return fr, oc.make_config(CUBE), oc.OcFramesHolder(fr)


def test_sampler_strata_order_band_and_classes(cube_inputs):
    fr, cfg, F = cube_inputs
    b = oc.sample_rays(cfg, F, 3, 7, 512)
    N, Ns, Ng = CUBE.n_samples, CUBE.n_strat, CUBE.n_guided
    near, far, g, tr = np.float32(CUBE.near), np.float32(CUBE.far), 0.1, np.float32(CUBE.trunc)
    assert b["t"].shape == (512, N)
    assert np.all(np.diff(b["t"], axis=1) >= 0)
    for i in range(512):
        t, D = b["t"][i].astype(np.float64), float(b["D"][i])
        if D > 0:
            strat = t[(t < D - g - 1e-6) | (t > D + g + 1e-6)]
            guided = t[np.abs(t - D) <= g + 1e-6]
            assert len(guided) >= Ng
            # every stratum of [near, far] holds exactly one stratified sample
            edges = near + np.arange(Ns + 1) * (far - near) / Ns
            counts = np.histogram(t, bins=edges)[0]
            inside_band = np.histogram(guided, bins=edges)[0]
            assert np.all(counts - inside_band <= 1)
            assert len(strat) <= Ns
        else:
            edges = near + np.arange(N + 1) * (far - near) / N
            counts = np.histogram(t, bins=edges)[0]
            assert np.all(counts == 1)
        bb = D - b["t"][i]
        want = np.where(D > 0, np.where(np.abs(bb) <= tr, 1, np.where(bb > tr, 2, 0)), 0)
        assert np.array_equal(b["cls"][i], want)
    assert b["counts"][0] == int((b["D"] > 0).sum())
    assert b["counts"][1] == int((b["cls"] == 1).sum()) and b["counts"][2] == int((b["cls"] == 2).sum())


def test_sampled_pixel_rays_hit_the_rendered_surface(cube_inputs):
    """o + D r of a sampled pixel lies on the scene surface: the oracle's ray generation
    (pixel centre, intrinsics, c2w, z-depth) agrees with the independently written renderer."""
    fr, cfg, F = cube_inputs
    b = oc.sample_rays(cfg, F, 3, 1, 1024)
    ok = b["D"] > 0
    x = b["o"][ok].astype(np.float64) + b["D"][ok, None].astype(np.float64) * b["r"][ok].astype(np.float64)
    d = sg.cube_scene().sdf(x)
    assert np.abs(d).max() < 2e-5
    # r has unit camera-z: R^T r = ((u+.5-cx)/fx, (v+.5-cy)/fy, 1)
    Rm = fr.c2w[0, :, :3].astype(np.float64)
    cam = b["r"].astype(np.float64) @ Rm
    np.testing.assert_allclose(cam[:, 2], 1.0, atol=1e-6)
    u = b["pix"] % CUBE.width
    np.testing.assert_allclose(cam[:, 0], (u + 0.5 - CUBE.cx) / CUBE.fx, atol=1e-6)


def test_pixels_drawn_uniformly_over_frames(cube_inputs):
    fr, cfg, F = cube_inputs
    b = oc.sample_rays(cfg, F, 9, 0, 20000)
    npx = CUBE.width * CUBE.height
    assert b["pix"].min() >= 0 and b["pix"].max() < npx
    hist = np.histogram(b["pix"], bins=10, range=(0, npx))[0]
    assert np.all(np.abs(hist - 2000) < 5 * math.sqrt(2000))


def test_smoothness_points_near_observed_surface(cube_inputs):
    fr, cfg, F = cube_inputs
    s = oc.sample_smooth(cfg, F, 3, 0, 2048)
    assert s["n_valid"][0] == s["valid"].sum() > 1900
    v = s["valid"] == 1
    d = sg.cube_scene().sdf(s["xs"][v])
    assert np.abs(d).max() <= math.sqrt(3) * CUBE.trunc + 1e-4
    np.testing.assert_allclose(np.linalg.norm(s["eps"][v], axis=1), CUBE.delta_s, rtol=1e-6)


# ----------------------------------------------------------------------------------------
# volume rendering (Sec. 3.2)
# ----------------------------------------------------------------------------------------
def test_weights_telescope_and_stay_in_range():
    rng = np.random.default_rng(4)
    for _ in range(50):
        N = int(rng.integers(2, 97))
        phi = rng.normal(0, 0.3, N)
        d = np.sort(rng.uniform(0.1, 4, N)).astype(np.float32)
        alpha, T, w, dh, ws = oc.composite(phi, float(rng.uniform(5, 200)), d)
        assert np.all(alpha >= 0) and np.all(alpha <= 1) and alpha[-1] == 0
        assert np.all(w >= 0)
        assert abs(ws - (1 - np.prod(1 - alpha))) < 1e-12
        assert ws <= 1 + 1e-12
        np.testing.assert_allclose(T[1:], np.cumprod(1 - alpha)[:-1], rtol=1e-12)


def test_single_zero_crossing_concentrates_weight_at_the_surface():
    """For phi decreasing through 0 at depth d_s, the NeuS weights concentrate on the interval
    holding the crossing as s grows: d_hat -> the sample starting that interval (weights are
    attributed to sample depths, so the limit lies within one spacing of d_s)."""
    d = np.linspace(0.5, 2.5, 801).astype(np.float32)
    spacing = 2.0 / 800
    ds = 1.37 + 0.3 * spacing
    phi = ds - d.astype(np.float64)
    k = int(np.searchsorted(d, ds)) - 1  # d[k] <= ds < d[k+1]
    for s in (50.0, 500.0, 5000.0, 50000.0):
        _, _, w, dh, ws = oc.composite(phi, s, d)
        assert ws > 0.99
        assert abs(dh / ws - ds) < spacing
    assert w[k] / ws > 0.99 and abs(dh / ws - float(d[k])) < 1e-4


def _sphere_setup(kappa):
    th = zero_params(CUBE)
    c, rad = np.array([-0.4, 0.0, 0.0]), 0.5
    set_level_field(CUBE, th, 3, 0, lambda X: np.linalg.norm(X - c, axis=-1) - rad)
    passthrough_decoder(CUBE, th, 12, kappa=kappa)
    return th, c, rad


def test_analytic_sphere_rendered_depth():
    """An analytic sphere SDF baked into the finest grid renders the ray-sphere intersection
    depth within 1 cm (8 cm voxels, r = 0.5 m, s = 400 1/m)."""
    th, c, rad = _sphere_setup(math.log(400.0))
    cfg = oc.make_config(CUBE)
    rng = np.random.default_rng(5)
    R, N = 16, 512
    o = np.tile([-1.2, 0.0, 0.0], (R, 1)) + rng.uniform(-0.05, 0.05, (R, 3)) * [0, 1, 1]
    r = np.tile([1.0, 0.0, 0.0], (R, 1)) + rng.uniform(-0.1, 0.1, (R, 3)) * [0, 1, 1]
    oo, rr = o.astype(np.float64), r.astype(np.float32).astype(np.float64)
    oo = o.astype(np.float32).astype(np.float64)
    A = (rr * rr).sum(1)
    B = ((oo - c) * rr).sum(1)
    C = ((oo - c) ** 2).sum(1) - rad ** 2
    t_hit = (-B - np.sqrt(B * B - A * C)) / A
    t = np.tile(np.linspace(0.1, 1.0, N), (R, 1))
    bt = hand_batch(o, r, t, t_hit)
    out = oc.step(cfg, th, bt, None, want_grad=False)
    assert np.all(out["wsum"] > 0.98)
    assert np.abs(out["d_hat"] / out["wsum"] - t_hit).max() < 0.01


# ----------------------------------------------------------------------------------------
# losses (Sec. 3.2-3.4)
# ----------------------------------------------------------------------------------------
def _plane_batch(shift, R=8, N=40):
    """Rays along +x hitting the plane x = 0.5; phi = (0.5 - x) + shift baked in the grid."""
    rng = np.random.default_rng(6)
    th = zero_params(CUBE)
    set_level_field(CUBE, th, 3, 2, lambda X: (0.5 - X[..., 0]) + shift)
    passthrough_decoder(CUBE, th, 14)
    o = np.c_[np.full(R, -1.0), rng.uniform(-0.5, 0.5, (R, 2))]
    r = np.tile([1.0, 0.0, 0.0], (R, 1))
    t = np.sort(rng.uniform(0.3, 1.8, (R, N)), axis=1)
    return th, hand_batch(o, r, t, np.full(R, 1.5))


@pytest.mark.parametrize("shift", [0.0, 0.03, -0.03])
def test_plane_sdf_and_free_space_losses(shift):
    """phi = b + shift at every sample (plane SDF is affine, so trilinear is exact):
    L_sdf = |shift| over S_tr; L_fs = max(0, shift) over S_fs (phi > 0 there)."""
    th, bt = _plane_batch(shift)
    assert (bt["cls"] == 1).sum() > 10 and (bt["cls"] == 2).sum() > 10
    out = oc.step(oc.make_config(CUBE), th, bt, None, want_grad=False)
    assert abs(out["loss"][2] - abs(shift)) < 2e-6
    assert abs(out["loss"][3] - max(0.0, shift)) < 2e-6


def test_constant_negative_sdf_free_space_penalty():
    """phi = -0.2 everywhere: every free-space sample pays exp(5 * 0.2) - 1 = e - 1."""
    th = zero_params(CUBE)
    set_level_field(CUBE, th, 0, 0, lambda X: np.full(X.shape[:-1], -0.2))
    passthrough_decoder(CUBE, th, 0)
    _, bt = _plane_batch(0.0)
    out = oc.step(oc.make_config(CUBE), th, bt, None, want_grad=False)
    assert abs(out["loss"][3] - (math.e - 1)) < 1e-6


def test_transparent_rays_render_nothing():
    """phi increasing along every ray gives alpha = 0, so c_hat = d_hat = 0:
    L_rgb = mean ||I||^2 and L_d = mean D over rays with D > 0."""
    th = zero_params(CUBE)
    set_level_field(CUBE, th, 3, 0, lambda X: X[..., 0])
    passthrough_decoder(CUBE, th, 12)
    rng = np.random.default_rng(7)
    R = 12
    o = np.c_[np.full(R, -1.0), rng.uniform(-0.5, 0.5, (R, 2))]
    r = np.tile([1.0, 0.0, 0.0], (R, 1))
    t = np.sort(rng.uniform(0.1, 2.0, (R, 20)), axis=1)
    D = np.where(np.arange(R) % 3 == 0, 0.0, rng.uniform(0.5, 2, R))
    rgb = rng.uniform(0, 1, (R, 3))
    bt = hand_batch(o, r, t, D, rgb)
    out = oc.step(oc.make_config(CUBE), th, bt, None, want_grad=False)
    rgb32 = rgb.astype(np.float32).astype(np.float64)
    D32 = D.astype(np.float32).astype(np.float64)
    assert abs(out["loss"][0] - (rgb32 ** 2).sum(1).mean()) < 1e-12
    assert abs(out["loss"][1] - D32[D32 > 0].mean()) < 1e-12


# ----------------------------------------------------------------------------------------
# smoothness (Sec. 3.3)
# ----------------------------------------------------------------------------------------
def _smooth_points(P=64, seed=8):
    rng = np.random.default_rng(seed)
    xs = rng.uniform(-0.9, 0.9, (P, 3)).astype(np.float32)
    v = rng.normal(size=(P, 3))
    eps = (0.004 * v / np.linalg.norm(v, axis=1, keepdims=True)).astype(np.float32)
    return dict(xs=xs, eps=eps, valid=np.ones(P, np.uint8))


def test_smoothness_zero_on_affine_field():
    th = zero_params(CUBE)
    set_level_field(CUBE, th, 2, 1, lambda X: X @ np.array([0.3, -0.7, 0.2]) + 0.1)
    passthrough_decoder(CUBE, th, 9)
    _, bt = _plane_batch(0.0, R=1, N=4)
    out = oc.step(oc.make_config(CUBE), th, bt, _smooth_points(), want_grad=False)
    assert out["loss"][4] < 1e-12  # binary32 vertex values: the field is affine up to rounding


def test_smoothness_bilinear_closed_form():
    """phi = x*y lies in the trilinear span, so grad phi = (y, x, 0) exactly and
    ||grad phi(x) - grad phi(x + eps)||^2 = eps_x^2 + eps_y^2 (points well inside cells' span)."""
    th = zero_params(CUBE)
    set_level_field(CUBE, th, 3, 0, lambda X: X[..., 0] * X[..., 1])
    passthrough_decoder(CUBE, th, 12)
    sm = _smooth_points()
    _, bt = _plane_batch(0.0, R=1, N=4)
    out = oc.step(oc.make_config(CUBE), th, bt, sm, want_grad=False)
    e = sm["eps"].astype(np.float64)
    want = (e[:, 0] ** 2 + e[:, 1] ** 2).mean()
    assert abs(out["loss"][4] - want) < 1e-5 * want  # binary32 vertex values


# ----------------------------------------------------------------------------------------
# gradients: central finite differences of the oracle's forward pass
# ----------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def tiny_problem():
    fr = sg.make_frames(TINY)
    cfg = oc.make_config(TINY)
    F = oc.OcFramesHolder(fr)
    bt = oc.sample_rays(cfg, F, 3, 0, TINY.rays)
    sm = oc.sample_smooth(cfg, F, 3, 0, TINY.n_smooth)
    th = sg.parity_params(TINY, seed=12, grid_std=0.2).astype(np.float64)
    th[-1] = math.log(8.0)
    return cfg, bt, sm, th


def _fd_check(cfg, bt, sm, th, dloss, h, tol, idx, same_piece_only=False):
    """Central differences of the oracle's forward loss against its reverse-mode gradient.

    same_piece_only: compare only entries whose +-h evaluations take every branch decision
    (ReLU masks, alpha > 0, signs, free-space max) as the unperturbed one does, i.e. lie on
    the same smooth piece of the loss; at least 90% of the entries must qualify."""
    out = oc.step(cfg, th, bt, sm, dloss=dloss, want_margins=True)
    g = out["grad"]
    sig0 = out["margins"][7]

    def total(x):
        r = oc.step(cfg, x, bt, sm, want_grad=False, want_margins=True)
        lo = r["loss"]
        return (lo[5] if dloss is None else float(np.dot(lo, dloss))), r["margins"][7]

    fd = np.zeros(len(idx))
    keep = np.ones(len(idx), bool)
    for j, i in enumerate(idx):
        x = th.copy()
        x[i] += h
        fp, sp = total(x)
        x[i] -= 2 * h
        fm, sm_ = total(x)
        fd[j] = (fp - fm) / (2 * h)
        keep[j] = (sp == sig0 and sm_ == sig0) or not same_piece_only
    assert keep.mean() >= 0.9
    scale = np.abs(g[idx]).max()
    err = np.abs(fd - g[idx])[keep].max() / scale
    assert err < tol, (err, out["margins"])
    return out


def test_gradients_match_central_differences(tiny_problem):
    cfg, bt, sm, th = tiny_problem
    _, n_grid, n_tot = TINY.layout()
    out = oc.step(cfg, th, bt, sm, want_margins=True)
    assert out["margins"][0] > 1e-2  # every hidden unit far from its ReLU kink
    touched = np.nonzero(out["grad"][:n_grid])[0]
    assert len(touched) > 100
    idx = np.r_[touched, np.arange(n_grid, n_tot)]
    _fd_check(cfg, bt, sm, th, None, 1e-6, 1e-6, idx)


def test_gradients_match_central_differences_per_term_seeds(tiny_problem):
    """Upstream seeds per loss term (autograd use): gradient of sum_k dloss_k * L_k."""
    cfg, bt, sm, th = tiny_problem
    _, n_grid, n_tot = TINY.layout()
    dloss = np.array([0.3, -1.1, 0.7, 2.0, 5.0, 0.25])
    out = oc.step(cfg, th, bt, sm, dloss=dloss)
    touched = np.nonzero(out["grad"][:n_grid])[0]
    idx = np.r_[touched[::3], np.arange(n_grid, n_tot, 2)]
    _fd_check(cfg, bt, sm, th, dloss, 1e-6, 1e-6, idx)


def test_smoothness_second_order_gradient_alone(tiny_problem):
    """d/dtheta and d/domega of the smoothness term alone (the second-order path)."""
    cfg, bt, sm, th = tiny_problem
    _, n_grid, n_tot = TINY.layout()
    dloss = np.array([0, 0, 0, 0, 1.0, 0])
    out = oc.step(cfg, th, bt, sm, dloss=dloss)
    g = out["grad"]
    assert np.abs(g[:n_grid]).max() > 0 and np.abs(g[n_grid:n_grid + 512]).max() > 0
    touched = np.nonzero(g[:n_grid])[0]
    idx = np.r_[touched, np.arange(n_grid, n_tot)]
    _fd_check(cfg, bt, sm, th, dloss, 1e-6, 1e-6, idx)


def test_gradients_match_central_differences_h1e3(tiny_problem):
    """The h = 1e-3 central-difference check on the 16^3 grid."""
    cfg, bt, sm, th = tiny_problem
    _, n_grid, n_tot = TINY.layout()
    out = oc.step(cfg, th, bt, sm)
    touched = np.nonzero(out["grad"][:n_grid])[0]
    idx = np.r_[touched[::4], np.arange(n_grid, n_tot, 3)]
    _fd_check(cfg, bt, sm, th, None, 1e-3, 1e-4, idx, same_piece_only=True)


# ----------------------------------------------------------------------------------------
# SDF query backward (phi and grad_x phi as differentiable outputs, Supp. Sec. 1)
# ----------------------------------------------------------------------------------------
def _query_objective(cfg, th, x, dsdf, dgrad):
    phi, g = oc.query_sdf(cfg, th, x)
    return float(np.dot(dsdf, phi) + np.sum(dgrad * g))


@pytest.mark.parametrize("h,tol", [(1e-6, 1e-6), (1e-3, 1e-4)])
def test_query_sdf_backward_matches_central_differences(tiny_problem, h, tol):
    cfg, _, _, th = tiny_problem
    _, n_grid, n_tot = TINY.layout()
    rng = np.random.default_rng(4)
    x = rng.uniform(-1.2, 1.2, (40, 3)).astype(np.float32)
    dsdf, dgrad = rng.normal(size=40), rng.normal(size=(40, 3))
    g = oc.query_sdf_backward(cfg, th, x, dsdf, dgrad)
    touched = np.nonzero(g[:n_grid])[0]
    assert len(touched) > 100
    idx = np.r_[touched[::2], np.arange(n_grid, n_tot)]
    fd = np.empty(len(idx))
    for j, i in enumerate(idx):
        xp, xm = th.copy(), th.copy()
        xp[i] += h
        xm[i] -= h
        fd[j] = (_query_objective(cfg, xp, x, dsdf, dgrad) - _query_objective(cfg, xm, x, dsdf, dgrad)) / (2 * h)
    err = np.abs(fd - g[idx]) / np.abs(g[idx]).max()
    # at h = 1e-3 a ReLU unit of some point may switch inside [theta - h, theta + h]
    assert (np.median(err) < tol and np.mean(err < tol) > 0.98) if h > 1e-5 else err.max() < tol, err.max()


def test_query_sdf_backward_terms_separate_and_add(tiny_problem):
    """The two upstream seeds act linearly and independently; kappa and the colour decoder
    get no gradient from an SDF query."""
    cfg, _, _, th = tiny_problem
    _, n_grid, n_tot = TINY.layout()
    rng = np.random.default_rng(5)
    x = rng.uniform(-1.0, 1.0, (16, 3)).astype(np.float32)
    ds, dg = rng.normal(size=16), rng.normal(size=(16, 3))
    g1 = oc.query_sdf_backward(cfg, th, x, ds, None)
    g2 = oc.query_sdf_backward(cfg, th, x, None, dg)
    g12 = oc.query_sdf_backward(cfg, th, x, 2 * ds, -dg)
    np.testing.assert_allclose(g12, 2 * g1 - g2, rtol=1e-12, atol=1e-14)
    offs = dict(zip([n for n, _ in sg.MLP_SHAPES], np.cumsum([0] + [int(np.prod(s)) for _, s in sg.MLP_SHAPES])))
    colour = slice(n_grid + offs["W3"], n_tot)
    assert not np.any(g1[colour]) and not np.any(g2[colour])
    # d phi / d b2 = (1, 0, ..., 0): the SDF seeds sum into b2[0]
    assert abs(g1[n_grid + offs["b2"]] - ds.sum()) < 1e-12


def test_query_sdf_backward_affine_field_closed_form():
    """phi = z_k (pass-through decoder) on an affine field: grad_x phi = c is constant and
    a . grad_x phi is linear in the level's vertex values, with d/d theta_v = a . d w_v / d x
    summed over the points; its total over the vertices is 0 (the weights' gradients
    sum to zero in every cell)."""
    th = zero_params(CUBE)
    set_level_field(CUBE, th, 2, 1, lambda X: X @ np.array([0.3, -0.7, 0.2]) + 0.1)
    passthrough_decoder(CUBE, th, 9)
    cfg = oc.make_config(CUBE)
    rng = np.random.default_rng(6)
    x = rng.uniform(-0.9, 0.9, (12, 3)).astype(np.float32)
    a = rng.normal(size=(12, 3))
    g = oc.query_sdf_backward(cfg, th, x, None, a)
    offs, n_grid, _ = CUBE.layout()
    n2 = int(np.prod(CUBE.dims[2])) * 4
    lvl = g[offs[2]:offs[2] + n2].reshape(-1, 4)
    assert np.abs(lvl[:, 1]).max() > 0
    assert abs(lvl[:, 1].sum()) < 1e-9 * np.abs(lvl[:, 1]).max() * len(x)
    # and the SDF seed alone puts the trilinear weights (summing to 1 per point) on feature 1
    g1 = oc.query_sdf_backward(cfg, th, x, np.ones(12), None)
    lv1 = g1[offs[2]:offs[2] + n2].reshape(-1, 4)
    assert abs(lv1[:, 1].sum() - 12.0) < 1e-9


# ----------------------------------------------------------------------------------------
# Adam (Kingma & Ba 2015) with the paper's per-group learning rates
# ----------------------------------------------------------------------------------------
def test_adam_first_two_steps_closed_form():
    rng = np.random.default_rng(9)
    n, n_grid = 1000, 600
    p0 = rng.normal(size=n)
    g1 = rng.normal(size=n)
    g2 = rng.normal(size=n)
    p, m, v = p0.copy(), np.zeros(n), np.zeros(n)
    g = g1.copy()
    oc.adam(p, g, m, v, n_grid, 1, 1e-2, 1e-3)
    lr = np.where(np.arange(n) < n_grid, 1e-2, 1e-3)
    # bias-corrected first step: m_hat = g, v_hat = g^2
    np.testing.assert_allclose(p, p0 - lr * g1 / (np.abs(g1) + 1e-8), rtol=0, atol=1e-15)
    assert np.all(g == 0)
    g = g2.copy()
    oc.adam(p, g, m, v, n_grid, 2, 1e-2, 1e-3)
    m2 = 0.9 * 0.1 * g1 + 0.1 * g2
    v2 = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    step2 = lr * (m2 / (1 - 0.81)) / (np.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    np.testing.assert_allclose(p, p0 - lr * g1 / (np.abs(g1) + 1e-8) - step2, atol=1e-14)


def test_hyperparameter_golden_matches_workload_readings():
    """The workloads keep the paper's loss weights, learning rates and free-space exponent."""
    g = json.load(open(os.path.join(GOLDEN, "hyperparameters.json")))
    w = sg.WORKLOADS["room-8192x96"]
    lam = g["lambda"]
    assert w.lambdas == (lam["rgb"], lam["depth"], lam["sdf"], lam["fs"], lam["smooth"])
    assert (w.lr_grid, w.lr_mlp) == (g["lr_grids"], g["lr_decoders"])
    assert w.kappa_fs == g["fs_exponent"]
    assert g["delta_s_range_m"][0] <= w.delta_s <= g["delta_s_range_m"][1]
    assert w.voxels[:3] == tuple(g["voxel_sizes_m"][:3])
