"""Input builders shared by the tests (no method arithmetic: grids filled with known fields,
decoders set to pass one feature through, hand-made ray batches)."""
from __future__ import annotations

import math

import numpy as np

import scenegen as sg

CUBE = sg.WORKLOADS["cube-1024x64"]
# tiny 4-level grid on the cube scene, finest level 16^3 vertices (gradient checks)
TINY = CUBE.with_(name="tiny-16", voxels=(2.56 / 1, 2.56 / 3, 2.56 / 7, 2.56 / 15), rays=6, n_strat=12, n_guided=4,
                  n_smooth=8)


def vertex_positions(w, level):
    """Vertex coordinates [nz,ny,nx,3] (metres) of one grid level, x fastest."""
    nx, ny, nz = w.dims[level]
    v = np.float64(np.float32(w.voxels[level]))
    o = np.asarray(w.extent_min, np.float32).astype(np.float64)
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([o[0] + xx * v, o[1] + yy * v, o[2] + zz * v], -1)


def set_level_field(w, theta, level, feat, fn):
    """theta[level][..., feat] = fn(vertex positions)."""
    offs, _, _ = w.layout()
    nx, ny, nz = w.dims[level]
    view = theta[offs[level]:offs[level] + nx * ny * nz * sg.FEAT].reshape(nz, ny, nx, sg.FEAT)
    view[..., feat] = fn(vertex_positions(w, level))
    return theta


def passthrough_decoder(w, theta, zindex, colour_logit=0.0, kappa=math.log(20.0)):
    """Decoder weights with phi = z[zindex] exactly (relu(v) - relu(-v) = v), constant colour."""
    _, n_grid, _ = w.layout()
    theta[n_grid:] = 0.0
    m = sg.mlp_views(theta, n_grid)
    m["W1"][0, zindex] = 1.0
    m["W1"][1, zindex] = -1.0
    m["W2"][0, 0] = 1.0
    m["W2"][0, 1] = -1.0
    m["b4"][:] = colour_logit
    m["kappa"][0] = kappa
    return theta


def zero_params(w):
    return np.zeros(w.layout()[2], np.float32)


def hand_batch(o, r, t, D, rgb=None, trunc=0.1):
    """A ray batch built directly (R rays, N samples each) with classes from the bound b = D - t."""
    o = np.asarray(o, np.float32).reshape(-1, 3)
    r = np.asarray(r, np.float32).reshape(-1, 3)
    t = np.asarray(t, np.float32).reshape(len(o), -1)
    D = np.asarray(D, np.float32).reshape(-1)
    R, N = t.shape
    rgb = np.zeros((R, 3), np.float32) if rgb is None else np.asarray(rgb, np.float32).reshape(R, 3)
    b = D[:, None] - t
    cls = np.where(D[:, None] > 0, np.where(np.abs(b) <= np.float32(trunc), 1, np.where(b > np.float32(trunc), 2, 0)),
                   0).astype(np.uint8)
    return dict(o=o, r=r, t=t, D=D, rgb=rgb, cls=cls)


def sdf_parity_params(w, scene, seed=21, grid_std=0.05, bias=0.25, pass_offset=3.0, mix=0.1):
    """Parameters for element-wise GPU-vs-oracle parity: the scene's exact SDF baked into
    feature 0 of the finest level, random features elsewhere, and decoders whose every
    hidden unit stays far from its ReLU kink.

    Hidden units 0 and 1 carry phi = z[12] exactly through two always-on units
    (0.5 relu(v + B) - 0.5 relu(B - v) = v for |v| < B); the other units get biases of
    alternating sign and magnitude `bias`, and add a small nonlinear term (weight `mix`).
    A realistic SDF makes adjacent samples' opacities differ, so the alpha > 0 decisions are
    clear-cut in binary32 as well as in FP64.
    """
    import math
    rng = np.random.default_rng(seed)
    offs, n_grid, n_tot = w.layout()
    theta = np.zeros(n_tot, np.float32)
    theta[:n_grid] = rng.normal(0.0, grid_std, n_grid).astype(np.float32)
    nx, ny, nz = w.dims[3]
    X = vertex_positions(w, 3)
    sdf = scene.sdf(X.reshape(-1, 3)).reshape(nz, ny, nx)
    set_level_field(w, theta, 3, 0, lambda _: sdf)
    m = sg.mlp_views(theta, n_grid)
    m["W1"][:] = rng.uniform(-0.25, 0.25, m["W1"].shape)
    m["W1"][:, 12] = 0.0  # the SDF feature reaches phi only through the pass-through units
    m["b1"][:] = np.where(np.arange(32) % 2 == 0, bias, -bias)
    m["W1"][0, :] = 0.0
    m["W1"][1, :] = 0.0
    m["W1"][0, 12] = 1.0
    m["W1"][1, 12] = -1.0
    m["b1"][0] = m["b1"][1] = pass_offset
    m["W2"][:] = rng.uniform(-0.18, 0.18, m["W2"].shape)
    m["W2"][0, :] = rng.uniform(-mix, mix, 32)
    m["W2"][1:, :2] = 0.0  # the colour features do not see the pass-through units
    m["W2"][0, 0], m["W2"][0, 1] = 0.5, -0.5
    m["b2"][:] = rng.uniform(-0.1, 0.1, 16)
    m["b2"][0] = 0.0
    m["W3"][:] = rng.uniform(-0.2, 0.2, m["W3"].shape)
    m["b3"][:] = np.where(np.arange(32) % 2 == 0, bias, -bias)
    m["W4"][:] = rng.uniform(-0.5, 0.5, m["W4"].shape)
    m["b4"][:] = rng.uniform(-0.2, 0.2, 3)
    m["kappa"][0] = math.log(20.0)
    return theta
