"""Input builders shared by the tests (no method arithmetic: grids filled with known fields,
decoders set to pass one feature through, hand-made ray batches)."""
from __future__ import annotations

import math

import numpy as np

import scenegen as sg
from scenegen import set_level_field, vertex_positions  # noqa: F401 (re-exported for the tests)

CUBE = sg.WORKLOADS["cube-1024x64"]
# tiny 4-level grid on the cube scene, finest level 16^3 vertices (gradient checks)
TINY = CUBE.with_(name="tiny-16", voxels=(2.56 / 1, 2.56 / 3, 2.56 / 7, 2.56 / 15), rays=6, n_strat=12, n_guided=4,
                  n_smooth=8)


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


# the scene's exact SDF baked into the finest level, decoders whose hidden units switch from
# sample to sample (input builders shared with the smoke check)
sdf_parity_params = sg.sdf_switching_params
paper_parity_params = sg.paper_switching_params
