"""Pin of the oracle's colour path for the workload's decoders (the colour decoder
c = sigmoid(W4 relu(W3 h + b3) + b4) fed by h = outputs 1..15 of the geometry decoder),
rendered through the NeuS weights of Sec. 3.2 Eq. volume_rendering.

Closed form: the geometry decoder carries phi = z[14] (a plane SDF) and routes three affine
grid fields A_c into three of its colour features through pairs of hidden units
(relu(v) - relu(-v) = v); the colour decoder passes each of those features into one channel
with its own gain g_c and bias b4_c through another pair.  Trilinear interpolation
reproduces affine fields exactly (pinned elsewhere), so every sample's colour is
sigmoid(g_c A_c(x_k) + b4_c) and c_hat_c = sum_k w_k sigmoid(g_c A_c(x_k) + b4_c) with the
oracle's own compositing weights w_k (pinned by the compositing tests) and x_k = o + t_k r
in binary32.

The pin is then shown to catch mistakes planted in a copy of the oracle: the colour decoder
reading outputs 0..14 instead of 1..15, a dropped sigmoid, and W4 read transposed.
"""
import math

import numpy as np
import pytest

import oracle as oc
import scenegen as sg
from helpers import CUBE, hand_batch, passthrough_decoder, set_level_field

# (z index of the field, colour feature j it is routed to, gain g_c, bias b4_c, field A_c)
CHANNELS = [
    (9, 4, 1.0, 0.1, (np.array([0.7, -1.3, 0.4]), 0.2)),     # level 2, feature 1 -> h[4] -> red
    (4, 9, -1.5, -0.2, (np.array([-0.5, 0.3, 0.8]), -0.1)),  # level 1, feature 0 -> h[9] -> green
    (3, 14, 0.8, 0.3, (np.array([0.2, 0.9, -0.6]), 0.3)),    # level 0, feature 3 -> h[14] -> blue
]


def _colour_params():
    th = np.zeros(CUBE.layout()[2], np.float32)
    set_level_field(CUBE, th, 3, 2, lambda X: 0.5 - X[..., 0])  # plane SDF in z[14]
    for zi, _, _, _, (a, a0) in CHANNELS:
        set_level_field(CUBE, th, zi // 4, zi % 4, lambda X, a=a, a0=a0: X @ a + a0)
    passthrough_decoder(CUBE, th, zindex=14, kappa=math.log(20.0))
    m = sg.mlp_views(th, CUBE.layout()[1])
    for c, (zi, j, g, b, _) in enumerate(CHANNELS):
        u = 2 + 2 * c  # geometry hidden units u, u+1 carry z[zi]
        m["W1"][u, zi], m["W1"][u + 1, zi] = 1.0, -1.0
        m["W2"][1 + j, u], m["W2"][1 + j, u + 1] = 1.0, -1.0  # output 1 + j = h[j] = A_c
        m["W3"][2 * c, j], m["W3"][2 * c + 1, j] = 1.0, -1.0  # colour hidden units 2c, 2c+1 carry h[j]
        m["W4"][c, 2 * c], m["W4"][c, 2 * c + 1] = g, -g
        m["b4"][c] = b
    return th


def _rays(R=6, N=48, seed=9, spread=0.3):
    rng = np.random.default_rng(seed)
    o = np.c_[np.full(R, -1.0), rng.uniform(-0.4, 0.4, (R, 2))]
    r = np.c_[np.ones(R), rng.uniform(-spread, spread, (R, 2))]
    t = np.sort(rng.uniform(0.3, 2.2, (R, N)), axis=1)
    return hand_batch(o, r, t, np.full(R, 1.5))


def _colour_pin():
    """Raises AssertionError unless the rendered colour equals the closed form."""
    th = _colour_params()
    bt = _rays()
    out = oc.step(oc.make_config(CUBE), th, bt, None, want_grad=False, want_weights=True)
    x = (bt["o"][:, None, :] + (bt["t"][..., None] * bt["r"][:, None, :]).astype(np.float32)).astype(np.float64)
    assert out["wsum"].min() > 0.5  # the plane at x = 0.5 is crossed on every ray
    for c, (_, _, g, b, (a, a0)) in enumerate(CHANNELS):
        want = (out["w"] / (1.0 + np.exp(-(g * (x @ a + a0) + b)))).sum(axis=1)
        np.testing.assert_allclose(out["rgb_hat"][:, c], want, rtol=0, atol=2e-6)


def test_colour_decoder_closed_form():
    _colour_pin()


def test_colour_channels_differ():
    """The three channels carry different fields, gains and biases, so a channel mix-up or a
    transposed output layer cannot give the closed form by accident."""
    th = _colour_params()
    out = oc.step(oc.make_config(CUBE), th, _rays(), None, want_grad=False)
    c = out["rgb_hat"]
    assert np.abs(c[:, 0] - c[:, 1]).min() > 1e-2 and np.abs(c[:, 1] - c[:, 2]).min() > 1e-2


PLANTED = {
    # the colour decoder fed outputs 0..14 (phi and h_1..h_14) instead of h = outputs 1..15
    "slice": [("s += m->W3[j * OC_HF + k] * A->out[1 + k];", "s += m->W3[j * OC_HF + k] * A->out[k];")],
    # the output layer without its sigmoid
    "no_sigmoid": [("A->c[j] = sigm(s);", "A->c[j] = s;")],
    # W4 [3][32] read as if it were stored [32][3]
    "w4_transposed": [("s += m->W4[j * OC_H2 + k] * A->a2[k];", "s += m->W4[k * OC_RGB + j] * A->a2[k];")],
}


@pytest.mark.parametrize("mistake", sorted(PLANTED))
def test_colour_pin_catches_planted_mistakes(mistake):
    so = oc.build_variant(PLANTED[mistake], mistake)
    with oc.using_variant(so):
        with pytest.raises(AssertionError):
            _colour_pin()
    _colour_pin()  # the real oracle again
