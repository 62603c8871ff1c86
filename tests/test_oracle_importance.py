"""Pins of the oracle's hierarchical importance sampler (Sec. 3.2: N_c = 96 coarse samples
and 3 steps of 12, as in NeuS) against invariants and closed forms: strata, the interval
strata of a flat distribution, concentration at an analytic surface, the rays of the plain
sampler and the SDF query."""
import math

import numpy as np
import pytest

import oracle as oc
import scenegen as sg
from helpers import CUBE, hand_batch, passthrough_decoder, set_level_field, zero_params

NC, STEPS, M = 96, 3, 12


@pytest.fixture(scope="module")
def cube():
    return oc.make_config(CUBE), oc.OcFramesHolder(sg.make_frames(CUBE))


def _fine(coarse, final):
    """The samples that the importance steps added (final minus the coarse multiset)."""
    out = []
    for c, f in zip(coarse, final):
        rest = list(f)
        for v in c:
            rest.remove(v)
        out.append(np.array(rest, np.float32))
    return out


def test_same_rays_as_the_plain_sampler_sorted_and_classified(cube):
    cfg, F = cube
    th = sg.parity_params(CUBE, seed=4).astype(np.float64)
    b = oc.sample_importance(cfg, F, th, 3, 7, 80, NC, STEPS, M)
    a = oc.sample_rays(cfg, F, 3, 7, 80)
    for k in ("pix", "o", "r", "rgb", "D"):
        assert np.array_equal(a[k], b[k]), k
    assert b["t"].shape == (80, NC + STEPS * M)
    assert np.all(np.diff(b["t"], axis=1) >= 0)
    ref = hand_batch(b["o"], b["r"], b["t"], b["D"], trunc=CUBE.trunc)["cls"]
    assert np.array_equal(ref, b["cls"])
    assert b["counts"][0] == (b["D"] > 0).sum()
    assert b["counts"][1] == (b["cls"] == 1).sum() and b["counts"][2] == (b["cls"] == 2).sum()
    # phi at the final samples is the SDF query there
    x = (b["o"][:, None, :] + (b["t"][..., None] * b["r"][:, None, :]).astype(np.float32)).astype(np.float32)
    phi, _ = oc.query_sdf(cfg, th, x.reshape(-1, 3), want_grad=False)
    np.testing.assert_allclose(b["phi"].ravel(), phi, rtol=0, atol=0)
    # the coarse depths are kept: the run without importance steps is a sub-multiset
    c = oc.sample_importance(cfg, F, th, 3, 7, 80, NC, 0, M)
    fine = _fine(c["t"], b["t"])
    assert all(len(f) == STEPS * M for f in fine)


def test_coarse_samples_one_per_stratum(cube):
    cfg, F = cube
    th = sg.parity_params(CUBE, seed=4).astype(np.float64)
    c = oc.sample_importance(cfg, F, th, 11, 0, 64, NC, 0, M)
    d = (np.float64(np.float32(CUBE.far)) - np.float64(np.float32(CUBE.near))) / NC
    lo = np.float64(np.float32(CUBE.near)) + np.arange(NC) * d
    t = c["t"].astype(np.float64)
    assert np.all(t >= lo - 1e-6) and np.all(t <= lo + d + 1e-6)
    # the position inside each stratum is uniform (jittered, independently per ray and stratum)
    frac = ((t - lo) / d).ravel()
    hist = np.histogram(frac, bins=10, range=(0, 1))[0] / frac.size
    assert np.all(np.abs(hist - 0.1) < 0.02), hist
    assert len(np.unique(c["t"][:, 0])) > 60


def test_flat_distribution_draws_one_per_interval_stratum(cube):
    """phi constant (> 0) gives alpha = 0 everywhere, so each of the n - 1 intervals holds
    mass 1/(n - 1): draw j (u in [j/M, (j+1)/M)) lands in interval floor(u (n - 1)), i.e.
    between coarse samples floor(j (n-1)/M) and ceil((j+1)(n-1)/M)."""
    cfg, F = cube
    th = zero_params(CUBE).astype(np.float64)
    set_level_field(CUBE, th, 0, 0, lambda X: np.full(X.shape[:-1], 0.3))
    passthrough_decoder(CUBE, th, 0)
    c = oc.sample_importance(cfg, F, th, 5, 2, 40, NC, 0, M)
    b = oc.sample_importance(cfg, F, th, 5, 2, 40, NC, 1, M)
    for tc, f in zip(c["t"], _fine(c["t"], b["t"])):
        f = np.sort(f)
        for j in range(M):
            k0, k1 = math.floor(j * (NC - 1) / M), math.ceil((j + 1) * (NC - 1) / M)
            assert tc[k0] <= f[j] <= tc[min(k1, NC - 1)], (j, f[j], tc[k0], tc[k1])


def test_flat_distribution_inverse_cdf_closed_form(cube):
    """With every interval of mass 1/(n - 1) the inverse CDF is piecewise linear through the
    knots (k/(n - 1), t_k): draw j at u_j = (j + xi_j)/M, xi_j the 24-bit SplitMix64 draw of
    stream 3, slot 1 + N_c + j, lands at t_k + (u_j (n - 1) - k)(t_k+1 - t_k), k = floor(u_j (n - 1))."""
    cfg, F = cube
    th = zero_params(CUBE).astype(np.float64)
    set_level_field(CUBE, th, 0, 0, lambda X: np.full(X.shape[:-1], 0.3))
    passthrough_decoder(CUBE, th, 0)
    seed, step = 5, 2
    c = oc.sample_importance(cfg, F, th, seed, step, 24, NC, 0, M)
    b = oc.sample_importance(cfg, F, th, seed, step, 24, NC, 1, M)
    for i, (tc, f) in enumerate(zip(c["t"], _fine(c["t"], b["t"]))):
        tc = tc.astype(np.float64)
        f = np.sort(f).astype(np.float64)
        for j in range(M):
            xi = (oc.draw(seed, 3, step, i, 1 + NC + j) >> 40) * 2.0 ** -24
            v = (j + xi) / M * (NC - 1)
            k = min(int(math.floor(v)), NC - 2)
            want = tc[k] + (v - k) * (tc[k + 1] - tc[k])
            assert abs(f[j] - want) <= 1e-6 * max(1.0, abs(want)), (i, j, f[j], want)


def test_importance_samples_gather_at_a_sharp_surface(cube):
    """phi = -z exactly (affine field, pass-through decoder) and s = 5000: on a ray going up
    through z = 0 inside the grid box the weight sits in the coarse interval that holds the
    crossing t* = -o_z / r_z, so nearly every importance sample falls there."""
    cfg, F = cube
    th = zero_params(CUBE).astype(np.float64)
    set_level_field(CUBE, th, 3, 1, lambda X: -X[..., 2])
    passthrough_decoder(CUBE, th, 13, kappa=math.log(5000.0))
    R = 400
    c = oc.sample_importance(cfg, F, th, 9, 1, R, NC, 0, M)
    b = oc.sample_importance(cfg, F, th, 9, 1, R, NC, STEPS, M)
    o, r = b["o"].astype(np.float64), b["r"].astype(np.float64)
    used = inside = 0
    for i, (tc, f) in enumerate(zip(c["t"], _fine(c["t"], b["t"]))):
        if not (o[i, 2] < 0 and r[i, 2] > 0):
            continue
        ts = -o[i, 2] / r[i, 2]
        xc = o[i] + ts * r[i]
        if not (CUBE.near + 0.1 < ts < CUBE.far - 0.1 and np.all(np.abs(xc[:2]) < 1.2)):
            continue
        k = np.searchsorted(tc, ts) - 1
        lo, hi = tc[max(k - 1, 0)], tc[min(k + 2, NC - 1)]
        used += len(f)
        inside += int(np.sum((f >= lo) & (f <= hi)))
    assert used >= 20 * STEPS * M
    assert inside >= 0.97 * used, (inside, used)


def test_reproducible_and_keyed(cube):
    cfg, F = cube
    th = sg.parity_params(CUBE, seed=4).astype(np.float64)
    a = oc.sample_importance(cfg, F, th, 3, 7, 16, NC, STEPS, M)
    b = oc.sample_importance(cfg, F, th, 3, 7, 16, NC, STEPS, M)
    c = oc.sample_importance(cfg, F, th, 3, 8, 16, NC, STEPS, M)
    assert np.array_equal(a["t"], b["t"]) and not np.array_equal(a["t"], c["t"])
    with pytest.raises(ValueError):
        oc.sample_importance(cfg, F, th, 3, 7, 4, NC, 1, 65)
