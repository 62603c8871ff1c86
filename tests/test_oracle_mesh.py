"""Pins of the oracle's mesh extraction (the isosurface of phi on a lattice, Sec. 4) against
closed forms and invariants: planes (exact positions, area and normals) and a sphere
(watertight genus-0 surface, area, enclosed volume, radius)."""
import math

import numpy as np
import pytest

import oracle as oc
from helpers import CUBE, passthrough_decoder, set_level_field, zero_params


def _field(fn, level=3, feat=0):
    th = zero_params(CUBE).astype(np.float64)
    set_level_field(CUBE, th, level, feat, fn)
    passthrough_decoder(CUBE, th, 4 * level + feat)
    return th


def _areas_normals(tris):
    e1, e2 = tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0]
    n = np.cross(e1, e2)
    return 0.5 * np.linalg.norm(n, axis=1), n


def _edges(tris):
    """Undirected edges keyed by their two vertices' exact coordinates, with multiplicity."""
    keys = {}
    for t in tris:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            k = tuple(sorted((tuple(t[a]), tuple(t[b]))))
            keys[k] = keys.get(k, 0) + 1
    return keys


@pytest.fixture(scope="module")
def cfg():
    return oc.make_config(CUBE)


def test_axis_plane_exact(cfg):
    """phi = z - 0.13 (affine, so trilinear is exact): every vertex at z = 0.13, the surface
    covers the lattice's 2 x 2 m cross-section exactly, every normal is +z."""
    th = _field(lambda X: X[..., 2] - 0.13)
    tris, phi = oc.extract_mesh(cfg, th, (-1.0, -1.0, -1.0), 0.1, (21, 21, 21))
    assert len(tris) > 0
    assert np.abs(tris[..., 2] - 0.13).max() < 1e-9
    area, n = _areas_normals(tris)
    assert abs(area.sum() - 4.0) < 1e-6 * 4.0 + 1e-9
    assert np.all(n[:, 2] > 0) and np.abs(n[:, :2]).max() < 1e-9
    # the lattice values are the field at the binary32 lattice points
    z = (np.float32(-1.0) + np.arange(21, dtype=np.float32) * np.float32(0.1)).astype(np.float64)
    np.testing.assert_allclose(phi[:, 5, 7], z - 0.13, atol=1e-12)


def test_oblique_plane_positions_and_orientation(cfg):
    nvec = np.array([0.3, -0.5, 0.81])
    th = _field(lambda X: X @ nvec - 0.05)
    tris, _ = oc.extract_mesh(cfg, th, (-0.9, -0.8, -0.7), 0.07, (26, 24, 21))
    assert len(tris) > 100
    assert np.abs(tris.reshape(-1, 3) @ nvec - 0.05).max() < 1e-9
    _, n = _areas_normals(tris)
    cosang = (n @ nvec) / (np.linalg.norm(n, axis=1) * np.linalg.norm(nvec))
    assert np.all(cosang > 1 - 1e-9)


@pytest.mark.parametrize("iso", [0.0, 0.1])
def test_sphere_watertight_genus0_area_volume(cfg, iso):
    """phi = |x| - 0.5 on the finest level (trilinear approximates it to O(h^2)): the isosurface
    phi = iso is closed (every edge in exactly two triangles), has Euler characteristic 2,
    and its area and enclosed volume match a sphere of radius 0.5 + iso within 2 %."""
    r = 0.5
    th = _field(lambda X: np.linalg.norm(X, axis=-1) - r)
    tris, _ = oc.extract_mesh(cfg, th, (-0.9, -0.9, -0.9), 0.05, (37, 37, 37), iso=iso)
    R = r + iso
    edges = _edges(tris)
    assert set(edges.values()) == {2}
    verts = {tuple(v) for v in tris.reshape(-1, 3)}
    assert len(verts) - len(edges) + len(tris) == 2
    area, n = _areas_normals(tris)
    assert abs(area.sum() - 4 * math.pi * R * R) < 0.02 * 4 * math.pi * R * R
    vol = np.einsum("ij,ij->i", tris[:, 0], n).sum() / 6.0  # divergence theorem: outward normals
    assert abs(vol - 4 / 3 * math.pi * R ** 3) < 0.02 * 4 / 3 * math.pi * R ** 3
    rad = np.linalg.norm(tris.reshape(-1, 3), axis=1)
    assert np.abs(rad - R).max() < 0.01


def test_no_surface_and_truncation(cfg):
    th = _field(lambda X: np.full(X.shape[:-1], 0.4))
    tris, _ = oc.extract_mesh(cfg, th, (-0.5, -0.5, -0.5), 0.1, (5, 5, 5))
    assert len(tris) == 0
    th = _field(lambda X: X[..., 0] - 0.02)
    full, _ = oc.extract_mesh(cfg, th, (-0.5, -0.5, -0.5), 0.1, (11, 11, 11))
    part, _ = oc.extract_mesh(cfg, th, (-0.5, -0.5, -0.5), 0.1, (11, 11, 11), max_tris=7)
    assert len(part) == 7 and np.array_equal(part, full[:7])
