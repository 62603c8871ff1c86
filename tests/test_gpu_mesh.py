"""Mesh extraction (gs_extract_mesh) against the FP64 oracle: lattice SDF values, the same
triangles (matched by position), a closed genus-0 surface on the GPU's own output, and the
room workload's learned-SDF shape at a coarse lattice."""
import numpy as np
import pytest
import torch

import oracle as oc
import scenegen as sg
from gpu_common import Problem
from helpers import CUBE, passthrough_decoder, sdf_parity_params, set_level_field, zero_params

pytestmark = pytest.mark.gpu


def _match(got, ref, tol, min_frac=1.0):
    """Pairs every GPU triangle with the oracle triangle of nearest centroid (one to one) and
    compares their vertices in order (the orientation included); at least min_frac of the
    oracle's triangles must be matched within tol."""
    from scipy.spatial import cKDTree
    cg, cr = got.mean(axis=1), ref.mean(axis=1)
    dist, idx = cKDTree(cr).query(cg)
    ok = dist <= tol
    ok &= np.abs(got - ref[idx]).reshape(len(got), -1).max(axis=1) <= tol
    pairs = idx[ok]
    assert len(np.unique(pairs)) == len(pairs)
    assert len(pairs) >= min_frac * len(ref), (len(pairs), len(got), len(ref))
    assert len(got) - len(pairs) <= (1.0 - min_frac) * len(ref), (len(pairs), len(got), len(ref))


@pytest.fixture(scope="module")
def sphere():
    p = Problem(CUBE)
    th = zero_params(CUBE)
    set_level_field(CUBE, th, 3, 0, lambda X: np.linalg.norm(X, axis=-1) - 0.5)
    passthrough_decoder(CUBE, th, 12)
    return p, th


def test_sphere_matches_oracle_and_is_closed(sphere):
    p, th = sphere
    lo, step, dims = (-0.8818, -0.8902, -0.8766), 0.05, (36, 36, 36)
    ref, phi_ref = oc.extract_mesh(p.cfg, th, lo, step, dims)
    # no lattice value within FP32 rounding (about 1e-7 here) of the surface
    assert np.abs(phi_ref).min() > 2e-5
    tris, n = p.ctx.extract_mesh(torch.from_numpy(th).cuda(), lo, step, dims)
    got = tris.cpu().numpy().astype(np.float64)
    _match(got, ref, 1e-5)
    # closed and genus 0 on the GPU's own (FP32) vertices
    edges = {}
    for t in tris.cpu().numpy():
        for a, b in ((0, 1), (1, 2), (2, 0)):
            k = tuple(sorted((tuple(t[a]), tuple(t[b]))))
            edges[k] = edges.get(k, 0) + 1
    assert set(edges.values()) == {2}
    verts = {tuple(v) for v in tris.cpu().numpy().reshape(-1, 3)}
    assert len(verts) - len(edges) + n == 2


def test_lattice_values_and_truncated_output(sphere):
    p, th = sphere
    lo, step, dims = (-0.6, -0.5, -0.4), 0.1, (13, 11, 9)
    ref, phi_ref = oc.extract_mesh(p.cfg, th, lo, step, dims, iso=0.05)
    phi = torch.empty((dims[2], dims[1], dims[0]), device="cuda")
    _, n = p.ctx.extract_mesh(torch.from_numpy(th).cuda(), lo, step, dims, iso=0.05, phi=phi)
    np.testing.assert_allclose(phi.cpu().numpy(), phi_ref, atol=2e-6)
    assert n == len(ref)
    # too little room: the count is complete, only max_tris triangles are written
    L = p.ctx.L
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    small = torch.full((5, 3, 3), -7.0, device="cuda")
    import ctypes
    lo_h = (ctypes.c_float * 3)(*lo)
    st = L.gs_extract_mesh(p.ctx.h, ctypes.c_void_p(torch.from_numpy(th).cuda().data_ptr()), lo_h, step, *dims, 0.05,
                           ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(small.data_ptr()), 5,
                           ctypes.c_void_p(cnt.data_ptr()), None)
    torch.cuda.synchronize()
    assert st == 0 and int(cnt.item()) == n and not torch.any(small == -7.0)


def test_no_surface(sphere):
    p, th = sphere
    tris, n = p.ctx.extract_mesh(torch.from_numpy(th).cuda(), (-0.1, -0.1, -0.1), 0.05, (5, 5, 5))
    assert n == 0  # every lattice value is inside the sphere


def test_room_learned_sdf_coarse_lattice():
    """The room workload's parameters with the scene's SDF baked in, a 6 cm lattice over the
    whole room: the same triangles as the oracle's, except where a lattice value lies within
    FP32 rounding of the surface."""
    w = sg.WORKLOADS["room-8192x96"]
    p = Problem(w, n_frames=2)
    th = sdf_parity_params(w, sg.room_scene(), seed=31)
    lo, step = (0.03, 0.03, 0.03), 0.06
    dims = (int(7.94 / step) + 1, int(5.94 / step) + 1, int(2.94 / step) + 1)
    ref, phi_ref = oc.extract_mesh(p.cfg, th, lo, step, dims)
    phi = torch.empty((dims[2], dims[1], dims[0]), device="cuda")
    tris, n = p.ctx.extract_mesh(torch.from_numpy(th).cuda(), lo, step, dims, phi=phi)
    d = np.abs(phi.cpu().numpy() - phi_ref)
    assert d.max() <= 1e-5 * max(1.0, np.abs(phi_ref).max()), d.max()
    near = int((np.abs(phi_ref) < 2e-5).sum())  # lattice values whose sign FP32 may not share
    assert len(ref) > 10000
    # a near-surface lattice value can change the triangles of its 8 cells (12 each at most)
    slack = 96 * near / len(ref)
    _match(tris.cpu().numpy().astype(np.float64), ref, 1e-4, min_frac=1.0 - slack)
