"""Host-side checks of the mesh extraction's cell decomposition (no GPU): the CUDA kernel counts
a cell's triangles from per-tetrahedron corner masks and emits them from the tetrahedron table;
both must describe the oracle's six tetrahedra around the corner-0-to-corner-7 diagonal, and
those six must tile the unit cell (corner q at (q & 1, (q >> 1) & 1, q >> 2))."""
import itertools
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _read(rel):
    with open(os.path.join(ROOT, rel)) as f:
        return f.read()


def _int_rows(src, name):
    m = re.search(name + r"\s*\[6\]\s*\[4\]\s*=\s*\{(.*?)\};", src, re.S)
    assert m, name
    return [tuple(int(v) for v in row.split(",")) for row in re.findall(r"\{([^{}]*)\}", m.group(1))]


def _cuda_tables():
    src = _read("paper_2206_14735_gb300/csrc/gs_mesh.cu")
    tets = _int_rows(src, "kTets")
    m = re.search(r"kTetMask\s*\[6\]\s*=\s*\{([^}]*)\}", src)
    assert m
    masks = [int(v.strip().rstrip("uU"), 16) for v in m.group(1).split(",")]
    return tets, masks


def _corner(q):
    return np.array([q & 1, (q >> 1) & 1, q >> 2], float)


def test_masks_encode_the_emitted_tetrahedra():
    tets, masks = _cuda_tables()
    assert len(tets) == 6 and len(masks) == 6
    for t, m in zip(tets, masks):
        assert m == sum(1 << q for q in t), (t, hex(m))


def test_cuda_and_oracle_decompose_the_cell_alike():
    tets, _ = _cuda_tables()
    oracle = _int_rows(_read("oracle/gosurf_oracle.c"), "oc_tets")
    assert {frozenset(t) for t in tets} == {frozenset(t) for t in oracle}


def test_six_tetrahedra_tile_the_cell():
    tets, _ = _cuda_tables()
    vols = []
    for t in tets:
        assert 0 in t and 7 in t  # all share the main diagonal
        p = [_corner(q) for q in t]
        vols.append(abs(np.linalg.det(np.stack([p[1] - p[0], p[2] - p[0], p[3] - p[0]]))) / 6.0)
    np.testing.assert_allclose(vols, 1.0 / 6.0)
    # every point of the cell lies in exactly one tetrahedron (away from their shared faces)
    rng = np.random.default_rng(0)
    X = rng.uniform(0.0, 1.0, (4000, 3))
    inside = np.zeros(len(X), int)
    for t in tets:
        p = np.stack([_corner(q) for q in t])
        T = (p[1:] - p[0]).T
        lam = np.linalg.solve(T, (X - p[0]).T).T
        bary = np.concatenate([1.0 - lam.sum(1, keepdims=True), lam], 1)
        inside += np.all(bary > -1e-12, axis=1)
    assert np.all(inside == 1)


def test_triangle_count_rule_matches_a_direct_count():
    """cnt from the masks (popcount of below-iso corners per tetrahedron: 1 or 3 -> one
    triangle, 2 -> two) over all 256 sign patterns of a cell, against counting the crossed
    edges of each tetrahedron (3 crossed edges -> a triangle, 4 -> a quad split in two)."""
    tets, masks = _cuda_tables()
    for m in range(256):
        cnt = 0
        for tm in masks:
            ni = bin(m & tm).count("1")
            cnt += 0 if ni in (0, 4) else (2 if ni == 2 else 1)
        direct = 0
        for t in tets:
            crossed = sum(((m >> a) & 1) != ((m >> b) & 1) for a, b in itertools.combinations(t, 2))
            direct += {0: 0, 3: 1, 4: 2}[crossed]
        assert cnt == direct, m
