"""Seeded synthetic inputs shared by the CUDA path's tests, the bench and the CPU oracle.

This package makes inputs only: scene primitives, posed RGB-D frames rendered by exact
ray casting of those primitives, workload configurations and seeded parameter
initialisations.  It contains no step of the reconstruction method (no feature-grid
interpolation, decoding, volume rendering, loss or update), so the CUDA library and the
oracle stay independent of each other while reading identical inputs.

Workloads stand in for the paper's datasets (ScanNet and the Neural RGB-D synthetic
scenes are not available here): a 2.56 m cube with a sphere and a box seen by one
160x120 camera, and an 8x6x3 m room built from seeded primitives seen along a smooth
1000-pose trajectory at 640x480, the room scale of the paper's performance table.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()

SEED_SCENE, SEED_TRAJ, SEED_RAYS, SEED_INIT = 1, 2, 3, 4

MLP_SHAPES = [("W1", (32, 16)), ("b1", (32,)), ("W2", (16, 32)), ("b2", (16,)),
              ("W3", (32, 15)), ("b3", (32,)), ("W4", (3, 32)), ("b4", (3,)), ("kappa", (1,))]
MLP_PARAMS = sum(int(np.prod(s)) for _, s in MLP_SHAPES)  # 1684
FEAT = 4
LEVELS = 4
# the paper's architecture (Sec. 3.1): a colour grid of 6 features per vertex at the finest
# level, and two decoders with two hidden layers of 32 (the colour decoder also reads the
# unit viewing direction)
COLOUR_FEAT = 6
PAPER_MLP_SHAPES = [("gW1", (32, 16)), ("gb1", (32,)), ("gW2", (32, 32)), ("gb2", (32,)), ("gw3", (1, 32)),
                    ("gb3", (1,)), ("cW1", (32, 9)), ("cb1", (32,)), ("cW2", (32, 32)), ("cb2", (32,)),
                    ("cW3", (3, 32)), ("cb3", (3,)), ("kappa", (1,))]
PAPER_MLP_PARAMS = sum(int(np.prod(s)) for _, s in PAPER_MLP_SHAPES)  # 3109


class _Prim(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("pad", ctypes.c_int32), ("a", ctypes.c_double * 3),
                ("b", ctypes.c_double * 3), ("r", ctypes.c_double), ("col", ctypes.c_double * 3)]


def build(force: bool = False) -> str:
    """Compile the frame renderer (gcc, OpenMP) into scenegen/_build/; returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    so = os.path.join(_BUILD, "libscenegen.so")
    src = os.path.join(_HERE, "raycast.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", src, "-o", tmp, "-lm"])
        os.replace(tmp, so)
    return so


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            lib.sg_render.restype = None
            lib.sg_render.argtypes = [ctypes.POINTER(_Prim), ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p]
            lib.sg_sdf.restype = ctypes.c_double
            lib.sg_sdf.argtypes = [ctypes.POINTER(_Prim), ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
            lib.sg_sdf_batch.restype = None
            lib.sg_sdf_batch.argtypes = [ctypes.POINTER(_Prim), ctypes.c_int, ctypes.c_void_p, ctypes.c_longlong,
                                         ctypes.c_void_p]
            _LIB = lib
    return _LIB


# --------------------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------------------
@dataclass
class Scene:
    prims: list  # (kind, a, b, r, col)
    shade_mode: int

    def _array(self):
        arr = (_Prim * len(self.prims))()
        for i, (kind, a, b, r, col) in enumerate(self.prims):
            arr[i].kind = kind
            arr[i].a[:] = list(a)
            arr[i].b[:] = list(b)
            arr[i].r = r
            arr[i].col[:] = list(col)
        return arr

    def sdf(self, x) -> np.ndarray:
        """Exact scene SDF at points x [P,3] (float64)."""
        x = np.ascontiguousarray(np.asarray(x, dtype=np.float64).reshape(-1, 3))
        out = np.empty(len(x))
        _lib().sg_sdf_batch(self._array(), len(self.prims), x.ctypes.data, len(x), out.ctypes.data)
        return out


def cube_scene() -> Scene:
    """Sphere r=0.5 m at (-0.4,0,0) and an axis-aligned box (centre (0.55,0,0), half extent 0.3 m)."""
    return Scene(prims=[(2, (-0.4, 0.0, 0.0), (0, 0, 0), 0.5, (1, 1, 1)),
                        (1, (0.55, 0.0, 0.0), (0.3, 0.3, 0.3), 0.0, (1, 1, 1))], shade_mode=0)


def _ellipse_path(n=256):
    a = np.linspace(0, 2 * np.pi, n, endpoint=False)
    return np.stack([4 + 3 * np.cos(a), 3 + 2 * np.sin(a), 1.55 + 0.15 * np.sin(3 * a)], 1)


def room_scene(seed: int = SEED_SCENE, size=(8.0, 6.0, 3.0)) -> Scene:
    """Room interior (floor, ceiling, four walls) plus 20 boxes, 10 spheres and 5 capsules.

    Objects rest on the floor or against a wall and keep clear of the camera trajectory.
    """
    rng = np.random.default_rng(seed)
    sx, sy, sz = size
    prims = [(0, (sx / 2, sy / 2, sz / 2), (sx / 2, sy / 2, sz / 2), 0.0, (0.8, 0.78, 0.72))]
    path = _ellipse_path()

    def clear(c, rad):
        return np.min(np.linalg.norm(path - np.asarray(c)[None], axis=1)) > rad + 0.45

    def colour():
        return tuple(0.25 + 0.7 * rng.random(3))

    n_box = 0
    while n_box < 20:
        h = rng.uniform(0.2, 1.5, 3) / 2
        if rng.random() < 0.7:  # on the floor
            c = (rng.uniform(h[0], sx - h[0]), rng.uniform(h[1], sy - h[1]), h[2])
        else:  # against a wall (x=0 or x=sx), at a seeded height
            wx = h[0] if rng.random() < 0.5 else sx - h[0]
            c = (wx, rng.uniform(h[1], sy - h[1]), rng.uniform(h[2], sz - h[2]))
        if clear(c, float(np.linalg.norm(h))):
            prims.append((1, c, tuple(h), 0.0, colour()))
            n_box += 1
    n_sph = 0
    while n_sph < 10:
        r = rng.uniform(0.15, 0.5)
        c = (rng.uniform(r, sx - r), rng.uniform(r, sy - r), r if rng.random() < 0.6 else rng.uniform(r, sz - r))
        if clear(c, r):
            prims.append((2, c, (0, 0, 0), r, colour()))
            n_sph += 1
    n_cap = 0
    while n_cap < 5:
        r = rng.uniform(0.05, 0.2)
        L = rng.uniform(0.3, 1.5)
        if rng.random() < 0.5:  # standing on the floor
            x, y = rng.uniform(r, sx - r), rng.uniform(r, sy - r)
            a, b = (x, y, r), (x, y, r + L)
        else:  # lying on the floor along x or y
            if rng.random() < 0.5:
                x, y = rng.uniform(r, sx - r - L), rng.uniform(r, sy - r)
                a, b = (x, y, r), (x + L, y, r)
            else:
                x, y = rng.uniform(r, sx - r), rng.uniform(r, sy - r - L)
                a, b = (x, y, r), (x, y + L, r)
        mid = tuple((np.asarray(a) + np.asarray(b)) / 2)
        if clear(mid, L / 2 + r):
            prims.append((3, a, b, r, colour()))
            n_cap += 1
    return Scene(prims=prims, shade_mode=1)


# --------------------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------------------
def look_at(pos, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """c2w [3,4] for an OpenCV camera (x right, y down, z forward) at pos looking at target."""
    pos, target, up = (np.asarray(v, dtype=np.float64) for v in (pos, target, up))
    fwd = target - pos
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, up)
    if np.linalg.norm(right) < 1e-9:
        right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    return np.concatenate([np.stack([right, down, fwd], 1), pos[:, None]], 1)


def cube_poses(seed: int = SEED_TRAJ, n: int = 1) -> np.ndarray:
    """Seeded camera positions on the radius-1.1 m sphere, looking at the origin."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        v = rng.normal(size=3)
        v /= np.linalg.norm(v)
        out.append(look_at(1.1 * v, (0, 0, 0), up=(0, 0, 1) if abs(v[2]) < 0.95 else (0, 1, 0)))
    return np.stack(out)


def room_poses(n: int = 1000, seed: int = SEED_TRAJ) -> np.ndarray:
    """Smooth closed trajectory: ellipse of radii 3x2 m at 1.4-1.7 m height, look-at point
    orbiting the room centre, plus seeded low-frequency jitter."""
    rng = np.random.default_rng(seed)
    amp = rng.uniform(0.01, 0.04, (3, 3))
    ph = rng.uniform(0, 2 * np.pi, (3, 3))
    ps = rng.uniform(0, 2 * np.pi, 2)
    out = []
    for k in range(n):
        a = 2 * np.pi * k / n
        jit = np.array([sum(amp[m, ax] * np.sin((m + 1) * 2 * a + ph[m, ax]) for m in range(3)) for ax in range(3)])
        pos = np.array([4 + 3 * np.cos(a), 3 + 2 * np.sin(a), 1.55 + 0.15 * np.sin(3 * a)]) + jit
        tgt = np.array([4 + 1.2 * np.cos(2 * a + ps[0]), 3 + 0.8 * np.sin(2 * a + ps[1]), 0.8 + 0.2 * np.sin(a)])
        out.append(look_at(pos, tgt))
    return np.stack(out)


# --------------------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------------------
def grid_dims(extent_min, extent_max, voxels):
    """Vertex counts per level (nx, ny, nz): ceil(E / v) + 1 per axis, vertex-aligned grid."""
    dims = []
    for v in voxels:
        dims.append(tuple(int(math.ceil((hi - lo) / v - 1e-6)) + 1 for lo, hi in zip(extent_min, extent_max)))
    return dims


@dataclass
class Workload:
    name: str
    extent_min: tuple
    extent_max: tuple
    voxels: tuple           # level 0 (coarsest) .. 3 (finest), metres
    rays: int
    n_strat: int
    n_guided: int
    near: float
    far: float
    frames: int
    height: int
    width: int
    fx: float
    fy: float
    cx: float
    cy: float
    scene: str              # "cube" | "room"
    noise_k: float = 0.0
    drop_p: float = 0.0
    blob_frac: float = 0.0
    trunc: float = 0.10
    guide_half: float = 0.10
    kappa_fs: float = 5.0
    lambdas: tuple = (10.0, 1.0, 10.0, 1.0, 1.0)  # rgb, depth, sdf, fs, smooth
    n_smooth: int = 4096
    delta_s: float = 0.004
    lr_grid: float = 1e-2
    lr_mlp: float = 1e-3
    betas: tuple = (0.9, 0.999)
    adam_eps: float = 1e-8
    precision: str = "fp32"
    prop_samples: int = 0   # learned proposal: samples per ray of a proposal batch (0 = off)
    prop_guided: int = 8    # of those, depth-guided when D > 0
    lr_prop: float = 1e-3
    imp_coarse: int = 0     # hierarchical importance sampler: coarse samples (0 = off)
    imp_steps: int = 0      # importance steps
    imp_per_step: int = 0   # samples added per step
    arch: str = "compact"   # "compact": 16-32-16 / 15-32-3 decoders; "paper": colour grid + 2-hidden-layer decoders
    extra: dict = field(default_factory=dict)

    @property
    def n_samples(self) -> int:
        """Samples per ray of the workload's batches (the importance sampler's when it is on)."""
        if self.imp_coarse > 0:
            return self.imp_coarse + self.imp_steps * self.imp_per_step
        return self.n_strat + self.n_guided

    @property
    def dims(self):
        return grid_dims(self.extent_min, self.extent_max, self.voxels)

    @property
    def mlp_shapes(self):
        return PAPER_MLP_SHAPES if self.arch == "paper" else MLP_SHAPES

    def layout(self):
        """Flat parameter vector: grid levels 0..3 as [nz][ny][nx][4] float32, then (paper
        architecture) the colour grid [nz][ny][nx][6] of level 3 padded to a multiple of 4
        floats, then the decoder block.  Returns (level offsets, grid floats, total floats)."""
        offs, o = [], 0
        for (nx, ny, nz) in self.dims:
            offs.append(o)
            o += nx * ny * nz * FEAT
        if self.arch == "paper":
            o += self.colour_floats()
            return offs, o, o + PAPER_MLP_PARAMS
        return offs, o, o + MLP_PARAMS

    def colour_offset(self) -> int:
        """Float offset of the colour grid (paper architecture): right after the geometry levels."""
        return sum(nx * ny * nz * FEAT for (nx, ny, nz) in self.dims)

    def colour_floats(self) -> int:
        nx, ny, nz = self.dims[3]
        return (nx * ny * nz * COLOUR_FEAT + 3) // 4 * 4

    def with_(self, **kw) -> "Workload":
        d = dict(self.__dict__)
        d.update(kw)
        return Workload(**d)


WORKLOADS = {
    # 2.56 m cube, 1 camera 160x120, 1024 rays x (48 stratified + 16 depth-guided)
    "cube-1024x64": Workload(
        name="cube-1024x64", extent_min=(-1.28, -1.28, -1.28), extent_max=(1.28, 1.28, 1.28),
        voxels=(0.64, 0.32, 0.16, 0.08), rays=1024, n_strat=48, n_guided=16, near=0.1, far=4.0,
        frames=1, height=120, width=160, fx=130.0, fy=130.0, cx=80.0, cy=60.0, scene="cube"),
    # 8x6x3 m room, 1000 poses at 640x480, 8192 rays x (64 + 32), FP32
    "room-8192x96": Workload(
        name="room-8192x96", extent_min=(0.0, 0.0, 0.0), extent_max=(8.0, 6.0, 3.0),
        voxels=(0.96, 0.24, 0.06, 0.02), rays=8192, n_strat=64, n_guided=32, near=0.1, far=6.0,
        frames=1000, height=480, width=640, fx=525.0, fy=525.0, cx=320.0, cy=240.0, scene="room",
        noise_k=0.001, drop_p=0.05),
}
WORKLOADS["room-bf16-32768x96"] = WORKLOADS["room-8192x96"].with_(name="room-bf16-32768x96", rays=32768,
                                                                   precision="bf16")
WORKLOADS["room-diff-65536x96"] = WORKLOADS["room-8192x96"].with_(name="room-diff-65536x96", rays=65536)
# the paper's own sampler (Sec. 3.2, Sec. 4): 96 coarse samples and 3 importance steps of 12
WORKLOADS["room-imp-8192x132"] = WORKLOADS["room-8192x96"].with_(name="room-imp-8192x132", imp_coarse=96, imp_steps=3,
                                                                  imp_per_step=12)
# learned-proposal form: 30% of every depth frame zeroed in contiguous blobs, 65536 rays,
# 32 samples per ray (24 drawn from the proposal + 8 depth-guided), plain 64 + 32 as fallback
WORKLOADS["room-prop-65536x32"] = WORKLOADS["room-8192x96"].with_(name="room-prop-65536x32", rays=65536,
                                                                   blob_frac=0.3, prop_samples=32, prop_guided=8)
# the precision form with the learned proposal: BF16 gathers and decoders (FP32 master,
# gradients and moments), 8 proposal + 24 depth-guided samples per ray where the observed
# depth exists (all 32 from the proposal where it is missing), plain 64 + 32 as fallback
WORKLOADS["room-prop-bf16-65536x32"] = WORKLOADS["room-prop-65536x32"].with_(name="room-prop-bf16-65536x32",
                                                                             precision="bf16", prop_guided=24)
# the paper's architecture (Sec. 3.1): colour grid at the finest level, view direction,
# decoders with two hidden layers of 32
WORKLOADS["cube-paper-1024x64"] = WORKLOADS["cube-1024x64"].with_(name="cube-paper-1024x64", arch="paper")
WORKLOADS["room-paper-8192x96"] = WORKLOADS["room-8192x96"].with_(name="room-paper-8192x96", arch="paper")
# the paper's method as a whole (Sec. 3-4): its architecture, its sampler (96 coarse + 3 x 12)
# and (bench --eikonal) its Eikonal term
WORKLOADS["room-paper-imp-8192x132"] = WORKLOADS["room-paper-8192x96"].with_(name="room-paper-imp-8192x132",
                                                                             imp_coarse=96, imp_steps=3,
                                                                             imp_per_step=12)


@dataclass
class Frames:
    rgb: np.ndarray    # uint8 [F,H,W,3]
    depth: np.ndarray  # float32 [F,H,W], 0 = missing
    c2w: np.ndarray    # float32 [F,3,4]
    fx: float
    fy: float
    cx: float
    cy: float
    gt_depth: np.ndarray | None = None


def make_frames(w: Workload, n_frames: int | None = None, with_gt: bool = False) -> Frames:
    """Render the workload's frames (optionally only the first n_frames poses)."""
    F = w.frames if n_frames is None else n_frames
    if w.scene == "cube":
        scene, poses = cube_scene(), cube_poses(n=F)
    else:
        scene, poses = room_scene(), room_poses(n=w.frames)[:F]
    poses = np.ascontiguousarray(poses, dtype=np.float64)
    H, W = w.height, w.width
    rgb = np.empty((F, H, W, 3), np.uint8)
    depth = np.empty((F, H, W), np.float32)
    gt = np.empty((F, H, W), np.float32) if with_gt else None
    arr = scene._array()
    _lib().sg_render(arr, len(scene.prims), scene.shade_mode, poses.ctypes.data, F, H, W, w.fx, w.fy, w.cx, w.cy,
                     w.noise_k, w.drop_p, w.blob_frac, SEED_SCENE, rgb.ctypes.data, depth.ctypes.data,
                     gt.ctypes.data if gt is not None else None)
    return Frames(rgb=rgb, depth=depth, c2w=poses.astype(np.float32), fx=w.fx, fy=w.fy, cx=w.cx, cy=w.cy,
                  gt_depth=gt)


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
    view = theta[offs[level]:offs[level] + nx * ny * nz * FEAT].reshape(nz, ny, nx, FEAT)
    view[..., feat] = fn(vertex_positions(w, level))
    return theta


def sdf_params(w, scene, seed=21, grid_std=0.05, bias=0.25, pass_offset=3.0, mix=0.1):
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
    m = mlp_views(theta, n_grid)
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


def sdf_switching_params(w, scene, seed=21, grid_std=0.1, bias=0.02, mix=0.1, phi_shift=0.03):
    """Parameters for element-wise GPU-vs-oracle parity whose hidden ReLU units switch from
    sample to sample: the scene's exact SDF baked into feature 0 of the finest level (so the
    rendering is that of a real surface), random features of O(0.1) elsewhere, and both
    decoders with weights U(+-0.25) / U(+-0.2) and biases U(+-bias) near zero, so that every
    unit other than the two pass-through units is on for some samples and off for others.

    Hidden units 0 and 1 of the geometry decoder carry phi = z[12] + phi_shift exactly as
    relu(v) - relu(-v) = v (no offset: near the surface, where phi is small, its binary32 and
    bfloat16 roundings stay small too); the shift keeps the truncated-SDF loss well above
    them.  The switching units add a nonlinear term to phi (weights `mix`) and form the colour
    features.  Samples whose units lie within binary32 rounding of a kink are flagged by the
    oracle and left out by the parity tests."""
    import math
    rng = np.random.default_rng(seed)
    offs, n_grid, n_tot = w.layout()
    theta = np.zeros(n_tot, np.float32)
    theta[:n_grid] = rng.normal(0.0, grid_std, n_grid).astype(np.float32)
    nx, ny, nz = w.dims[3]
    X = vertex_positions(w, 3)
    sdf = scene.sdf(X.reshape(-1, 3)).reshape(nz, ny, nx)
    set_level_field(w, theta, 3, 0, lambda _: sdf)
    m = mlp_views(theta, n_grid)
    m["W1"][:] = rng.uniform(-0.25, 0.25, m["W1"].shape)
    m["W1"][:, 12] = 0.0  # the SDF feature reaches phi only through the pass-through units
    m["b1"][:] = rng.uniform(-bias, bias, 32)
    m["W1"][0, :] = 0.0
    m["W1"][1, :] = 0.0
    m["W1"][0, 12] = 1.0
    m["W1"][1, 12] = -1.0
    m["b1"][0] = m["b1"][1] = 0.0
    m["W2"][:] = rng.uniform(-0.25, 0.25, m["W2"].shape)
    m["W2"][0, :] = rng.uniform(-mix, mix, 32)
    m["W2"][1:, :2] = 0.0  # the colour features do not see the pass-through units
    m["W2"][0, 0], m["W2"][0, 1] = 1.0, -1.0
    m["b2"][:] = rng.uniform(-bias, bias, 16)
    m["b2"][0] = phi_shift
    m["W3"][:] = rng.uniform(-0.25, 0.25, m["W3"].shape)
    m["b3"][:] = rng.uniform(-bias, bias, 32) * 0.2
    m["W4"][:] = rng.uniform(-1.0, 1.0, m["W4"].shape)
    m["b4"][:] = rng.uniform(-0.2, 0.2, 3)
    m["kappa"][0] = math.log(20.0)
    return theta


def init_params(w: Workload, seed: int = SEED_INIT) -> np.ndarray:
    """Default initialisation: grid features N(0, 1e-4^2); MLP weights U(+-1/sqrt(fan_in)),
    biases 0; kappa = ln 20 (s = 20 1/m)."""
    rng = np.random.default_rng(seed)
    offs, n_grid, n_total = w.layout()
    theta = np.empty(n_total, np.float32)
    theta[:n_grid] = rng.normal(0.0, 1e-4, n_grid).astype(np.float32)
    if w.arch == "paper":
        _zero_colour_padding(w, theta)
    o = n_grid
    for name, shape in w.mlp_shapes:
        n = int(np.prod(shape))
        if name.startswith("W") or name[1:2] in ("W", "w"):
            bound = 1.0 / math.sqrt(shape[1])
            theta[o:o + n] = rng.uniform(-bound, bound, n).astype(np.float32)
        elif name == "kappa":
            theta[o] = np.float32(math.log(20.0))
        else:
            theta[o:o + n] = 0.0
        o += n
    return theta


def parity_params(w: Workload, seed: int = 11, grid_std: float = 0.05, bias: float = 0.25,
                  kappa: float = math.log(20.0)) -> np.ndarray:
    """Parameters for element-wise parity tests.

    Grid features are N(0, grid_std^2) so that decoded values vary along every ray; the two
    hidden layers get biases of alternating sign and magnitude `bias`, which keeps every
    hidden pre-activation far from the ReLU kink (units are always on or always off), so an
    FP32 and an FP64 evaluation take the same branch at every sample.
    """
    rng = np.random.default_rng(seed)
    theta = init_params(w, seed)
    offs, n_grid, n_total = w.layout()
    theta[:n_grid] = rng.normal(0.0, grid_std, n_grid).astype(np.float32)
    o = n_grid
    for name, shape in MLP_SHAPES:
        n = int(np.prod(shape))
        if name in ("b1", "b3"):
            sign = np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
            theta[o:o + n] = (sign * bias).astype(np.float32)
        elif name in ("b2", "b4"):
            theta[o:o + n] = rng.uniform(-0.1, 0.1, n).astype(np.float32)
        elif name == "kappa":
            theta[o] = np.float32(kappa)
        o += n
    return theta


def _zero_colour_padding(w, theta):
    nx, ny, nz = w.dims[3]
    theta[w.colour_offset() + nx * ny * nz * COLOUR_FEAT:w.colour_offset() + w.colour_floats()] = 0.0


def colour_view(w, theta) -> np.ndarray:
    """The colour grid [nz][ny][nx][6] of a paper-architecture parameter vector (a view)."""
    nx, ny, nz = w.dims[3]
    o = w.colour_offset()
    return theta[o:o + nx * ny * nz * COLOUR_FEAT].reshape(nz, ny, nx, COLOUR_FEAT)


def paper_sdf_params(w, scene, seed=23, grid_std=0.05, mix=0.1):
    """Paper-architecture parameters for element-wise parity (the analogue of sdf_params):
    the scene's exact SDF in feature 0 of the finest geometry level, random features elsewhere
    (colour grid included), and decoders whose every hidden unit stays far from its kink.

    Geometry: hidden-1 units 0, 1 carry z[12] as relu(z + 3), relu(3 - z); hidden-2 unit 0
    takes 0.5 (difference) + 3 = z + 3 (always on) and gw3[0] = 1, gb3 = -3, so phi = z[12]
    plus a small term (weights `mix`) from the other units.  Those units have biases of
    alternating sign (0.25 in layer 1, 0.5 in layer 2) and weights small enough that no
    pre-activation reaches zero.  Colour: biases of alternating sign 0.5, small weights on
    the viewing direction."""
    assert w.arch == "paper"
    rng = np.random.default_rng(seed)
    offs, n_grid, n_tot = w.layout()
    theta = np.zeros(n_tot, np.float32)
    theta[:n_grid] = rng.normal(0.0, grid_std, n_grid).astype(np.float32)
    _zero_colour_padding(w, theta)
    nx, ny, nz = w.dims[3]
    X = vertex_positions(w, 3)
    sdf = scene.sdf(X.reshape(-1, 3)).reshape(nz, ny, nx)
    set_level_field(w, theta, 3, 0, lambda _: sdf)
    m = mlp_views(theta, n_grid, PAPER_MLP_SHAPES)
    alt = np.where(np.arange(32) % 2 == 0, 1.0, -1.0)
    m["gW1"][:] = rng.uniform(-0.25, 0.25, (32, 16))
    m["gW1"][:, 12] = 0.0
    m["gW1"][:2, :] = 0.0
    m["gW1"][0, 12], m["gW1"][1, 12] = 1.0, -1.0
    m["gb1"][:] = 0.25 * alt
    m["gb1"][0] = m["gb1"][1] = 3.0
    m["gW2"][:] = rng.uniform(-0.05, 0.05, (32, 32))
    m["gW2"][:, :2] = 0.0
    m["gW2"][0, :] = 0.0
    m["gW2"][0, 0], m["gW2"][0, 1] = 0.5, -0.5
    m["gb2"][:] = 0.5 * alt
    m["gb2"][0] = 3.0
    m["gw3"][0, :] = rng.uniform(-mix, mix, 32)
    m["gw3"][0, 0] = 1.0
    m["gb3"][0] = -3.0
    m["cW1"][:] = rng.uniform(-0.25, 0.25, (32, 9))
    m["cW1"][:, 6:] = rng.uniform(-0.1, 0.1, (32, 3))
    m["cb1"][:] = 0.5 * alt
    m["cW2"][:] = rng.uniform(-0.03, 0.03, (32, 32))
    m["cb2"][:] = 0.5 * alt
    m["cW3"][:] = rng.uniform(-0.5, 0.5, (3, 32))
    m["cb3"][:] = rng.uniform(-0.2, 0.2, 3)
    m["kappa"][0] = math.log(20.0)
    return theta


def paper_switching_params(w, scene, seed=23, grid_std=0.1, bias=0.02, mix=0.1, phi_shift=0.03):
    """Paper-architecture parameters whose hidden ReLU units switch from sample to sample
    (the analogue of sdf_switching_params): the scene's exact SDF in feature 0 of the finest
    geometry level, random features of O(0.1) elsewhere (colour grid included), and all four
    hidden layers with biases U(+-bias) near zero, so every unit but the pass-through ones is
    on for some samples and off for others.

    Geometry: hidden-1 units 0, 1 carry relu(z[12]), relu(-z[12]); hidden-2 units 0, 1 take
    their differences z and -z, and gw3 = (1, -1, ...), gb3 = phi_shift, so phi = z[12] +
    phi_shift (relu(v) - relu(-v) = v, no offset) plus a term (weights `mix`) from the
    switching units."""
    assert w.arch == "paper"
    rng = np.random.default_rng(seed)
    offs, n_grid, n_tot = w.layout()
    theta = np.zeros(n_tot, np.float32)
    theta[:n_grid] = rng.normal(0.0, grid_std, n_grid).astype(np.float32)
    _zero_colour_padding(w, theta)
    nx, ny, nz = w.dims[3]
    X = vertex_positions(w, 3)
    sdf = scene.sdf(X.reshape(-1, 3)).reshape(nz, ny, nx)
    set_level_field(w, theta, 3, 0, lambda _: sdf)
    m = mlp_views(theta, n_grid, PAPER_MLP_SHAPES)
    m["gW1"][:] = rng.uniform(-0.25, 0.25, (32, 16))
    m["gW1"][:, 12] = 0.0
    m["gW1"][:2, :] = 0.0
    m["gW1"][0, 12], m["gW1"][1, 12] = 1.0, -1.0
    m["gb1"][:] = rng.uniform(-bias, bias, 32)
    m["gb1"][0] = m["gb1"][1] = 0.0
    m["gW2"][:] = rng.uniform(-0.3, 0.3, (32, 32))
    m["gW2"][:, :2] = 0.0
    m["gW2"][:2, :] = 0.0
    m["gW2"][0, 0], m["gW2"][0, 1] = 1.0, -1.0
    m["gW2"][1, 0], m["gW2"][1, 1] = -1.0, 1.0
    m["gb2"][:] = rng.uniform(-bias, bias, 32) * 0.2
    m["gb2"][0] = m["gb2"][1] = 0.0
    m["gw3"][0, :] = rng.uniform(-mix, mix, 32)
    m["gw3"][0, 0], m["gw3"][0, 1] = 1.0, -1.0
    m["gb3"][0] = phi_shift
    m["cW1"][:] = rng.uniform(-0.5, 0.5, (32, 9))
    m["cb1"][:] = rng.uniform(-bias, bias, 32)
    m["cW2"][:] = rng.uniform(-0.3, 0.3, (32, 32))
    m["cb2"][:] = rng.uniform(-bias, bias, 32) * 0.2
    m["cW3"][:] = rng.uniform(-1.0, 1.0, (3, 32))
    m["cb3"][:] = rng.uniform(-0.2, 0.2, 3)
    m["kappa"][0] = math.log(20.0)
    return theta


def mlp_views(theta: np.ndarray, n_grid: int, shapes=None) -> dict:
    """Named views of the MLP block of a flat parameter vector (shapes: MLP_SHAPES by default,
    PAPER_MLP_SHAPES for the paper's architecture)."""
    out, o = {}, n_grid
    for name, shape in (MLP_SHAPES if shapes is None else shapes):
        n = int(np.prod(shape))
        out[name] = theta[o:o + n].reshape(shape)
        o += n
    return out
