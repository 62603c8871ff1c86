"""Plain FP64 CPU oracle of one GO-Surf optimisation step (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package.  The product (the CUDA library and its Python binding) never does,
and this package never imports the product: the two share only the seeded inputs made by
``scenegen``.

The arithmetic lives in ``gosurf_oracle.c`` (compiled here with gcc, -O2,
-ffp-contract=off, OpenMP); this module only marshals numpy arrays.  Every function cites
the passage of the paper it follows in the C source.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()

LEVELS, FEAT, MLP_PARAMS = 4, 4, 1684
CLS_NONE, CLS_TR, CLS_FS = 0, 1, 2


class OcConfig(ctypes.Structure):
    _fields_ = [("dims", (ctypes.c_int32 * 3) * 4), ("voxel", ctypes.c_float * 4), ("origin", ctypes.c_float * 3),
                ("n_strat", ctypes.c_int32), ("n_guided", ctypes.c_int32), ("near_m", ctypes.c_float),
                ("far_m", ctypes.c_float), ("guide_half", ctypes.c_float), ("trunc", ctypes.c_float),
                ("kappa_fs", ctypes.c_float), ("lam", ctypes.c_float * 5), ("n_smooth", ctypes.c_int32),
                ("delta_s", ctypes.c_float), ("arch", ctypes.c_int32)]


class OcFrames(ctypes.Structure):
    _fields_ = [("F", ctypes.c_int32), ("H", ctypes.c_int32), ("W", ctypes.c_int32), ("rgb", ctypes.c_void_p),
                ("depth", ctypes.c_void_p), ("c2w", ctypes.c_void_p), ("fx", ctypes.c_float), ("fy", ctypes.c_float),
                ("cx", ctypes.c_float), ("cy", ctypes.c_float)]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (this builds the checker; it does not run it)."""
    os.makedirs(_BUILD, exist_ok=True)
    so = os.path.join(_BUILD, "liboracle.so")
    src = os.path.join(_HERE, "gosurf_oracle.c")
    if force or not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
        tmp = so + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-fno-fast-math", src, "-o", tmp, "-lm"])
        os.replace(tmp, so)
    return so


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            _LIB = _load(build())
    return _LIB


def _load(path: str):
    """Open one build of the oracle and declare its entry points."""
    L = ctypes.CDLL(path)
    vp, i32, i64, u64, u32, dbl = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64,
                                   ctypes.c_uint32, ctypes.c_double)
    L.oc_sm64.restype = u64
    L.oc_sm64.argtypes = [u64]
    L.oc_composite.restype = None
    L.oc_composite.argtypes = [i32, vp, dbl, vp, vp, vp, vp, vp, vp]
    L.oc_draw.restype = u64
    L.oc_draw.argtypes = [u64, u64, u64, u64, u64]
    L.oc_sample_rays.restype = None
    L.oc_sample_rays.argtypes = [vp, vp, u64, u32, i32] + [vp] * 8
    L.oc_sample_smooth.restype = None
    L.oc_sample_smooth.argtypes = [vp, vp, u64, u32, i32, vp, vp, vp, vp]
    L.oc_step.restype = i32
    L.oc_step.argtypes = [vp, vp, i32, i32] + [vp] * 6 + [i32] + [vp] * 12
    L.oc_prop_forward.restype = None
    L.oc_prop_forward.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    L.oc_prop_ce.restype = dbl
    L.oc_prop_ce.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp]
    L.oc_prop_sample.restype = None
    L.oc_prop_sample.argtypes = [vp, i32, i32, i32, vp, vp, ctypes.c_uint64, ctypes.c_uint32, vp, vp, vp]
    L.oc_query_sdf.restype = None
    L.oc_query_sdf.argtypes = [vp, vp, vp, i32, vp, vp]
    L.oc_query_sdf_backward.restype = None
    L.oc_eikonal_pose_grad.restype = None
    L.oc_eikonal_pose_grad.argtypes = [vp, vp, vp, vp, vp, i32, i32] + [vp] * 5 + [dbl, vp]
    L.oc_hidden_at.restype = None
    L.oc_hidden_at.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp, vp, vp]
    L.oc_query_sdf_backward.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    L.oc_eikonal.restype = i64
    L.oc_eikonal.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, dbl, vp, vp, vp]
    L.oc_sample_importance.restype = i32
    L.oc_sample_importance.argtypes = [vp, vp, vp, u64, u32, i32, i32, i32, i32] + [vp] * 9
    L.oc_extract_mesh.restype = i64
    L.oc_extract_mesh.argtypes = [vp, vp, vp, ctypes.c_float, i32, i32, i32, dbl, vp, i64, vp]
    L.oc_step_dz.restype = i32
    L.oc_step_dz.argtypes = [vp, vp, i32, i32] + [vp] * 6 + [i32] + [vp] * 7
    L.oc_pose_apply.restype = None
    L.oc_pose_apply.argtypes = [vp, vp, i32, vp]
    L.oc_rays_of_pixels.restype = None
    L.oc_rays_of_pixels.argtypes = [vp, vp, i32, vp, vp]
    L.oc_pose_grad.restype = None
    L.oc_pose_grad.argtypes = [vp, vp, vp, vp, vp, i32, i32] + [vp] * 6
    L.oc_voxel_index.restype = None
    L.oc_voxel_index.argtypes = [vp, vp, i32, vp]
    L.oc_trilinear_coeffs.restype = None
    L.oc_trilinear_coeffs.argtypes = [vp, vp, vp]
    L.oc_trilinear_hessian.restype = None
    L.oc_trilinear_hessian.argtypes = [vp, vp, vp]
    L.oc_adam.restype = None
    L.oc_adam.argtypes = [vp, vp, vp, vp, i64, i64, i32, dbl, dbl, dbl, dbl, dbl]
    L.oc_num_threads.restype = i32
    L.oc_paper_param_count.restype = i64
    L.oc_paper_param_count.argtypes = [vp, vp]
    L.oc_step_paper.restype = i32
    L.oc_step_paper.argtypes = [vp, vp, i32, i32] + [vp] * 6 + [i32] + [vp] * 12
    L.oc_step_paper_dz.restype = i32
    L.oc_step_paper_dz.argtypes = [vp, vp, i32, i32] + [vp] * 6 + [i32] + [vp] * 7
    L.oc_pose_grad_paper.restype = None
    L.oc_pose_grad_paper.argtypes = [vp, vp, vp, vp, vp, i32, i32] + [vp] * 6
    return L


def build_variant(replacements, tag: str) -> str:
    """Compile a copy of the oracle with textual replacements [(old, new), ...] applied, for
    tests that plant a mistake in the oracle and check that a pin catches it.  Each `old`
    must occur exactly once in the source.  Returns the library's path."""
    import hashlib
    src = open(os.path.join(_HERE, "gosurf_oracle.c")).read()
    for old, new in replacements:
        assert src.count(old) == 1, old
        src = src.replace(old, new)
    key = hashlib.sha256(src.encode()).hexdigest()[:16]
    d = os.path.join(_BUILD, "variants")
    os.makedirs(d, exist_ok=True)
    so = os.path.join(d, f"liboracle_{tag}_{key}.so")
    if not os.path.exists(so):
        c = os.path.join(d, f"oracle_{tag}_{key}.c")
        with open(c, "w") as f:
            f.write(src)
        tmp = so + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                               "-fno-fast-math", c, "-o", tmp, "-lm"])
        os.replace(tmp, so)
    return so


class using_variant:
    """Context manager: every oracle call inside uses the library at `path`."""

    def __init__(self, path: str):
        self.path = path

    def __enter__(self):
        global _LIB
        lib()
        with _LOCK:
            self.saved = _LIB
            _LIB = _load(self.path)
        return self

    def __exit__(self, *exc):
        global _LIB
        with _LOCK:
            _LIB = self.saved
        return False


def make_config(w) -> OcConfig:
    """Oracle configuration from a scenegen.Workload."""
    c = OcConfig()
    for l, d in enumerate(w.dims):
        for a in range(3):
            c.dims[l][a] = d[a]
        c.voxel[l] = w.voxels[l]
    c.origin[:] = list(w.extent_min)
    c.n_strat, c.n_guided = w.n_strat, w.n_guided
    c.near_m, c.far_m, c.guide_half, c.trunc, c.kappa_fs = w.near, w.far, w.guide_half, w.trunc, w.kappa_fs
    c.lam[:] = list(w.lambdas)
    c.n_smooth, c.delta_s = w.n_smooth, w.delta_s
    c.arch = 1 if getattr(w, "arch", "compact") == "paper" else 0
    return c


class OcFramesHolder:
    """Keeps the numpy arrays alive next to the ctypes struct that points at them."""

    def __init__(self, frames, c2w=None):
        self.rgb = np.ascontiguousarray(frames.rgb, dtype=np.uint8)
        self.depth = np.ascontiguousarray(frames.depth, dtype=np.float32)
        self.c2w = np.ascontiguousarray(frames.c2w if c2w is None else c2w, dtype=np.float32)
        F, H, W = self.depth.shape
        self.s = OcFrames(F, H, W, self.rgb.ctypes.data, self.depth.ctypes.data, self.c2w.ctypes.data,
                          frames.fx, frames.fy, frames.cx, frames.cy)


def sm64(x: int) -> int:
    return int(lib().oc_sm64(x))


def composite(phi, s, d):
    """NeuS compositing of one ray: returns alpha, T, w, d_hat, wsum."""
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float32)
    N = len(phi)
    alpha, T, w = np.empty(N), np.empty(N), np.empty(N)
    dh, ws = np.empty(1), np.empty(1)
    lib().oc_composite(N, _p(phi), s, _p(d), _p(alpha), _p(T), _p(w), _p(dh), _p(ws))
    return alpha, T, w, float(dh[0]), float(ws[0])


def draw(seed, stream, step, index, slot) -> int:
    return int(lib().oc_draw(seed, stream, step, index, slot))


def sample_rays(cfg: OcConfig, frames: OcFramesHolder, seed: int, step: int, R: int) -> dict:
    N = cfg.n_strat + cfg.n_guided
    out = dict(pix=np.empty(R, np.int64), o=np.empty((R, 3), np.float32), r=np.empty((R, 3), np.float32),
               rgb=np.empty((R, 3), np.float32), D=np.empty(R, np.float32), t=np.empty((R, N), np.float32),
               cls=np.empty((R, N), np.uint8), counts=np.empty(4, np.int64))
    lib().oc_sample_rays(ctypes.byref(cfg), ctypes.byref(frames.s), seed, step, R, *[_p(out[k]) for k in
                                                                                     ("pix", "o", "r", "rgb", "D", "t",
                                                                                      "cls", "counts")])
    return out


def sample_importance(cfg: OcConfig, frames: OcFramesHolder, theta, seed: int, step: int, R: int, n_coarse: int,
                      n_steps: int, per_step: int) -> dict:
    """Hierarchical importance sampling (N_c coarse + n_steps x per_step): the rays of
    sample_rays for (seed, step) with N = n_coarse + n_steps * per_step depths; phi [R][N]."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    N = n_coarse + n_steps * per_step
    out = dict(pix=np.empty(R, np.int64), o=np.empty((R, 3), np.float32), r=np.empty((R, 3), np.float32),
               rgb=np.empty((R, 3), np.float32), D=np.empty(R, np.float32), t=np.empty((R, N), np.float32),
               cls=np.empty((R, N), np.uint8), counts=np.empty(4, np.int64), phi=np.empty((R, N)))
    rc = lib().oc_sample_importance(ctypes.byref(cfg), ctypes.byref(frames.s), _p(th), seed, step, R, n_coarse,
                                    n_steps, per_step, *[_p(out[k]) for k in ("pix", "o", "r", "rgb", "D", "t", "cls",
                                                                              "counts", "phi")])
    if rc != 0:
        raise ValueError("oc_sample_importance rejected its arguments")
    return out


def sample_smooth(cfg: OcConfig, frames: OcFramesHolder, seed: int, step: int, P: int) -> dict:
    out = dict(xs=np.empty((P, 3), np.float32), eps=np.empty((P, 3), np.float32), valid=np.empty(P, np.uint8),
               n_valid=np.empty(1, np.int64))
    lib().oc_sample_smooth(ctypes.byref(cfg), ctypes.byref(frames.s), seed, step, P,
                           *[_p(out[k]) for k in ("xs", "eps", "valid", "n_valid")])
    return out


def step_dz(cfg: OcConfig, theta, batch: dict, smooth: dict | None, dloss=None):
    """Losses, gradient and dL/dz of every main sample of one step: [R][N][16] for the
    workload's model; for the paper's architecture (cfg.arch == 1) [R][N][32] holding dL/dz
    (16), dL/dW_beta(x) (6), dL/d(viewing direction) (3) and zeros."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    R, N = batch["t"].shape
    if smooth is None:
        P, xs, eps, valid = 0, np.zeros((1, 3), np.float32), np.zeros((1, 3), np.float32), np.zeros(1, np.uint8)
    else:
        P, xs, eps, valid = len(smooth["valid"]), smooth["xs"], smooth["eps"], smooth["valid"]
    loss, grad, dz = np.zeros(6), np.zeros_like(th), np.zeros((R, N, 32 if cfg.arch == 1 else 16))
    dl = None if dloss is None else np.ascontiguousarray(dloss, dtype=np.float64)
    rc = (lib().oc_step_paper_dz if cfg.arch == 1 else lib().oc_step_dz)(ctypes.byref(cfg), _p(th), R, N, _p(batch["o"]), _p(batch["r"]), _p(batch["rgb"]),
                          _p(batch["D"]), _p(batch["t"]), _p(batch["cls"]), P, _p(xs), _p(eps), _p(valid), _p(dl),
                          _p(loss), _p(grad), _p(dz))
    if rc != 0:
        raise ValueError("oc_step_dz rejected its arguments")
    return dict(loss=loss, grad=grad, dz=dz)


def pose_apply(c2w0, xi) -> np.ndarray:
    """Refined camera-to-world [F][3][4] (FP64): R0 Exp(nu), t0 + dt for xi [F][6] = (dt, nu)."""
    c2w0 = np.ascontiguousarray(c2w0, dtype=np.float32).reshape(-1, 3, 4)
    xi = np.ascontiguousarray(xi, dtype=np.float64).reshape(len(c2w0), 6)
    out = np.empty((len(c2w0), 3, 4))
    lib().oc_pose_apply(_p(c2w0), _p(xi), len(c2w0), _p(out))
    return out


def rays_of_pixels(frames: OcFramesHolder, pix):
    pix = np.ascontiguousarray(pix, dtype=np.int64)
    o, r = np.empty((len(pix), 3), np.float32), np.empty((len(pix), 3), np.float32)
    lib().oc_rays_of_pixels(ctypes.byref(frames.s), _p(pix), len(pix), _p(o), _p(r))
    return o, r


def pose_grad(cfg: OcConfig, frames: OcFramesHolder, theta, c2w, xi, batch: dict, dz) -> np.ndarray:
    """dL/dxi [F][6] of the rays of batch (pix, o, r, t) from the step's dL/dz [R][N][16]."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    c2w = np.ascontiguousarray(c2w, dtype=np.float64)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    F = len(c2w)
    R, N = batch["t"].shape
    g = np.zeros((F, 6))
    (lib().oc_pose_grad_paper if cfg.arch == 1 else lib().oc_pose_grad)(ctypes.byref(cfg), ctypes.byref(frames.s), _p(th), _p(c2w), _p(xi), R, N,
                       _p(np.ascontiguousarray(batch["pix"], dtype=np.int64)), _p(batch["o"]), _p(batch["r"]),
                       _p(batch["t"]), _p(np.ascontiguousarray(dz, dtype=np.float64)), _p(g))
    return g


def eikonal_pose_grad(cfg: OcConfig, frames: OcFramesHolder, theta, c2w, xi, batch: dict, dscale: float = 1.0):
    """dscale * dL_eik/dxi [F][6]: the Eikonal term's pose gradient through the free-space
    samples' positions (x-Hessian of phi), for either architecture."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    c2w = np.ascontiguousarray(c2w, dtype=np.float64)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    F = len(c2w)
    R, N = batch["t"].shape
    g = np.zeros((F, 6))
    lib().oc_eikonal_pose_grad(ctypes.byref(cfg), ctypes.byref(frames.s), _p(th), _p(c2w), _p(xi), R, N,
                               _p(np.ascontiguousarray(batch["pix"], dtype=np.int64)), _p(batch["o"]),
                               _p(batch["r"]), _p(batch["t"]), _p(np.ascontiguousarray(batch["cls"], np.uint8)),
                               ctypes.c_double(dscale), _p(g))
    return g


def paper_param_count(cfg: OcConfig) -> tuple[int, int]:
    """(total floats, grid floats) of the flat vector of the paper's architecture."""
    ng = np.zeros(1, np.int64)
    n = lib().oc_paper_param_count(ctypes.byref(cfg), _p(ng))
    return int(n), int(ng[0])


def step(cfg: OcConfig, theta, batch: dict, smooth: dict | None, dloss=None, want_grad=True, want_margins=False,
         want_weights=False):
    """Losses (and gradients) of one step.  theta: flat parameters (promoted to FP64).
    cfg.arch selects the decoders: 0 the workload's (oc_step), 1 the paper's (oc_step_paper)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    R, N = batch["t"].shape
    if smooth is None:
        P = 0
        xs = eps = np.zeros((1, 3), np.float32)
        valid = np.zeros(1, np.uint8)
    else:
        P = len(smooth["valid"])
        xs, eps, valid = smooth["xs"], smooth["eps"], smooth["valid"]
    loss = np.zeros(6)
    rgb_hat, d_hat, wsum = np.zeros((R, 3)), np.zeros(R), np.zeros(R)
    grad = np.zeros_like(th) if want_grad else None
    margins = np.zeros(10) if want_margins else None
    amb = np.zeros((R, N), np.uint8) if want_margins else None
    dl = None if dloss is None else np.ascontiguousarray(dloss, dtype=np.float64)
    w = np.zeros((R, N)) if want_weights else None
    fn = lib().oc_step_paper if cfg.arch == 1 else lib().oc_step
    rc = fn(ctypes.byref(cfg), _p(th), R, N, _p(batch["o"]), _p(batch["r"]), _p(batch["rgb"]),
                       _p(batch["D"]), _p(batch["t"]), _p(batch["cls"]), P, _p(xs), _p(eps), _p(valid), _p(dl),
                       _p(loss), _p(rgb_hat), _p(d_hat), _p(wsum), _p(grad), _p(margins), _p(amb), _p(w))
    if rc != 0:
        raise ValueError("oc_step rejected its arguments")
    return dict(loss=loss, rgb_hat=rgb_hat, d_hat=d_hat, wsum=wsum, grad=grad, margins=margins, amb=amb, w=w)


# ---- learned proposal sampler (a sample-count reduction; not part of the paper) ----
PROP_BINS = 32
PROP_PARAMS = 32 * 11 + 32 + 32 * 32 + 32 + 32 + 1  # 1473


def prop_forward(cfg: OcConfig, theta, q, o, r) -> np.ndarray:
    """Proposal distribution p [R][32] (FP64)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    qq = np.ascontiguousarray(q, dtype=np.float64)
    o = np.ascontiguousarray(o, dtype=np.float32).reshape(-1, 3)
    r = np.ascontiguousarray(r, dtype=np.float32).reshape(-1, 3)
    p = np.empty((len(o), PROP_BINS))
    lib().oc_prop_forward(ctypes.byref(cfg), _p(th), _p(qq), len(o), _p(o), _p(r), _p(p))
    return p


def prop_ce(cfg: OcConfig, theta, q, o, r, t, w, want_grad=True):
    """Cross-entropy training loss of the proposal against the binned weights w [R][N]
    at depths t [R][N]; returns (loss, gradient w.r.t. q or None, rays used)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    qq = np.ascontiguousarray(q, dtype=np.float64)
    o = np.ascontiguousarray(o, dtype=np.float32).reshape(-1, 3)
    r = np.ascontiguousarray(r, dtype=np.float32).reshape(-1, 3)
    t = np.ascontiguousarray(t, dtype=np.float32)
    w = np.ascontiguousarray(w, dtype=np.float64)
    R, N = t.shape
    g = np.zeros(PROP_PARAMS) if want_grad else None
    n = np.zeros(1, np.int64)
    ce = lib().oc_prop_ce(ctypes.byref(cfg), _p(th), _p(qq), R, N, _p(o), _p(r), _p(t), _p(w), _p(g), _p(n))
    return ce, g, int(n[0])


def prop_sample(cfg: OcConfig, D, p, N: int, n_guided: int, seed: int, step: int) -> dict:
    """Depths drawn from the proposal p [R][32] (binary32, bit-exact), sorted, with classes."""
    D = np.ascontiguousarray(D, dtype=np.float32)
    p = np.ascontiguousarray(p, dtype=np.float32)
    R = len(D)
    t = np.empty((R, N), np.float32)
    cls = np.empty((R, N), np.uint8)
    counts = np.zeros(4, np.int64)
    lib().oc_prop_sample(ctypes.byref(cfg), R, N, n_guided, _p(D), _p(p), seed, step, _p(t), _p(cls), _p(counts))
    return dict(t=t, cls=cls, counts=counts)


def query_sdf(cfg: OcConfig, theta, x, want_grad=True):
    th = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3)
    sdf = np.empty(len(x))
    grad = np.empty((len(x), 3)) if want_grad else None
    lib().oc_query_sdf(ctypes.byref(cfg), _p(th), _p(x), len(x), _p(sdf), _p(grad))
    return sdf, grad


def hidden_at(cfg: OcConfig, theta, x, d=None):
    """Hidden pre-activations at points (diagnostic): (kink [P], [h1, h2, ...] each [P][32]).
    kink is the smallest distance of any evaluated hidden unit from its ReLU kink relative to
    the magnitude of its terms.  Workload decoders: the geometry and the colour decoder's
    hidden layer.  Paper architecture: the geometry decoder's two layers, and with unit
    viewing directions d [P][3] also the colour decoder's two."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3)
    P = len(x)
    dd = None if d is None else np.ascontiguousarray(d, dtype=np.float64).reshape(P, 3)
    kink = np.empty(P)
    hs = [np.empty((P, 32)) for _ in range(4)]
    lib().oc_hidden_at(ctypes.byref(cfg), _p(th), _p(x), _p(dd), P, _p(kink), *[_p(h) for h in hs])
    n = 4 if (cfg.arch == 1 and dd is not None) else 2
    return kink, hs[:n]


# relative distance below which the oracle flags a hidden unit as possibly decided
# differently by binary32 arithmetic (amb bit 3; OC_KINK_REL in the C source)
KINK_REL = 1e-5


def query_sdf_backward(cfg: OcConfig, theta, x, dsdf=None, dgrad=None) -> np.ndarray:
    """d/dtheta of sum_i dsdf_i phi(x_i) + dgrad_i . grad_x phi(x_i) (flat, FP64)."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3)
    ds = None if dsdf is None else np.ascontiguousarray(dsdf, dtype=np.float64).reshape(len(x))
    dg = None if dgrad is None else np.ascontiguousarray(dgrad, dtype=np.float64).reshape(len(x), 3)
    grad = np.zeros(len(th))
    lib().oc_query_sdf_backward(ctypes.byref(cfg), _p(th), _p(x), len(x), _p(ds), _p(dg), _p(grad))
    return grad


def eikonal(cfg: OcConfig, theta, batch: dict, dscale: float = 1.0, want_grad=True):
    """Eikonal term over the batch's free-space samples: (L_eik, dscale * dL_eik/dtheta or
    None, |S_fs|, |grad_x phi| per sample [R][N] (-1 outside S_fs))."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    t = np.ascontiguousarray(batch["t"], dtype=np.float32)
    R, N = t.shape
    o = np.ascontiguousarray(batch["o"], dtype=np.float32).reshape(R, 3)
    r = np.ascontiguousarray(batch["r"], dtype=np.float32).reshape(R, 3)
    cls = np.ascontiguousarray(batch["cls"], dtype=np.uint8).reshape(R, N)
    loss = np.zeros(1)
    grad = np.zeros(len(th)) if want_grad else None
    gnorm = np.empty((R, N))
    n = lib().oc_eikonal(ctypes.byref(cfg), _p(th), R, N, _p(o), _p(r), _p(t), _p(cls), ctypes.c_double(dscale),
                         _p(loss), _p(grad), _p(gnorm))
    if n < 0:
        raise ValueError("oc_eikonal rejected its arguments")
    return float(loss[0]), grad, int(n), gnorm


def extract_mesh(cfg: OcConfig, theta, lo, step: float, dims, iso: float = 0.0, max_tris: int | None = None):
    """Isosurface phi = iso on the lattice lo + (i, j, k) * step, dims = (nx, ny, nz): returns
    (triangles [T][3][3] FP64, lattice phi [nz][ny][nx])."""
    th = np.ascontiguousarray(theta, dtype=np.float64)
    lo = np.ascontiguousarray(lo, dtype=np.float32).reshape(3)
    nx, ny, nz = (int(d) for d in dims)
    phi = np.empty((nz, ny, nx))
    cap = max_tris if max_tris is not None else 12 * (nx - 1) * (ny - 1) * (nz - 1)
    tris = np.empty((max(cap, 1), 3, 3))
    n = lib().oc_extract_mesh(ctypes.byref(cfg), _p(th), _p(lo), ctypes.c_float(step), nx, ny, nz,
                              ctypes.c_double(iso), _p(tris), cap, _p(phi))
    return tris[:min(n, cap)], phi


def voxel_index(cfg: OcConfig, x) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, 3)
    out = np.empty((len(x), LEVELS), np.int64)
    lib().oc_voxel_index(ctypes.byref(cfg), _p(x), len(x), _p(out))
    return out


def trilinear_coeffs(f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    w, J = np.empty(8), np.empty((8, 3))
    lib().oc_trilinear_coeffs(_p(f), _p(w), _p(J))
    return w, J


def trilinear_hessian(theta8, f):
    th = np.ascontiguousarray(theta8, dtype=np.float64)
    f = np.ascontiguousarray(f, dtype=np.float64)
    h = np.empty(3)
    lib().oc_trilinear_hessian(_p(th), _p(f), _p(h))
    return h  # h12, h13, h23


def adam(p, g, m, v, n_grid, t, lr_grid, lr_mlp, b1=0.9, b2=0.999, eps=1e-8):
    """In-place FP64 Adam on float64 arrays (g is zeroed)."""
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().oc_adam(_p(p), _p(g), _p(m), _p(v), len(p), n_grid, t, lr_grid, lr_mlp, b1, b2, eps)


def num_threads() -> int:
    return int(lib().oc_num_threads())
