"""Shared set-up of the GPU parity tests: run the CUDA path through the C ABI and the FP64
oracle on the same seeded inputs, and compare."""
from __future__ import annotations

import numpy as np
import torch

import oracle as oc
import paper_2206_14735_gb300 as gs
import scenegen as sg

LOSS_RTOL = 1e-5      # relative error per loss term
GRAD_TOL = 1e-4       # max |g - g_ref| / max |g_ref| per parameter tensor
GRAD_ELEM_RTOL = 1e-3  # element-wise, where |g_ref| > 1e-2 max |g_ref|


def ensure_built():
    from paper_2206_14735_gb300 import build as b
    b.build()


class Problem:
    """One workload on both sides: device frames + context, oracle frames + config."""

    def __init__(self, w, n_frames=None, max_rays=None):
        ensure_built()
        self.w = w
        self.frames = sg.make_frames(w, n_frames=n_frames)
        self.cfg = oc.make_config(w)
        self.ofr = oc.OcFramesHolder(self.frames)
        self.ctx = gs.Context(w, max_rays=max_rays)
        f = self.frames
        self.dfr = gs.DeviceFrames(f.rgb, f.depth, f.c2w, f.fx, f.fy, f.cx, f.cy)
        self.offs, self.n_grid, self.n_tot = w.layout()

    def gpu_sample(self, seed, step, R=None, P=None):
        R = self.w.rays if R is None else R
        P = self.w.n_smooth if P is None else P
        b = gs.Batch.allocate(R, self.w.n_samples, P)
        self.ctx.sample_rays(self.dfr, seed, step, b)
        torch.cuda.synchronize()
        return b

    def oracle_sample(self, seed, step, R=None, P=None):
        R = self.w.rays if R is None else R
        P = self.w.n_smooth if P is None else P
        bt = oc.sample_rays(self.cfg, self.ofr, seed, step, R)
        sm = oc.sample_smooth(self.cfg, self.ofr, seed, step, P) if P > 0 else None
        return bt, sm

    def split_grad(self, g):
        """Flat parameter-shaped vector -> named tensors."""
        out = {}
        for l in range(4):
            nx, ny, nz = self.w.dims[l]
            out[f"grid{l}"] = g[self.offs[l]:self.offs[l] + nx * ny * nz * 4]
        if self.w.arch == "paper":
            out["colour_grid"] = g[self.w.colour_offset():self.n_grid]
        o = self.n_grid
        for name, shape in self.w.mlp_shapes:
            n = int(np.prod(shape))
            out[name] = g[o:o + n]
            o += n
        return out


def sample_positions(bt):
    """x = o + t r in binary32, as both sides compute it."""
    t = bt["t"].astype(np.float32)
    return (bt["o"][:, None, :] + (t[..., None] * bt["r"][:, None, :]).astype(np.float32)).astype(np.float32)


def _classes(D, t, trunc):
    """Sample classes by the bound b = D - t (binary32), as the sampler assigns them."""
    b = (D[:, None] - t).astype(np.float32)
    tr = np.float32(trunc)
    return np.where(D[:, None] > 0, np.where(np.abs(b) <= tr, 1, np.where(b > tr, 2, 0)), 0).astype(np.uint8)


def unit_directions(bt):
    """Unit viewing direction of every sample [R*N][3] (the paper architecture's colour input)."""
    r = bt["r"].astype(np.float64)
    d = r / np.linalg.norm(r, axis=1, keepdims=True)
    return np.repeat(d, bt["t"].shape[1], axis=0)


def switching_fraction(p: Problem, theta, bt):
    """Fraction of the hidden ReLU units (every hidden layer of both decoders) that are on at
    some samples of the batch and off at others."""
    x = sample_positions(bt).reshape(-1, 3)
    d = unit_directions(bt) if p.w.arch == "paper" else None
    _, hs = oc.hidden_at(p.cfg, theta, x, d)
    on = np.concatenate([h > 0 for h in hs], axis=1)
    return float((on.any(axis=0) & (~on).any(axis=0)).mean())


def drop_kink_points(p: Problem, theta, sm):
    """Smoothness points whose gradient grad_x phi at x or x + eps has a hidden unit within
    binary32 rounding of its kink (the loss itself jumps there) are made inactive, in place:
    sm["valid"] and sm["n_valid"] are rewritten.  Returns how many were dropped."""
    if sm is None or len(sm["valid"]) == 0:
        return 0
    xe = (sm["xs"] + sm["eps"]).astype(np.float32)
    k0, _ = oc.hidden_at(p.cfg, theta, sm["xs"])
    k1, _ = oc.hidden_at(p.cfg, theta, xe)
    bad = (sm["valid"] > 0) & ((k0 < oc.KINK_REL) | (k1 < oc.KINK_REL))
    sm["valid"] = np.where(bad, 0, sm["valid"]).astype(np.uint8)
    sm["n_valid"] = np.array([int((sm["valid"] > 0).sum())], dtype=sm["n_valid"].dtype)
    return int(bad.sum())


def prepare_parity_batch(p: Problem, theta, bt, sm, max_iter=6, max_drop=0.1, min_switch=None, label=""):
    """Subset of the oracle batch on which no branch decision lies within binary32 rounding
    of a tie, so that the FP32 kernels and the FP64 oracle take every branch the same way.

    The oracle flags the samples whose alpha > 0 decision (when a flip would move dL/dphi by
    more than 1e-7), truncated-SDF sign, free-space maximum or hidden ReLU unit (when a flip
    would move the sample's gradient by more than 1e-9), and the rays whose sign of
    d_hat - D, is that close to a tie; the rays
    holding them are left out and both sides run on the remaining rays.  Smoothness points
    near a ReLU kink are made inactive in sm (in place).  With min_switch, asserts that at
    least that fraction of the hidden units switches within the batch.  Prints and bounds
    (max_drop) the rays left out.  Returns (batch, reference step, number of rays left out)."""
    if min_switch is not None:
        frac = switching_fraction(p, theta, bt)
        assert frac >= min_switch, frac
    n_pts = drop_kink_points(p, theta, sm)
    keep = np.ones(len(bt["D"]), bool)
    for _ in range(max_iter):
        sub = {k: (v[keep] if k != "counts" else v) for k, v in bt.items()}
        sub["counts"] = np.array([(sub["D"] > 0).sum(), (sub["cls"] == 1).sum(), (sub["cls"] == 2).sum(), 0],
                                 np.int64)
        ref = oc.step(p.cfg, theta, sub, sm, want_margins=True)
        bad = ref["amb"].any(axis=1)
        if not bad.any():
            dropped = int((~keep).sum())
            print(f"parity batch {label or p.w.name}: {dropped} of {len(keep)} rays "
                  f"({100.0 * dropped / max(len(keep), 1):.2f} %) and {n_pts} smoothness points left out"
                  + (f"; {100.0 * frac:.0f} % of hidden units switch" if min_switch is not None else ""))
            assert dropped <= max_drop * len(keep), (dropped, len(keep))
            return sub, ref, dropped
        keep[np.nonzero(keep)[0][bad]] = False
    raise AssertionError("could not move the parity batch away from binary32 ties")


def drop_kink_rays(p: Problem, theta, bt, classes=(oc.CLS_FS,)):
    """Rays none of whose samples of the given classes has a hidden unit within binary32
    rounding of its kink (for terms built on grad_x phi, which jumps there).  Returns the
    ray subset (counts recomputed) and the number of rays left out."""
    x = sample_positions(bt).reshape(-1, 3)
    kink, _ = oc.hidden_at(p.cfg, theta, x)
    near = (kink < oc.KINK_REL).reshape(bt["t"].shape) & np.isin(bt["cls"], classes)
    keep = ~near.any(axis=1)
    sub = {k: (v[keep] if k != "counts" else v) for k, v in bt.items()}
    sub["counts"] = np.array([(sub["D"] > 0).sum(), (sub["cls"] == 1).sum(), (sub["cls"] == 2).sum(), 0], np.int64)
    return sub, int((~keep).sum())


def far_from_kinks(p: Problem, theta, x):
    """Mask of the points x whose hidden units are all clear of their kinks in binary32."""
    kink, _ = oc.hidden_at(p.cfg, theta, x)
    return kink >= oc.KINK_REL


def upload_oracle_batch(bt, sm, counts_smooth, device="cuda"):
    """Device batch holding exactly the oracle's sampled inputs (for tests that modify them)."""
    R, N = bt["t"].shape
    P = 0 if sm is None else len(sm["valid"])
    b = gs.Batch.allocate(R, N, P, device=device)
    b.pix.copy_(torch.from_numpy(bt["pix"]))
    b.origin.copy_(torch.from_numpy(bt["o"]))
    b.dir.copy_(torch.from_numpy(bt["r"]))
    b.rgb.copy_(torch.from_numpy(bt["rgb"]))
    b.depth.copy_(torch.from_numpy(bt["D"]))
    b.t.copy_(torch.from_numpy(bt["t"]))
    b.cls.copy_(torch.from_numpy(bt["cls"]))
    if P > 0:
        b.xs[:P].copy_(torch.from_numpy(sm["xs"]))
        b.eps[:P].copy_(torch.from_numpy(sm["eps"]))
        b.valid[:P].copy_(torch.from_numpy(sm["valid"]))
    c = bt["counts"]
    b.counts.copy_(torch.tensor([int(c[0]), int(c[1]), int(c[2]), int(counts_smooth)], dtype=torch.int32))
    return b


def assert_grad_close(p: Problem, g_gpu, g_ref, tol=GRAD_TOL, elem_rtol=GRAD_ELEM_RTOL, skip=()):
    A, B = p.split_grad(np.asarray(g_gpu, np.float64)), p.split_grad(np.asarray(g_ref, np.float64))
    report = {}
    for k in A:
        if k in skip:
            continue
        ref, got = B[k], A[k]
        scale = np.abs(ref).max()
        if scale == 0:
            assert np.abs(got).max() == 0, k
            continue
        err = np.abs(got - ref).max() / scale
        big = np.abs(ref) > 1e-2 * scale
        rel = (np.abs(got - ref)[big] / np.abs(ref[big])).max() if big.any() else 0.0
        report[k] = (err, rel)
        assert err <= tol and rel <= elem_rtol, (k, err, rel, report)
    return report


def _surface_through(w, theta, x, bias_name):
    """theta with the SDF's output bias shifted so that phi(x) = 0: a surface through x, so
    that rays crossing x carry real opacity there (far from the scene's surface they are
    nearly transparent and every colour gradient is rounding noise)."""
    cfg = oc.make_config(w)
    s0 = oc.query_sdf(cfg, theta, np.asarray(x, np.float32)[None, :], want_grad=False)
    s0 = float(np.asarray(s0[0] if isinstance(s0, tuple) else s0).ravel()[0])
    o = w.layout()[1]
    for name, shape in w.mlp_shapes:
        if name == bias_name:
            break
        o += int(np.prod(shape))
    th = theta.copy()
    th[o] -= np.float32(s0)
    return th


def corner_case(p: Problem, theta, bias_name, corner, seed, step, R=256, max_drop=0.2):
    """Rays moved so that their samples cross a corner of the grid (the middle sample a quarter
    of a finest voxel inside it, the rest partly outside and clamped into the boundary cells),
    with the surface through that point; returns (theta, batch subset, oracle step)."""
    w = p.w
    bt, _ = p.oracle_sample(seed, step, R, 0)
    lo = np.array(w.extent_min, np.float64)
    hi = lo + (np.array(w.dims[3], np.float64) - 1) * w.voxels[3]
    target = hi - 0.25 * w.voxels[3] if corner == "max" else lo + 0.25 * w.voxels[3]
    theta = _surface_through(w, theta, target, bias_name)
    t_mid = np.median(bt["t"], axis=1)
    bt = dict(bt)
    bt["o"] = (target[None, :] - t_mid[:, None] * bt["r"].astype(np.float64)).astype(np.float32)
    bt_s, ref, _ = prepare_parity_batch(p, theta, bt, None, max_drop=max_drop, label=f"{w.name}, {corner} corner")
    x = sample_positions(bt_s).reshape(-1, 3)
    outside = ((x > hi[None, :]) | (x < lo[None, :])).any(axis=1)
    assert outside.mean() > 0.2 and (~outside).mean() > 0.05, outside.mean()
    assert ref["rgb_hat"].max() > 0.1  # the rays render something: the colour path is conditioned
    return theta, bt_s, ref
