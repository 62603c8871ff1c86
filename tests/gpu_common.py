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


def prepare_parity_batch(p: Problem, theta, bt, sm, max_iter=6, max_drop=0.1):
    """Subset of the oracle batch on which no branch decision lies within binary32 rounding
    of a tie, so that the FP32 kernels and the FP64 oracle take every branch the same way.

    The oracle flags the samples whose alpha > 0 decision (when a flip would move dL/dphi by
    more than 1e-7), truncated-SDF sign or free-space maximum is that close to a tie; the rays
    holding them are left out and both sides run on the remaining rays.  Returns (batch,
    reference step, number of rays left out)."""
    keep = np.ones(len(bt["D"]), bool)
    for _ in range(max_iter):
        sub = {k: (v[keep] if k != "counts" else v) for k, v in bt.items()}
        sub["counts"] = np.array([(sub["D"] > 0).sum(), (sub["cls"] == 1).sum(), (sub["cls"] == 2).sum(), 0],
                                 np.int64)
        ref = oc.step(p.cfg, theta, sub, sm, want_margins=True)
        bad = ref["amb"].any(axis=1)
        if not bad.any():
            dropped = int((~keep).sum())
            assert dropped <= max_drop * len(keep), dropped
            return sub, ref, dropped
        keep[np.nonzero(keep)[0][bad]] = False
    raise AssertionError("could not move the parity batch away from binary32 ties")


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
