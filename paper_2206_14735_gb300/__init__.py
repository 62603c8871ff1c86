"""GB300-native GO-Surf optimisation step (arXiv 2206.14735): Python binding.

The computation lives in ``libgosurf.so`` (hand-written sm_103a CUDA behind the C ABI of
``include/gosurf.h``).  This package allocates device buffers with PyTorch, passes their
pointers to the library's entry points (same names as the C functions) on the caller's
current CUDA stream, and wraps forward/backward in a ``torch.autograd.Function``.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import torch

from ._lib import (GS_ARCH_COMPACT, GS_ARCH_PAPER, GS_FEAT, GS_LEVELS, GS_MLP_PARAMS, GS_NUM_LOSS,
                   GS_PAPER_MLP_PARAMS, GS_PREC_BF16, GS_PREC_FP32, GS_PROP_BINS, GS_PROP_PARAMS, EXPORTS, GoSurfError,
                   GsBatch, GsConfig, GsFrames, lib, library_path)

__all__ = ["Context", "Batch", "DeviceFrames", "GoSurfStep", "SdfGrad", "GoSurfError", "make_config", "GS_MLP_PARAMS", "GS_NUM_LOSS",
           "GS_PAPER_MLP_PARAMS", "GS_ARCH_COMPACT", "GS_ARCH_PAPER",
           "library_path", "EXPORTS"]


def make_config(workload, max_rays=None, max_smooth=None, store_activations=False) -> GsConfig:
    """gs_config from any object with the workload attributes (dims, voxels, extent_min,
    n_strat, n_guided, near, far, guide_half, trunc, kappa_fs, lambdas, n_smooth, delta_s, rays)."""
    c = GsConfig()
    for l, d in enumerate(workload.dims):
        for a in range(3):
            c.dims[l][a] = int(d[a])
        c.voxel[l] = float(workload.voxels[l])
    c.origin[:] = [float(v) for v in workload.extent_min]
    c.n_strat, c.n_guided = int(workload.n_strat), int(workload.n_guided)
    c.near_m, c.far_m = float(workload.near), float(workload.far)
    c.guide_half, c.trunc, c.kappa_fs = float(workload.guide_half), float(workload.trunc), float(workload.kappa_fs)
    c.lam[:] = [float(v) for v in workload.lambdas]
    c.max_rays = int(max_rays if max_rays is not None else workload.rays)
    c.max_smooth = int(max_smooth if max_smooth is not None else workload.n_smooth)
    c.delta_s = float(workload.delta_s)
    c.precision = GS_PREC_BF16 if getattr(workload, "precision", "fp32") == "bf16" else GS_PREC_FP32
    c.store_activations = 1 if store_activations else 0
    c.prop_samples = int(getattr(workload, "prop_samples", 0))
    c.prop_guided = int(getattr(workload, "prop_guided", 0))
    c.imp_coarse = int(getattr(workload, "imp_coarse", 0))
    c.imp_steps = int(getattr(workload, "imp_steps", 0))
    c.imp_per_step = int(getattr(workload, "imp_per_step", 0))
    c.arch = GS_ARCH_PAPER if getattr(workload, "arch", "compact") == "paper" else GS_ARCH_COMPACT
    return c


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class DeviceFrames:
    """Posed RGB-D frames copied to the device once (they stay resident)."""

    def __init__(self, rgb, depth, c2w, fx, fy, cx, cy, device="cuda"):
        self.rgb = torch.as_tensor(rgb).to(device=device, dtype=torch.uint8).contiguous()
        self.depth = torch.as_tensor(depth).to(device=device, dtype=torch.float32).contiguous()
        self.c2w = torch.as_tensor(c2w).to(device=device, dtype=torch.float32).contiguous()
        F, H, W = self.depth.shape
        self.intr = (fx, fy, cx, cy)
        self.s = GsFrames(F, H, W, self.rgb.data_ptr(), self.depth.data_ptr(), self.c2w.data_ptr(), fx, fy, cx, cy)

    def with_poses(self, c2w) -> "DeviceFrames":
        """The same images with other camera-to-world matrices c2w [F][3][4] (a device tensor that
        the caller keeps alive, e.g. the output of Context.pose_apply)."""
        out = DeviceFrames.__new__(DeviceFrames)
        out.rgb, out.depth, out.c2w, out.intr = self.rgb, self.depth, c2w, self.intr
        F, H, W = self.depth.shape
        out.s = GsFrames(F, H, W, self.rgb.data_ptr(), self.depth.data_ptr(), c2w.data_ptr(), *self.intr)
        return out


@dataclass
class Batch:
    """Device buffers of one ray batch (gs_batch)."""
    R: int
    N: int
    P: int
    pix: torch.Tensor
    origin: torch.Tensor
    dir: torch.Tensor
    rgb: torch.Tensor
    depth: torch.Tensor
    t: torch.Tensor
    cls: torch.Tensor
    xs: torch.Tensor
    eps: torch.Tensor
    valid: torch.Tensor
    counts: torch.Tensor
    w: torch.Tensor | None = None  # [R][N] rendering weights (written by forward passes when present)
    dz: torch.Tensor | None = None  # [R][N][16] dL/dz (written by backward passes when present;
    #                                 [R][N][32] records for the paper's architecture)
    eik: torch.Tensor | None = None  # [5][R][N][4] deferred Eikonal records (written by eikonal(), read by
    #                                  the next backward pass over this batch)

    @staticmethod
    def allocate(R: int, N: int, P: int, device="cuda", weights=False, dz=False, dz_width=16,
                 eik=False) -> "Batch":
        f = dict(device=device, dtype=torch.float32)
        return Batch(R=R, N=N, P=P, pix=torch.empty(R, device=device, dtype=torch.int64),
                     origin=torch.empty(R, 3, **f), dir=torch.empty(R, 3, **f), rgb=torch.empty(R, 3, **f),
                     depth=torch.empty(R, **f), t=torch.empty(R, N, **f),
                     cls=torch.empty(R, N, device=device, dtype=torch.uint8), xs=torch.empty(max(P, 1), 3, **f),
                     eps=torch.empty(max(P, 1), 3, **f), valid=torch.empty(max(P, 1), device=device, dtype=torch.uint8),
                     counts=torch.zeros(4, device=device, dtype=torch.int32),
                     w=torch.zeros(R, N, **f) if weights else None,
                     dz=torch.zeros(R, N, dz_width, **f) if dz else None,
                     eik=torch.zeros(5, R, N, 4, **f) if eik else None)

    def struct(self) -> GsBatch:
        return GsBatch(self.R, self.N, self.P, self.pix.data_ptr(), self.origin.data_ptr(), self.dir.data_ptr(),
                       self.rgb.data_ptr(), self.depth.data_ptr(), self.t.data_ptr(), self.cls.data_ptr(),
                       self.xs.data_ptr(), self.eps.data_ptr(), self.valid.data_ptr(), self.counts.data_ptr(),
                       None if self.w is None else self.w.data_ptr(), None if self.dz is None else self.dz.data_ptr(),
                       None if self.eik is None else self.eik.data_ptr())


class Context:
    """One gs_ctx (workspace sized at creation) on the current CUDA device."""

    def __init__(self, workload, max_rays=None, max_smooth=None, store_activations=False):
        self.L = lib()
        self.cfg = make_config(workload, max_rays, max_smooth, store_activations)
        h = ctypes.c_void_p()
        self._check(self.L.gs_create(ctypes.byref(self.cfg), ctypes.byref(h)), None)
        self.h = h
        ng = ctypes.c_int64()
        self.n_params = int(self.L.gs_param_count(ctypes.byref(self.cfg), ctypes.byref(ng)))
        self.n_grid = int(ng.value)

    def _check(self, st, h=...):
        if st != 0:
            handle = self.h if h is ... else h
            raise GoSurfError(st, self.L.gs_last_error(handle).decode())

    def close(self):
        if getattr(self, "h", None):
            self.L.gs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- entry points (same names as the C ABI, minus the gs_ prefix) ---
    def sample_rays(self, frames: DeviceFrames, seed: int, step: int, batch: Batch):
        b = batch.struct()
        self._check(self.L.gs_sample_rays(self.h, ctypes.byref(frames.s), seed, step, ctypes.byref(b), _stream()))

    def forward(self, theta, batch: Batch, loss, rgb_hat=None, d_hat=None, wsum=None, theta_bf16=None):
        b = batch.struct()
        self._check(self.L.gs_forward(self.h, _ptr(theta), _ptr(theta_bf16), ctypes.byref(b), _ptr(loss),
                                      _ptr(rgb_hat), _ptr(d_hat), _ptr(wsum), _stream()))

    def backward(self, theta, batch: Batch, dloss, grad, theta_bf16=None):
        b = batch.struct()
        self._check(self.L.gs_backward(self.h, _ptr(theta), _ptr(theta_bf16), ctypes.byref(b), _ptr(dloss),
                                       _ptr(grad), _stream()))

    def forward_backward(self, theta, batch: Batch, dloss, loss, grad, theta_bf16=None):
        b = batch.struct()
        self._check(self.L.gs_forward_backward(self.h, _ptr(theta), _ptr(theta_bf16), ctypes.byref(b), _ptr(dloss),
                                               _ptr(loss), _ptr(grad), _stream()))

    @property
    def bf16(self) -> bool:
        return self.cfg.precision == GS_PREC_BF16

    def adam_step(self, theta, grad, m, v, t, lr_grid, lr_mlp, beta1=0.9, beta2=0.999, eps=1e-8, theta_bf16=None,
                  n_grid=None):
        """n_grid: entries taking lr_grid (default: this context's grid size; 0 for a vector
        that is not the main parameter vector, e.g. the proposal network's)."""
        n = theta.numel()
        ng = self.n_grid if n_grid is None else n_grid
        self._check(self.L.gs_adam_step(self.h, _ptr(theta), _ptr(grad), _ptr(m), _ptr(v), n, ng, t,
                                        lr_grid, lr_mlp, beta1, beta2, eps, _ptr(theta_bf16), _stream()))

    def query_sdf(self, theta, x, sdf, grad=None):
        self._check(self.L.gs_query_sdf(self.h, _ptr(theta), _ptr(x), x.shape[0], _ptr(sdf), _ptr(grad), _stream()))

    def proposal_sample(self, frames: DeviceFrames, seed: int, step: int, batch: Batch, theta=None, prop=None,
                        pdf_in=None, pdf_out=None):
        b = batch.struct()
        self._check(self.L.gs_proposal_sample(self.h, _ptr(theta), _ptr(prop), ctypes.byref(frames.s), seed, step,
                                              _ptr(pdf_in), _ptr(pdf_out), ctypes.byref(b), _stream()))

    def sample_importance(self, frames: DeviceFrames, theta, seed: int, step: int, batch: Batch):
        """Hierarchical importance sampling of the rays of sample_rays(seed, step)."""
        b = batch.struct()
        self._check(self.L.gs_sample_importance(self.h, _ptr(theta), ctypes.byref(frames.s), seed, step,
                                                ctypes.byref(b), _stream()))

    def proposal_backward(self, theta, prop, batch: Batch, prop_grad, ce=None):
        b = batch.struct()
        self._check(self.L.gs_proposal_backward(self.h, _ptr(theta), _ptr(prop), ctypes.byref(b), _ptr(prop_grad),
                                                _ptr(ce), _stream()))

    def query_sdf_backward(self, theta, x, dsdf, dgrad, grad):
        self._check(self.L.gs_query_sdf_backward(self.h, _ptr(theta), _ptr(x), x.shape[0], _ptr(dsdf), _ptr(dgrad),
                                                 _ptr(grad), _stream()))

    def eikonal(self, theta, batch: Batch, loss=None, grad=None, dloss=None):
        """L_eik over the batch's free-space samples into loss [1]; grad += dloss * dL_eik/dtheta."""
        bs = batch.struct()
        self._check(self.L.gs_eikonal(self.h, _ptr(theta), ctypes.byref(bs), _ptr(dloss), _ptr(loss), _ptr(grad),
                                      _stream()))

    def pose_apply(self, c2w0, xi, c2w):
        """c2w [F][3][4] = the corrected poses [R0 Exp(nu) | t0 + dt] for xi [F][6] = (dt, nu)."""
        self._check(self.L.gs_pose_apply(self.h, _ptr(c2w0), _ptr(xi), c2w0.shape[0], _ptr(c2w), _stream()))

    def pose_backward(self, theta, frames: DeviceFrames, xi, batch: Batch, pose_grad):
        """pose_grad [F][6] += dL/dxi of the batch's per-ray losses (batch.dz from its backward pass)."""
        b = batch.struct()
        self._check(self.L.gs_pose_backward(self.h, _ptr(theta), ctypes.byref(frames.s), _ptr(xi), ctypes.byref(b),
                                            _ptr(pose_grad), _stream()))

    def eikonal_pose_backward(self, theta, frames: DeviceFrames, xi, batch: Batch, pose_grad, dloss=None):
        """pose_grad [F][6] += dloss * dL_eik/dxi: the Eikonal term's pose gradient through the
        free-space samples' positions (dloss: device float [1] or None for 1)."""
        b = batch.struct()
        self._check(self.L.gs_eikonal_pose_backward(self.h, _ptr(theta), ctypes.byref(frames.s), _ptr(xi),
                                                    ctypes.byref(b), _ptr(dloss), _ptr(pose_grad), _stream()))

    def extract_mesh(self, theta, lo, step: float, dims, iso: float = 0.0, max_tris: int | None = None,
                     phi=None):
        """Isosurface phi = iso on the lattice lo + (i, j, k) * step, dims = (nx, ny, nz):
        returns (triangles [T][3][3] on the device, T); phi [nz][ny][nx] may be given as scratch."""
        nx, ny, nz = (int(d) for d in dims)
        if phi is None:
            phi = torch.empty((nz, ny, nx), device=theta.device, dtype=torch.float32)
        cap = max_tris if max_tris is not None else 4 * (nx * ny + ny * nz + nx * nz)
        n = torch.zeros(1, device=theta.device, dtype=torch.int64)
        lo_h = (ctypes.c_float * 3)(*[float(v) for v in lo])
        while True:
            tris = torch.empty((max(cap, 1), 3, 3), device=theta.device, dtype=torch.float32)
            self._check(self.L.gs_extract_mesh(self.h, _ptr(theta), lo_h, float(step), nx, ny, nz, float(iso),
                                               _ptr(phi), _ptr(tris), cap, _ptr(n), _stream()))
            total = int(n.item())
            if total <= cap:
                return tris[:total], total
            cap = total

    def voxel_index(self, x, out):
        self._check(self.L.gs_voxel_index(self.h, _ptr(x), x.shape[0], _ptr(out), _stream()))

    def sync_status(self):
        self._check(self.L.gs_sync_status(self.h))


class GoSurfStep(torch.autograd.Function):
    """losses = GoSurfStep.apply(theta, ctx, batch): the six outputs of gs_forward
    (L_rgb, L_d, L_sdf, L_fs, L_smooth, total) as a differentiable function of the flat
    parameter vector; backward runs gs_backward with the incoming gradient as dloss."""

    @staticmethod
    def forward(fctx, theta, ctx: Context, batch: Batch, theta_bf16=None):
        loss = torch.empty(GS_NUM_LOSS, device=theta.device, dtype=torch.float32)
        ctx.forward(theta.detach(), batch, loss, theta_bf16=theta_bf16)
        fctx.save_for_backward(theta)
        fctx.gs = (ctx, batch, theta_bf16)
        return loss

    @staticmethod
    def backward(fctx, dloss):
        (theta,) = fctx.saved_tensors
        ctx, batch, theta_bf16 = fctx.gs
        grad = torch.zeros_like(theta)
        ctx.backward(theta.detach(), batch, dloss.contiguous().float(), grad, theta_bf16=theta_bf16)
        return grad, None, None, None


class SdfGrad(torch.autograd.Function):
    """sdf, grad_x = SdfGrad.apply(theta, ctx, x): the SDF phi(x) [P] and its spatial gradient
    [P][3] (gs_query_sdf) as differentiable functions of the flat parameter vector.  The
    backward pass runs gs_query_sdf_backward, so a loss on grad_x (an eikonal or smoothness
    term) reaches the grid and the decoder through the second-order path.  The points x are
    treated as constants."""

    @staticmethod
    def forward(fctx, theta, ctx: Context, x):
        x = x.detach().float().contiguous()
        sdf = torch.empty(x.shape[0], device=x.device, dtype=torch.float32)
        g = torch.empty(x.shape[0], 3, device=x.device, dtype=torch.float32)
        ctx.query_sdf(theta.detach(), x, sdf, g)
        fctx.save_for_backward(theta, x)
        fctx.gs = ctx
        return sdf, g

    @staticmethod
    def backward(fctx, dsdf, dgrad):
        theta, x = fctx.saved_tensors
        grad = torch.zeros_like(theta)
        ds = None if dsdf is None else dsdf.contiguous().float()
        dg = None if dgrad is None else dgrad.contiguous().float()
        fctx.gs.query_sdf_backward(theta.detach(), x, ds, dg, grad)
        return grad, None, None
