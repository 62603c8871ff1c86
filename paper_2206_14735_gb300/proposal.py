"""Training loop of the learned proposal sampler (an addition to the method: fewer samples
per ray) and the controller that falls back to the plain sampler.

Every step trains the proposal network on the main model's rendering weights of the batch
just rendered (gs_proposal_backward) and updates it with Adam.  Every ``eval_every`` steps
a held-out batch of ``holdout`` rays is rendered twice by the current model, once with the
plain samples and once with the proposal's; the depth L1 of both (the forward pass's L_d)
decides whether the next steps sample from the proposal (its L1 at most ``tolerance`` times
the plain one) or fall back to the plain sampler.  All arithmetic runs in the library's
kernels; this module only sequences the calls and reads two loss values per evaluation.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from ._lib import GS_NUM_LOSS, GS_PROP_PARAMS

PROP_PAD = (GS_PROP_PARAMS + 3) // 4 * 4  # Adam works on multiples of 4 floats


@dataclass
class FallbackController:
    """Sampler choice from held-out depth errors: proposal while its depth L1 stays within
    ``tolerance`` x the plain sampler's, plain otherwise.  Starts on the plain sampler."""
    tolerance: float = 1.05
    use_proposal: bool = False
    history: list = field(default_factory=list)

    def update(self, l1_proposal: float, l1_plain: float) -> bool:
        ok = bool(np.isfinite(l1_proposal)) and l1_proposal <= self.tolerance * l1_plain
        self.use_proposal = ok
        self.history.append((float(l1_proposal), float(l1_plain), ok))
        return ok


def init_proposal_params(seed: int = 7, scale: float = 0.1) -> np.ndarray:
    """Initial proposal parameters (padded to PROP_PAD floats): small normal weights, zero
    biases, so the first proposals are close to uniform."""
    rng = np.random.default_rng(seed)
    q = np.zeros(PROP_PAD, np.float32)
    q[:352] = rng.normal(0, scale, 352)                 # W1 [32][11]
    q[384:1408] = rng.normal(0, scale / 2, 1024)        # W2 [32][32]
    q[1440:1472] = rng.normal(0, scale, 32)             # w3
    return q


class ProposalTrainer:
    """One optimisation step of the main model with the proposal sampler (or the plain
    fallback), the proposal's own training step, and the periodic fallback decision."""

    def __init__(self, ctx, workload, frames, *, seed: int = 3, eval_every: int = 25, holdout: int | None = None,
                 tolerance: float = 1.05, q0: np.ndarray | None = None, train_rays: int | None = 16384,
                 mirror=None):
        from . import Batch  # local import: the package imports this module lazily
        w = workload
        self.ctx, self.w, self.frames, self.seed = ctx, w, frames, seed
        self.mirror = mirror  # BF16 form: the grid copy the gathers read (refreshed by every Adam step)
        self.eval_every = eval_every
        R, P = w.rays, w.n_smooth
        self.batch_plain = Batch.allocate(R, w.n_samples, P, weights=True)
        self.batch_prop = Batch.allocate(R, w.prop_samples, P, weights=True)
        Rh = holdout if holdout is not None else max(1, R // 100)
        self.hold_plain = Batch.allocate(Rh, w.n_samples, 0)
        self.hold_prop = Batch.allocate(Rh, w.prop_samples, 0)
        self.q = torch.from_numpy(init_proposal_params() if q0 is None else q0.astype(np.float32)).cuda()
        self.gq = torch.zeros_like(self.q)
        self.mq = torch.zeros_like(self.q)
        self.vq = torch.zeros_like(self.q)
        self.ce = torch.zeros(2, device="cuda")
        self.hold_loss = torch.zeros(2, GS_NUM_LOSS, device="cuda")
        self.controller = FallbackController(tolerance=tolerance)
        self.t_q = 0
        # the proposal learns from the first train_rays rays of each batch (rays are i.i.d.)
        self.train_rays = R if train_rays is None else min(R, train_rays)

    def batch(self, step: int, theta):
        """Sample this step's batch with the current sampler choice."""
        if self.controller.use_proposal:
            self.ctx.proposal_sample(self.frames, self.seed, step, self.batch_prop, theta=theta, prop=self.q)
            return self.batch_prop
        self.ctx.sample_rays(self.frames, self.seed, step, self.batch_plain)
        return self.batch_plain

    def train_proposal(self, theta, batch):
        """Cross-entropy step of the proposal on the weights the last forward pass wrote
        (first train_rays rays of the batch)."""
        from dataclasses import replace
        sub = batch if self.train_rays >= batch.R else replace(batch, R=self.train_rays)
        self.ctx.proposal_backward(theta, self.q, sub, self.gq, self.ce)
        self.t_q += 1
        self.ctx.adam_step(self.q, self.gq, self.mq, self.vq, self.t_q, 0.0, self.w.lr_prop, self.w.betas[0],
                           self.w.betas[1], self.w.adam_eps, n_grid=0)

    def evaluate(self, step: int, theta) -> bool:
        """Depth L1 of the plain and proposal samplers on a held-out batch (rays drawn with
        another seed); updates the controller."""
        hs = self.seed + 7919
        self.ctx.sample_rays(self.frames, hs, step, self.hold_plain)
        self.ctx.forward(theta, self.hold_plain, self.hold_loss[0], theta_bf16=self.mirror)
        self.ctx.proposal_sample(self.frames, hs, step, self.hold_prop, theta=theta, prop=self.q)
        self.ctx.forward(theta, self.hold_prop, self.hold_loss[1], theta_bf16=self.mirror)
        l = self.hold_loss[:, 1].cpu().numpy()
        return self.controller.update(float(l[1]), float(l[0]))

    def step(self, step: int, theta, grad, m, v, loss):
        """One full step: sample, fused forward/backward of the main model (writes the
        rendering weights), proposal training, Adam on both, periodic fallback decision."""
        b = self.batch(step, theta)
        self.ctx.forward_backward(theta, b, None, loss, grad, theta_bf16=self.mirror)
        self.train_proposal(theta, b)
        w = self.w
        self.ctx.adam_step(theta, grad, m, v, step + 1, w.lr_grid, w.lr_mlp, w.betas[0], w.betas[1], w.adam_eps,
                           theta_bf16=self.mirror)
        if self.eval_every > 0 and (step + 1) % self.eval_every == 0:
            self.evaluate(step, theta)
        return b
