"""Training through the rasterizer.

`render` is a torch.autograd.Function over gs_render / gs_backward (the
backward recomputes the preprocess); `Trainer` runs the training step of the
paper: the loss 0.8 L1 + 0.2 (1 - SSIM) + w_depth L_depth (Sec. 3.1, 3.2;
w_depth decayed exponentially from 0.5 to 0.0025, Sec. 4.1) plus the
depth-normal consistency (0.0125) and depth distortion (0) terms, the
decomposed-gradient densification statistics (Eq. 2), the elongation filter
(Sec. 3.2), clone / split / prune, and an FP32 Adam update of the
parametrisation (mu, quaternion, log-scale, logit-opacity, SH).  This module
only marshals arguments: every step runs in the library's kernels.
"""
from __future__ import annotations

import math

import torch

from . import binding as B

PARAMS = ("mu", "quat", "scale", "opacity", "sh")


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, quat, scale, opacity, sh, scene, cam, planes):
        out, frame = scene.render(cam)
        ctx.frame, ctx.scene, ctx.planes = frame, scene, planes
        return out

    @staticmethod
    def backward(ctx, grad_out):
        sc = ctx.scene
        grads = {k: torch.zeros_like(t) for k, t in zip(PARAMS, sc.params)}
        adj = grad_out[:B.ADJ_PLANES].contiguous()
        sc.backward(ctx.frame, [adj], [ctx.planes], grads)
        ctx.frame.release()
        return (grads["mu"], grads["quat"], grads["scale"], grads["opacity"], grads["sh"], None, None, None)


def render(scene: B.Scene, cam: dict, planes: int = 0x7FF):
    """Render planes [12, H, W] of `scene` as a differentiable function of the
    scene's parameter tensors (which must be the ones the scene was created
    with).  `planes` masks the adjoint planes the backward reads."""
    mu, quat, scale, opacity, sh = scene.params
    return _Render.apply(mu, quat, scale, opacity, sh, scene, cam, planes)


MASK_TRAIN = 0x7 | (1 << 3) | (1 << 5) | (1 << 6) | (0x7 << 7) | (1 << 10)  # rgb, alpha, invdepth, median, normal, dist


class Trainer:
    """Training state of one scene: raw parameters, Adam moments, densification
    statistics, and the step of the paper's schedule."""

    def __init__(self, mu, quat, log_scale, logit_opacity, sh, sh_degree, lr=None, w_normal=0.0125, w_dist=0.0,
                 depth_weights=(0.5, 0.0025), total_steps=30000, omega=0.9, grad_thr=0.0002, eta_thr=0.1):
        dev = mu.device
        self.sh_degree = int(sh_degree)
        self.raw = {"mu": mu.contiguous(), "quat": quat.contiguous(), "scale": log_scale.contiguous(),
                    "opacity": logit_opacity.contiguous(), "sh": sh.contiguous()}
        self.lr = dict(mu=1.6e-4, quat=1e-3, scale=5e-3, opacity=5e-2, sh=2.5e-3)
        if lr:
            self.lr.update(lr)
        self.w_normal, self.w_dist = w_normal, w_dist
        self.depth_weights, self.total_steps = depth_weights, total_steps
        self.omega, self.grad_thr, self.eta_thr = omega, grad_thr, eta_thr
        self.step_count = 0
        self._build(dev)

    def _build(self, dev):
        n = self.raw["mu"].shape[0]
        self.n = n
        self.m = {k: torch.zeros_like(v) for k, v in self.raw.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.raw.items()}
        self.scale, self.opacity = B.activate(self.raw["scale"], self.raw["opacity"])
        self.scene = B.Scene(self.raw["mu"], self.raw["quat"], self.scale, self.opacity, self.raw["sh"],
                             self.sh_degree)
        self.grads = {k: torch.zeros_like(v) for k, v in self.raw.items()}
        self.stats = torch.zeros((n, 4), device=dev)
        self.screen = torch.zeros((3, n, 2), device=dev)

    def depth_weight(self):
        a, b = self.depth_weights
        t = min(self.step_count / max(self.total_steps, 1), 1.0)
        return a * math.exp(t * math.log(b / a))

    def step(self, views):
        """One training step over a batch of views [(cam, target rgb [3,H,W],
        target inverse depth [H,W] or None)]; returns the summed losses
        (device tensor [6]: l1, ssim, depth, total, normal, distortion)."""
        B.activate(self.raw["scale"], self.raw["opacity"], self.scale, self.opacity)
        for g in self.grads.values():
            g.zero_()
        self.screen.zero_()
        total = torch.zeros(6, device=self.raw["mu"].device)
        wd = self.depth_weight()
        for cam, tgt, tinv in views:
            H, W = int(cam["height"]), int(cam["width"])
            out, frame = self.scene.render(cam)
            adj = [torch.zeros((B.ADJ_PLANES, H, W), device=out.device) for _ in range(3)]
            losses, _, _, _ = B.loss(out, tgt, tinv, (0.8, 0.2, wd), adj_total=adj[0], adj_ssim=adj[1],
                                     adj_l1=adj[2])
            geo = B.geometry_loss(out, cam, self.w_normal, self.w_dist, adj[0])
            grads_act = {"mu": self.grads["mu"], "quat": self.grads["quat"], "scale": self.grads["scale"],
                         "opacity": self.grads["opacity"], "sh": self.grads["sh"]}
            self.scene.backward(frame, adj, [MASK_TRAIN, 0x7, 0x7], grads_act, self.screen)
            self.scene.densify_accumulate(frame, self.screen, self.stats)
            frame.release()
            total[:4] += losses
            total[4:] += geo
        B.activate_grad(self.scale, self.opacity, self.grads["scale"], self.grads["opacity"])
        self.step_count += 1
        for k in PARAMS:
            B.adam_step(self.raw[k], self.grads[k], self.m[k], self.v[k], self.lr[k], self.step_count)
        return total

    def densify(self, dense_thr, min_opacity=0.005, xi=None):
        """Clone / split / prune with the selection of Eq. 2 and the elongation
        filter; restarts the statistics.  xi: standard normals [N, 2, 2] for the
        split children (drawn here when None)."""
        B.activate(self.raw["scale"], self.raw["opacity"], self.scale, self.opacity)
        mask, _, _ = B.densify_select(self.stats, self.scale, self.omega, self.grad_thr, self.eta_thr)
        keep = B.elongation_filter(self.scale, self.eta_thr)
        action, offset, n_out = B.densify_plan(mask, self.raw["scale"], self.raw["opacity"], dense_thr, min_opacity,
                                               keep=keep, raw=True)
        if xi is None:
            xi = torch.randn((self.n, 2, 2), device=self.scale.device)
        new, src, fresh = B.densify_apply(self.raw, self.sh_degree, action, offset, n_out, xi, raw=True)
        m = {k: B.gather_rows(src, fresh, v) for k, v in self.m.items()}
        v = {k: B.gather_rows(src, fresh, t) for k, t in self.v.items()}
        self.raw = new
        self.scene.close()
        self._build(self.raw["mu"].device)
        self.m, self.v = m, v
        return n_out
