"""Training through the rasterizer.

`render` is a torch.autograd.Function over gs_render / gs_backward (the
backward recomputes the preprocess); `Trainer` runs the training step of the
paper: the loss 0.8 L1 + 0.2 (1 - SSIM) + w_depth L_depth (Sec. 3.1, 3.2;
w_depth decayed exponentially from 0.5 to 0.0025, Sec. 5.1) plus the
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


class Densify:
    """Per-view link between `loss` and `render` for the decomposed
    densification statistics (Eq. 2): the loss stores the adjoints of its SSIM
    and L1 terms here, and the render's backward replays them beside the total
    loss's adjoint, then adds the per-view screen-gradient norms to `stats`.

    accumulate: optional {name: tensor} for leaf parameters among mu, quat, sh
    whose .grad the caller has set to that tensor: the backward adds this
    view's gradient straight into it and hands autograd none for them, which
    saves a zeroed gradient per view and autograd's sum over views."""

    def __init__(self, stats, screen, accumulate=None):
        self.stats, self.screen, self.sets = stats, screen, None
        self.accumulate = accumulate or {}


class _Render(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, quat, scale, opacity, sh, scene, cam, planes, densify):
        out, frame = scene.render(cam)
        ctx.frame, ctx.scene, ctx.planes, ctx.densify = frame, scene, planes, densify
        return out

    @staticmethod
    def backward(ctx, grad_out):
        sc, d = ctx.scene, ctx.densify
        direct = d.accumulate if d is not None else {}
        grads = {k: direct[k] if k in direct else torch.zeros_like(t) for k, t in zip(PARAMS, sc.params)}
        adj = [grad_out[:B.ADJ_PLANES].contiguous()]
        masks = [ctx.planes]
        if d is not None and d.sets is not None:
            adj += d.sets
            masks += [0x7] * len(d.sets)
        if d is not None:
            screen = d.screen[:len(adj)]
            screen.zero_()
            sc.backward(ctx.frame, adj, masks, grads, screen)
            sc.densify_accumulate(ctx.frame, screen, d.stats)
            d.sets = None
        else:
            sc.backward(ctx.frame, adj, masks, grads)
        ctx.frame.release()
        out = [None if k in direct else grads[k] for k in PARAMS]
        return (*out, None, None, None, None)


def render(scene: B.Scene, cam: dict, planes: int = 0x7FF, densify: Densify = None, params=None):
    """Render planes [12, H, W] of `scene` as a differentiable function of its
    parameter tensors: `params` (mu, quat, scale, opacity, sh) when given,
    which must hold the memory the scene was created with, else the scene's
    own tensors.  `planes` masks the adjoint planes the backward reads."""
    params = scene.params if params is None else tuple(params)
    for a, b in zip(params, scene.params):
        if a.data_ptr() != b.data_ptr():
            raise ValueError("render: params do not hold the scene's parameter memory")
    return _Render.apply(*params, scene, cam, planes, densify)


class _Loss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, out, target, tinv, cam, weights, w_normal, w_dist, densify):
        H, W = out.shape[-2:]
        grad = torch.zeros((B.OUT_PLANES, H, W), device=out.device)  # the last plane has no adjoint
        adj = grad[:B.ADJ_PLANES]
        sets = [None, None]
        if densify is not None:
            sets = [torch.zeros_like(adj), torch.zeros_like(adj)]
        vec = torch.empty(6, device=out.device)
        B.loss(out, target, tinv, weights, adj_total=adj, adj_ssim=sets[0], adj_l1=sets[1], losses=vec[:4])
        vec[4:] = B.geometry_loss(out, cam, w_normal, w_dist, adj)
        if densify is not None:
            densify.sets = sets
        ctx.grad = grad
        ctx.mark_non_differentiable(vec)
        return vec[3] + vec[4] + vec[5], vec

    @staticmethod
    def backward(ctx, g, _):
        grad, ctx.grad = ctx.grad, None
        return grad.mul_(g), None, None, None, None, None, None, None


def loss(out, target, tinv, cam, weights=(0.8, 0.2, 0.5), w_normal=0.0125, w_dist=0.0, densify: Densify = None):
    """The training loss of one view as a differentiable function of the
    render: 0.8 L1 + 0.2 (1 - SSIM) + w_depth L_depth (Sec. 3.1, 3.2) plus the
    depth-normal consistency and distortion terms.  Returns (scalar loss,
    [6] = l1, ssim, depth, photometric total, normal, distortion).  With
    `densify`, also keeps the SSIM and L1 terms' adjoints for the render's
    backward (Eq. 2)."""
    return _Loss.apply(out, target, tinv, cam, tuple(float(w) for w in weights), float(w_normal), float(w_dist),
                       densify)


class _Activate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, log_scale, logit_opacity, scale, opacity):
        B.activate(log_scale, logit_opacity, scale, opacity)
        ctx.mark_dirty(scale, opacity)
        ctx.buffers = (scale.detach(), opacity.detach())  # rewritten only by the next step's activate
        return scale, opacity

    @staticmethod
    def backward(ctx, g_scale, g_opacity):
        scale, opacity = ctx.buffers
        ctx.buffers = None
        gs = g_scale.contiguous().clone()
        go = g_opacity.contiguous().clone()
        B.activate_grad(scale, opacity, gs, go)
        return gs, go, None, None


def activate(log_scale, logit_opacity, scale, opacity):
    """scale = exp(log_scale), opacity = sigmoid(logit_opacity), written into
    the given buffers, differentiable with respect to the raw values.  Returns
    aliases of the buffers that carry this call's graph (the buffers
    themselves keep none, so they can be rewritten by the next call)."""
    return _Activate.apply(log_scale, logit_opacity, scale.detach(), opacity.detach())


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

    def step(self, views, autograd=False):
        """One training step over a batch of views [(cam, target rgb [3,H,W],
        target inverse depth [H,W] or None)]; returns the summed losses
        (device tensor [6]: l1, ssim, depth, photometric total, normal,
        distortion).  autograd=False drives the library's calls directly
        (gradients accumulate across the views in one set of buffers);
        autograd=True builds the step from the differentiable `activate`,
        `render` and `loss` and one backward() of the summed loss.  Both end
        with the same FP32 Adam update."""
        if autograd:
            return self._step_autograd(views)
        B.activate(self.raw["scale"], self.raw["opacity"], self.scale, self.opacity)
        for g in self.grads.values():
            g.zero_()
        total = torch.zeros(6, device=self.raw["mu"].device)
        wd = self.depth_weight()
        for cam, tgt, tinv in views:
            H, W = int(cam["height"]), int(cam["width"])
            out, frame = self.scene.render(cam)
            adj = [torch.zeros((B.ADJ_PLANES, H, W), device=out.device) for _ in range(3)]
            losses, _, _, _ = B.loss(out, tgt, tinv, (0.8, 0.2, wd), adj_total=adj[0], adj_ssim=adj[1],
                                     adj_l1=adj[2])
            geo = B.geometry_loss(out, cam, self.w_normal, self.w_dist, adj[0])
            self.screen.zero_()  # the statistics take each view's own screen gradient
            self.scene.backward(frame, adj, [MASK_TRAIN, 0x7, 0x7], self.grads, self.screen)
            self.scene.densify_accumulate(frame, self.screen, self.stats)
            frame.release()
            total[:4] += losses
            total[4:] += geo
        B.activate_grad(self.scale, self.opacity, self.grads["scale"], self.grads["opacity"])
        self._adam({k: self.grads[k] for k in PARAMS})
        return total

    def _step_autograd(self, views):
        direct = {k: self.grads[k] for k in ("mu", "quat", "sh")}
        for k, t in self.raw.items():
            t.requires_grad_(True)
            t.grad = None
            if k in direct:
                direct[k].zero_()
                t.grad = direct[k]
        wd = self.depth_weight()
        scale, opacity = activate(self.raw["scale"], self.raw["opacity"], self.scale, self.opacity)
        params = (self.raw["mu"], self.raw["quat"], scale, opacity, self.raw["sh"])
        total, vecs = None, []
        for cam, tgt, tinv in views:
            d = Densify(self.stats, self.screen, direct)
            out = render(self.scene, cam, MASK_TRAIN, d, params)
            L, vec = loss(out, tgt, tinv, cam, (0.8, 0.2, wd), self.w_normal, self.w_dist, d)
            total = L if total is None else total + L
            vecs.append(vec)
        total.backward()
        self._adam({k: self.raw[k].grad for k in PARAMS})
        return torch.stack(vecs).sum(0)

    def _adam(self, grads):
        self.step_count += 1
        for k in PARAMS:
            B.adam_step(self.raw[k], grads[k], self.m[k], self.v[k], self.lr[k], self.step_count)

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
