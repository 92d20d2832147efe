"""Training loop on the GPU (next row #2): geometric loss terms, Adam,
densification, activations, the autograd render, and the full training loss's
gradient against central finite differences of the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2411_00771_gb300 import synthetic as syn
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def test_geometry_loss_matches_oracle():
    from paper_2411_00771_gb300 import binding as B
    scene, cam, _, _ = syn.tiny_scene(seed=21, n=3000, width=72, height=56, fx=64.0, sh_degree=1,
                                      log_scale_range=(-3.5, -1.5))
    sc, d, out, cnt, frame = gu.gpu_render(scene, cam)
    adj = torch.zeros((11, 56, 72), device="cuda")
    losses = B.geometry_loss(out, cam, 0.0125, 0.3, adj)
    torch.cuda.synchronize()
    o = out.cpu().numpy().astype(np.float64)
    L, radj = oracle.normal_loss(o, cam, weight=0.0125)
    got = losses.cpu().numpy()
    assert abs(got[0] - L) <= 1e-4 * abs(L) + 1e-9
    assert abs(got[1] - 0.3 * o[10].mean()) <= 1e-5 * abs(0.3 * o[10].mean()) + 1e-9
    a = adj.cpu().numpy()
    for p in (3, 6, 7, 8, 9):
        scale = np.abs(radj[p]).max()
        assert np.abs(a[p] - radj[p]).max() <= 1e-3 * scale + 1e-12, p
    assert np.all(a[10] == np.float32(0.3 / (56 * 72)))


@pytest.mark.parametrize("n,offset", [(1 << 20, 0), (1000003, 0), (4099, 1)])
def test_adam_matches_oracle(n, offset):
    """Four values per thread when every array is 16-byte aligned, one at a
    time for the tail and for misaligned arrays (offset by one float)."""
    from paper_2411_00771_gb300 import binding as B
    rng = np.random.default_rng(3)
    p0 = rng.normal(size=n).astype(np.float32)

    def dev(x):
        buf = torch.zeros(n + offset, device="cuda")
        buf[offset:] = torch.from_numpy(x).cuda()
        return buf[offset:]

    p, m, v = dev(p0.copy()), dev(np.zeros(n, np.float32)), dev(np.zeros(n, np.float32))
    rp, rm, rv = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for k in range(1, 4):
        g = rng.normal(size=n).astype(np.float32)
        B.adam_step(p, dev(g), m, v, 1e-3, k)
        rp, rm, rv = oracle.adam_step(rp, g, rm, rv, 1e-3, k)
    torch.cuda.synchronize()
    assert np.abs(p.cpu().numpy() - rp).max() <= 1e-6


@pytest.mark.parametrize("raw", [False, True])
def test_densify_plan_and_apply_match_oracle(raw):
    from paper_2411_00771_gb300 import binding as B
    rng = np.random.default_rng(5)
    scene, _, _, _ = syn.tiny_scene(seed=5, n=5000, sh_degree=2)
    n = 5000
    sel = (rng.random(n) < 0.3).astype(np.uint8)
    keep = (rng.random(n) < 0.9).astype(np.uint8)
    opac = np.asarray(scene["opacity"], np.float32).copy()
    opac[rng.random(n) < 0.05] = 0.001
    scale = np.asarray(scene["scale"], np.float32)
    xi = rng.normal(size=(n, 2, 2)).astype(np.float32)
    d = {k: torch.from_numpy(np.ascontiguousarray(v, np.float32)).cuda()
         for k, v in dict(mu=scene["mu"], quat=scene["quat"], scale=scale, opacity=opac, sh=scene["sh"]).items()}
    if raw:
        d["scale"] = torch.log(d["scale"])
        d["opacity"] = torch.logit(d["opacity"])
    thr = float(np.median(scale.max(axis=1)))
    action, offset, n_out = B.densify_plan(torch.from_numpy(sel).cuda(), d["scale"], d["opacity"], thr, 0.005,
                                           keep=torch.from_numpy(keep).cuda(), raw=raw)
    new, src, fresh = B.densify_apply(d, 2, action, offset, n_out, torch.from_numpy(xi).cuda(), raw=raw)
    torch.cuda.synchronize()
    ra, roff, rn = oracle.densify_plan(sel & keep, scale, opac, thr, 0.005)
    assert n_out == rn and np.array_equal(action.cpu().numpy(), ra)
    assert np.array_equal(offset.cpu().numpy().astype(np.int64), roff)
    rs = dict(scene)
    rs["opacity"], rs["scale"] = opac, scale
    ref, rsrc, rfresh = oracle.densify_apply(rs, ra, xi)
    assert np.array_equal(src.cpu().numpy(), rsrc) and np.array_equal(fresh.cpu().numpy(), rfresh)
    assert np.abs(new["mu"].cpu().numpy() - ref["mu"]).max() <= 1e-5 * max(1.0, np.abs(ref["mu"]).max())
    got_scale = new["scale"].cpu().numpy()
    if raw:
        got_scale = np.exp(got_scale)
    assert np.abs(got_scale - ref["scale"]).max() <= 1e-5 * ref["scale"].max()
    assert np.array_equal(new["sh"].cpu().numpy(), ref["sh"].astype(np.float32))
    # optimizer state follows the rows; fresh rows restart at zero
    m = torch.arange(n * 3, dtype=torch.float32, device="cuda").reshape(n, 3)
    g = B.gather_rows(src, fresh, m).cpu().numpy()
    exp = np.where(rfresh[:, None] == 1, 0.0, m.cpu().numpy()[rsrc])
    assert np.array_equal(g, exp)


def test_activations_and_their_gradients():
    from paper_2411_00771_gb300 import binding as B
    rng = np.random.default_rng(6)
    ls = torch.from_numpy(rng.normal(-2, 1, (1000, 2)).astype(np.float32)).cuda()
    lo = torch.from_numpy(rng.normal(0, 2, 1000).astype(np.float32)).cuda()
    s, o = B.activate(ls, lo)
    gs = torch.ones_like(s)
    go = torch.ones_like(o)
    B.activate_grad(s, o, gs, go)
    torch.cuda.synchronize()
    sl, ol = np.exp(ls.cpu().numpy().astype(np.float64)), 1 / (1 + np.exp(-lo.cpu().numpy().astype(np.float64)))
    assert np.abs(s.cpu().numpy() - sl).max() <= 1e-6 * sl.max() and np.abs(o.cpu().numpy() - ol).max() <= 1e-6
    assert np.abs(gs.cpu().numpy() - sl).max() <= 1e-6 * sl.max()
    assert np.abs(go.cpu().numpy() - ol * (1 - ol)).max() <= 1e-6


def test_autograd_render_matches_oracle_backward():
    from paper_2411_00771_gb300 import training as T
    scene, cam, _, _ = syn.tiny_scene(seed=31, n=800, width=64, height=48, fx=60.0, sh_degree=2,
                                      log_scale_range=(-3.5, -1.5))
    sc, d = gu.gpu_scene(scene)
    for t in d.values():
        t.requires_grad_(True)
    rng = np.random.default_rng(2)
    adj = rng.normal(size=(11, 48, 64))
    out = T.render(sc, cam)
    (out[:11] * torch.from_numpy(adj.astype(np.float32)).cuda()).sum().backward()
    torch.cuda.synchronize()
    ref = oracle.backward(scene, cam, adj[None])
    for k in ("mu", "quat", "scale", "opacity", "sh"):
        g = d[k].grad.cpu().numpy().astype(np.float64)
        assert gu.rel_err(g, ref[k].reshape(g.shape)) <= 1e-3, k


@pytest.mark.parametrize("autograd", [False, True])
def test_training_loss_gradient_against_finite_differences(autograd):
    """The 4M-surfel configuration's loss (L1, SSIM, depth, normal
    consistency, distortion) through the trained parametrisation (log-scale,
    logit-opacity): the GPU gradient, by the direct step or by autograd,
    against central FD of the FP64 oracle on a 64-surfel subset."""
    from paper_2411_00771_gb300 import binding as B
    from paper_2411_00771_gb300 import training as T
    scene, cam, tgt, tinv = syn.tiny_scene(seed=78, n=300, width=48, height=48, fx=48.0, sh_degree=1,
                                           log_scale_range=(-3.0, -1.5))
    wl, wn, wdist = (0.8, 0.2, 0.5), 0.0125 * 4, 0.01
    d = gu.to_dev(scene)
    log_s = torch.log(d["scale"]).contiguous()
    logit = torch.logit(d["opacity"]).contiguous()
    tr = T.Trainer(d["mu"], d["quat"], log_s, logit, d["sh"], scene["sh_degree"], lr=dict(mu=0, quat=0, scale=0,
                   opacity=0, sh=0), w_normal=wn, w_dist=wdist, depth_weights=(0.5, 0.5))
    tr.step([(cam, torch.from_numpy(tgt).cuda(), torch.from_numpy(tinv).cuda())], autograd=autograd)
    torch.cuda.synchronize()
    src = {k: tr.raw[k].grad for k in T.PARAMS} if autograd else tr.grads
    grads = {k: v.detach().cpu().numpy().astype(np.float64) for k, v in src.items()}
    s64 = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) else v) for k, v in scene.items()}
    raw = {"scale": np.log(s64["scale"]), "opacity": np.log(s64["opacity"] / (1 - s64["opacity"]))}

    def f(s):
        r = oracle.render(s, cam)["out"]
        return (oracle.loss(r, tgt, tinv, wl)["total"] + oracle.normal_loss(r, cam, wn)[0] + wdist * r[10].mean())

    rng = np.random.default_rng(0)
    pre = oracle.preprocess(scene, cam)
    subset = rng.choice(np.nonzero(pre["tiles"] > 0)[0], 64, replace=False)
    K = (scene["sh_degree"] + 1) ** 2

    def perturbed(key, idx, dx):
        s = dict(s64)
        if key in ("scale", "opacity"):  # the trained (raw) parametrisation
            r = raw[key].copy()
            r[idx] += dx
            s[key] = np.exp(r) if key == "scale" else 1 / (1 + np.exp(-r))
        else:
            s[key] = s64[key].copy()
            s[key][idx] += dx
        return s

    # A point is used only where the loss is smooth across the step: the
    # central differences at h and h/2 agree.  The normal-consistency term
    # follows the median depth, whose pair changes by a jump when a
    # transmittance crosses 1/2; a step across such a switch (or across the
    # alpha cutoff, the support boundary, the stop) breaks the agreement.
    checked, skipped = 0, 0
    for i in subset:
        for key, comp in (("mu", (rng.integers(3),)), ("quat", (rng.integers(4),)),
                          ("scale", (rng.integers(2),)), ("opacity", ()),
                          ("sh", (rng.integers(K), rng.integers(3)))):
            idx = (i,) + tuple(int(c) for c in comp)
            h = 1e-6
            fd = {hh: (f(perturbed(key, idx, hh)) - f(perturbed(key, idx, -hh))) / (2 * hh) for hh in (h, h / 2)}
            if abs(fd[h] - fd[h / 2]) > 1e-5 * max(abs(fd[h]), 1e-4):
                skipped += 1
                continue
            gv = grads[key][idx]
            assert abs(gv - fd[h]) <= 1e-3 * max(abs(fd[h]), 1e-4), (key, idx, gv, fd[h])
            checked += 1
    assert checked + skipped == 320 and checked >= 290, (checked, skipped)


def test_trainer_reduces_the_loss_and_densifies():
    from paper_2411_00771_gb300 import training as T
    scene, cam, _, _ = syn.tiny_scene(seed=90, n=2000, sh_degree=1)
    tgt_scene = dict(scene)
    tgt_scene["opacity"] = np.clip(np.asarray(scene["opacity"]) * 1.2, 0, 0.95).astype(np.float32)
    tsc, _ = gu.gpu_scene(tgt_scene)
    tout, _ = tsc.render(cam, save=False)
    tgt, tinv = tout[:3].contiguous(), tout[5].contiguous()
    d = gu.to_dev(scene)
    tr = T.Trainer(d["mu"], d["quat"], torch.log(d["scale"]), torch.logit(d["opacity"]), d["sh"], 1,
                   lr=dict(mu=1e-4, quat=1e-3, scale=5e-3, opacity=5e-2, sh=2.5e-3), total_steps=50)
    first = last = None
    for k in range(30):
        L = tr.step([(cam, tgt, tinv)])
        v = float(L[3])
        first = v if first is None else first
        last = v
    assert last < first
    n0 = tr.n
    n1 = tr.densify(dense_thr=0.05, xi=torch.zeros((n0, 2, 2), device="cuda"))
    assert n1 == tr.n and n1 > 0
    L = tr.step([(cam, tgt, tinv)])
    assert math.isfinite(float(L[3]))


def _two_views(n=3000, W=96, H=72):
    scene, cam, tgt, tinv = syn.tiny_scene(seed=101, n=n, width=W, height=H, fx=float(W), sh_degree=2,
                                           log_scale_range=(-3.5, -1.5))
    cam2 = dict(cam)
    yaw = 0.12
    cy, sy = math.cos(yaw), math.sin(yaw)
    cam2["R"] = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]]) @ np.asarray(cam["R"])
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    rng = np.random.default_rng(7)
    tgt2 = rng.random(tgt.shape).astype(np.float32)
    return scene, [(cam, t(tgt), t(tinv)), (cam2, t(tgt2), t(tinv))]


def _trainer(scene, **kw):
    from paper_2411_00771_gb300 import training as T
    d = gu.to_dev(scene)
    return T.Trainer(d["mu"], d["quat"], torch.log(d["scale"]).contiguous(), torch.logit(d["opacity"]).contiguous(),
                     d["sh"], scene["sh_degree"], w_normal=0.05, w_dist=0.01, **kw)


def test_autograd_step_equals_direct_step():
    """The step built from the differentiable activate / render / loss and one
    backward() over two views gives the direct step's losses, gradients,
    densification statistics and Adam update (up to the order of FP32 sums)."""
    from paper_2411_00771_gb300 import training as T
    scene, views = _two_views()
    a, b = _trainer(scene), _trainer(scene)
    La = a.step(views)
    Lb = b.step(views, autograd=True)
    torch.cuda.synchronize()
    assert torch.allclose(La, Lb, rtol=1e-6, atol=1e-9)
    for k in T.PARAMS:
        ga, gb = a.grads[k], b.raw[k].grad
        assert float((ga - gb).norm() / ga.norm().clamp_min(1e-30)) <= 1e-5, k
        assert torch.allclose(a.raw[k], b.raw[k].detach(), rtol=1e-5, atol=1e-7), k
    assert torch.allclose(a.stats, b.stats, rtol=1e-5, atol=1e-9)
    # a second step reuses the buffers and the moments
    a.step(views)
    b.step(views, autograd=True)
    torch.cuda.synchronize()
    for k in T.PARAMS:
        assert torch.allclose(a.raw[k], b.raw[k].detach(), rtol=1e-5, atol=1e-7), k


@pytest.mark.parametrize("autograd", [False, True])
def test_statistics_take_each_views_own_screen_gradient(autograd):
    """Eq. 2 sums, per view, the norm of that view's screen gradient: a
    two-view step must add what two one-view steps add (with the updates
    switched off so that both see the same parameters)."""
    scene, views = _two_views()
    zero = dict(mu=0.0, quat=0.0, scale=0.0, opacity=0.0, sh=0.0)
    const = (0.5, 0.5)  # the same depth weight at every step count
    a, b = _trainer(scene, lr=zero, depth_weights=const), _trainer(scene, lr=zero, depth_weights=const)
    a.step(views, autograd=autograd)
    b.step(views[:1], autograd=autograd)
    b.step(views[1:], autograd=autograd)
    torch.cuda.synchronize()
    assert float(a.stats[:, 3].sum()) > 0
    assert torch.allclose(a.stats, b.stats, rtol=1e-5, atol=1e-9)


def test_training_workload_view_at_full_size():
    """One view of the 4M-surfel training workload as the benchmark builds it
    (orbit 200 m up, 1600x900): 10 000 sampled pixels against the oracle, and
    the backward through a 256x256 window against a crop camera and the
    oracle."""
    scene, info = syn.city_scene(seed=20241101 + 3, n=4_000_000)
    rng = np.random.default_rng(20241101 + 4)
    cam = syn.orbit_camera(rng, 1600, 900, radius=rng.uniform(150.0, 250.0), altitude=200.0)
    sc, d, out, cnt, frame = gu.gpu_render(scene, cam)
    frame.release()
    ref = gu.compare_sampled(scene, cam, out.cpu().numpy(), cnt.cpu().numpy(), 10_000, seed=3)
    assert (ref["count"] > 0).mean() > 0.5
    del sc, d, out, cnt
    torch.cuda.empty_cache()
    gu.check_window_backward(scene, cam, 672, 324, 256, seed=4)
