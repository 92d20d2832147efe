"""Contribution-based vector quantisation of SH (Sec. 3.3; Appendix C) on the
GPU against the FP64 oracle, and rendering from the compressed layout.

Assignments are integer results decided by floating point: the oracle takes
the decision in FP64 on the same binary16 operands and flags every vector
whose two best scores lie within the FP32 evaluation error; elsewhere the
GPU's entry must be the oracle's, and on flagged vectors it must be within
that error of the best.  Centroid updates use exact sums on both sides, so
codebooks are compared bit for bit."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2411_00771_gb300 import synthetic as syn
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

TC, SIMT = 1, 2


def _sh_set(n, deg, seed, keep_frac=0.6):
    rng = np.random.default_rng(seed)
    C = 3 * (deg + 1) ** 2
    sh = rng.normal(0, 0.05, (n, C // 3, 3)).astype(np.float32)
    sh[:, 0, :] = rng.uniform(-1.0, 1.5, (n, 1)) + rng.normal(0, 0.1, (n, 3))  # DC: albedo-like
    keep = (rng.random(n) < keep_frac).astype(np.uint8)
    return sh, keep


def _dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


def _check_assign(got, x16, c16, flag_ok_frac=0.01):
    a, flag, d = oracle.vq_assign(x16, c16)
    assert flag.mean() <= flag_ok_frac, flag.mean()
    assert np.array_equal(got[~flag], a[~flag]), np.nonzero(got[~flag] != a[~flag])[0][:10]
    if flag.any():  # the GPU's entry is within the FP32 evaluation error of the best
        x = x16[flag].astype(np.float64)
        c = c16.astype(np.float64)
        dg = ((x - c[got[flag]]) ** 2).sum(1)
        eps = oracle.vq_score_error(x, c[got[flag]]) + oracle.vq_score_error(x, c[a[flag]])
        assert np.all(dg - d[flag] <= eps)
    return a, flag


def _near_data(x16, K, rng, noise=0.02):
    """K entries drawn from the vectors plus noise: close but not tied."""
    pick = x16[rng.choice(x16.shape[0], K, replace=False)].astype(np.float64)
    return oracle.half(pick + rng.normal(0, noise, pick.shape))


def _steps_without_ties(x16, u, iters):
    """The longest prefix of Lloyd's steps (at most iters) in which the
    oracle met no near-tie; its result."""
    c, a, obj, flags = oracle.vq_kmeans(x16, u, iters)
    first = next((t for t, f in enumerate(flags) if f.any()), None)
    if first is not None and first < iters:
        iters = first
        c, a, obj, flags = oracle.vq_kmeans(x16, u, iters)
    return iters, c, a, obj, flags


@pytest.mark.parametrize("method", [TC, SIMT])
@pytest.mark.parametrize("deg,n,K", [(3, 9001, 512), (2, 7003, 256), (1, 5000, 768), (0, 3001, 256)])
def test_assignment_matches_oracle(method, deg, n, K):
    """Operand widths 64, 32, 16 (degree 3, 2, 1/0) with a ragged last tile."""
    from paper_2411_00771_gb300 import binding as B
    sh, keep = _sh_set(n, deg, seed=deg * 10 + method)
    quant = keep == 0
    x16 = oracle.vq_vectors(sh, quant)
    rng = np.random.default_rng(deg + 100)
    c16 = _near_data(x16, K, rng)
    got = B.vq_assign(_dev(sh), deg, _dev(keep), _dev(c16), method=method).cpu().numpy()
    assert np.all(got[~quant] == -1)
    _check_assign(got[quant].astype(np.int64), x16, c16)


def test_assignment_with_the_paper_codebook_size():
    """K = 8192 entries (Appendix C) on the tensor cores."""
    from paper_2411_00771_gb300 import binding as B
    sh, keep = _sh_set(6000, 3, seed=5)
    quant = keep == 0
    x16 = oracle.vq_vectors(sh, quant)
    rng = np.random.default_rng(6)
    c16 = oracle.half(x16.astype(np.float64) + rng.normal(0, 0.02, (x16.shape[0], 48)))
    c16 = c16[rng.choice(c16.shape[0], 2048, replace=False)]
    c16 = np.concatenate([c16, oracle.half(rng.normal(0, 0.5, (8192 - 2048, 48)))])
    got = B.vq_assign(_dev(sh), 3, _dev(keep), _dev(c16), method=TC).cpu().numpy()
    _check_assign(got[quant].astype(np.int64), x16, c16)


@pytest.mark.parametrize("method", [TC, SIMT])
def test_kmeans_matches_oracle_bit_for_bit(method):
    """Lloyd's steps from the same draws: the same codebook, bit for bit, the
    same assignment and objective, as long as no step met a near-tie."""
    from paper_2411_00771_gb300 import binding as B
    # zero-mean coefficients: small scores, so these draws meet no near-tie
    # in any of the 4 steps (the oracle asserts it below)
    rng = np.random.default_rng(10)
    sh = rng.normal(0, 0.05, (8000, 16, 3)).astype(np.float32)
    keep = (rng.random(8000) < 0.6).astype(np.uint8)
    quant = keep == 0
    x16 = oracle.vq_vectors(sh, quant)
    K, iters = 256, 4
    u = np.random.default_rng(11).random(K, dtype=np.float32)
    c_ref, a_ref, obj_ref, flags = oracle.vq_kmeans(x16, u, iters)
    assert not any(f.any() for f in flags)
    cb, assign, obj, m = B.vq_kmeans(_dev(sh), 3, _dev(keep), K=K, iters=iters, init_u=_dev(u), method=method)
    assert m == quant.sum()
    assert np.array_equal(cb.cpu().numpy().view(np.uint16), c_ref.view(np.uint16))
    got = assign.cpu().numpy()
    assert np.all(got[~quant] == -1)
    assert np.array_equal(got[quant], a_ref)
    assert np.allclose(obj.cpu().numpy(), obj_ref, rtol=1e-9, atol=1e-9)


def test_kmeans_steps_until_the_first_near_tie_on_city_like_data():
    """DC-heavy SH (albedo-like colours): bit-for-bit up to the oracle's first
    near-tie, then the assignment off the flagged vectors."""
    from paper_2411_00771_gb300 import binding as B
    sh, keep = _sh_set(12000, 3, seed=7)
    x16 = oracle.vq_vectors(sh, keep == 0)
    u = np.random.default_rng(8).random(256, dtype=np.float32)
    iters, c_ref, a_ref, obj_ref, flags = _steps_without_ties(x16, u, 4)
    cb, assign, obj, m = B.vq_kmeans(_dev(sh), 3, _dev(keep), K=256, iters=iters, init_u=_dev(u), method=TC)
    assert np.array_equal(cb.cpu().numpy().view(np.uint16), c_ref.view(np.uint16))
    got = assign.cpu().numpy()[keep == 0]
    assert np.array_equal(got[~flags[-1]], a_ref[~flags[-1]])


def test_kmeans_objective_never_rises_and_paths_agree():
    """Lloyd's property on the GPU, and the tensor-core and CUDA-core
    assignments agree wherever the oracle sees no near-tie."""
    from paper_2411_00771_gb300 import binding as B
    sh, keep = _sh_set(40000, 2, seed=9, keep_frac=0.5)
    u = _dev(np.random.default_rng(10).random(512, dtype=np.float32))
    cb1, a1, o1, _ = B.vq_kmeans(_dev(sh), 2, _dev(keep), K=512, iters=6, init_u=u, method=TC)
    cb2, a2, o2, _ = B.vq_kmeans(_dev(sh), 2, _dev(keep), K=512, iters=6, init_u=u, method=SIMT)
    o1 = o1.cpu().numpy()
    m = int((keep == 0).sum())
    assert np.all(np.diff(o1) <= m * 27 * (2.0 ** -11 * 4) ** 2), np.diff(o1)
    assert o1[-1] < 0.9 * o1[0]
    # same codebook unless a near-tie went differently somewhere
    same = np.array_equal(cb1.cpu().numpy().view(np.uint16), cb2.cpu().numpy().view(np.uint16))
    if same:
        assert np.mean(a1.cpu().numpy() != a2.cpu().numpy()) < 0.002


def test_kmeans_degenerate_sizes():
    from paper_2411_00771_gb300 import binding as B
    sh, _ = _sh_set(500, 1, seed=11)
    # nothing quantised
    cb, assign, obj, m = B.vq_kmeans(_dev(sh), 1, _dev(np.ones(500, np.uint8)), K=256, iters=2)
    assert m == 0 and np.all(assign.cpu().numpy() == -1) and not cb.float().abs().sum().item()
    assert np.all(obj.cpu().numpy() == 0)
    # more entries than vectors (some entries repeat, some stay unused)
    keep = np.ones(500, np.uint8)
    keep[:100] = 0
    u = np.random.default_rng(12).random(512, dtype=np.float32)
    cb, assign, obj, m = B.vq_kmeans(_dev(sh), 1, _dev(keep), K=512, iters=2, init_u=_dev(u), method=TC)
    x16 = oracle.vq_vectors(sh, keep == 0)
    c_ref, a_ref, o_ref, flags = oracle.vq_kmeans(x16, u, 2)
    assert np.array_equal(cb.cpu().numpy().view(np.uint16), c_ref.view(np.uint16))
    assert np.allclose(obj.cpu().numpy(), o_ref, rtol=1e-9, atol=1e-12)
    assert float(obj[-1]) == 0.0  # every vector is its own entry's value
    # K not a multiple of 256 on the tensor cores is refused; the CUDA cores take it
    with pytest.raises(B.GsError):
        B.vq_kmeans(_dev(sh), 1, _dev(keep), K=300, iters=1, method=TC)
    cb, assign, _, _ = B.vq_kmeans(_dev(sh), 1, _dev(keep), K=300, iters=1, method=0)
    assert assign.cpu().numpy()[:100].max() < 300


def _compressed(scene, contrib, K=256, iters=2, seed=13, method=TC):
    from paper_2411_00771_gb300 import binding as B
    d = gu.to_dev(scene)
    params = tuple(d[k] for k in ("mu", "quat", "scale", "opacity", "sh"))
    u = np.random.default_rng(seed).random(K, dtype=np.float32)
    comp, info = B.compress(params, scene["sh_degree"], _dev(contrib), ratio=0.4, K=K, iters=iters, init_u=_dev(u),
                            method=method)
    return comp, info, u


def test_compressed_layout_matches_oracle():
    scene, cam, _, _ = syn.tiny_scene(seed=14, n=4000, sh_degree=3)
    contrib = np.random.default_rng(15).exponential(0.1, 4000).astype(np.float32)
    comp, info, u = _compressed(scene, contrib, seed=16)
    quant = oracle.vq_quantized(contrib, 0.4)
    assert np.array_equal(info["keep"].cpu().numpy() == 0, quant)
    x16 = oracle.vq_vectors(scene["sh"], quant)
    c_ref, a_ref, _, flags = oracle.vq_kmeans(x16, u, 2)
    assert not any(f.any() for f in flags)  # these draws meet no near-tie
    ref = oracle.vq_compress(scene, quant, c_ref, a_ref)
    for k in ("quat", "scale", "opacity", "sh_table"):
        g = comp[k].cpu().numpy()
        assert np.array_equal(g.view(np.uint16), ref[k].reshape(g.shape).view(np.uint16)), k
    assert np.array_equal(comp["sh_row"].cpu().numpy(), ref["sh_row"])
    # bytes per surfel: FP32 236 (SH 3) against binary16 + one row index
    n = 4000
    full = n * (3 + 4 + 2 + 1 + 48) * 4
    packed = n * (12 + 8 + 4 + 2 + 4) + comp["sh_table"].numel() * 2
    assert packed < 0.45 * full


def test_render_from_compressed_scene():
    """The compressed scene renders exactly as the FP32 scene holding the
    same binary16 values, and matches the oracle's render of the decompressed
    scene."""
    from paper_2411_00771_gb300 import binding as B
    scene, cam, _, _ = syn.tiny_scene(seed=16, n=3000, sh_degree=3)
    contrib = np.random.default_rng(17).exponential(0.1, 3000).astype(np.float32)
    comp, info, u = _compressed(scene, contrib, seed=14)
    csc = B.CompressedScene(comp)
    H, W = cam["height"], cam["width"]
    cnt_c = torch.empty((H, W), dtype=torch.int32, device="cuda")
    out_c, _ = csc.render(cam, n_contrib=cnt_c, save=False)
    # the FP32 scene of the same values
    fp = {"mu": comp["mu"], "quat": comp["quat"].float().contiguous(), "scale": comp["scale"].float().contiguous(),
          "opacity": comp["opacity"].float().contiguous(),
          "sh": comp["sh_table"][comp["sh_row"].long()].float().reshape(3000, 16, 3).contiguous()}
    fsc = B.Scene(fp["mu"], fp["quat"], fp["scale"], fp["opacity"], fp["sh"], 3)
    cnt_f = torch.empty((H, W), dtype=torch.int32, device="cuda")
    out_f, _ = fsc.render(cam, n_contrib=cnt_f, save=False)
    torch.cuda.synchronize()
    assert torch.equal(out_c, out_f) and torch.equal(cnt_c, cnt_f)
    # against the oracle's render of its own decompressed scene
    quant = oracle.vq_quantized(contrib, 0.4)
    x16 = oracle.vq_vectors(scene["sh"], quant)
    c_ref, a_ref, _, flags = oracle.vq_kmeans(x16, u, 2)
    assert not any(f.any() for f in flags)  # these draws meet no near-tie
    dec = oracle.vq_decompress(oracle.vq_compress(scene, quant, c_ref, a_ref))
    ref = oracle.render(dec, cam)
    any_flag = oracle.FLAG_ALPHA | oracle.FLAG_RHO | oracle.FLAG_TSTOP | oracle.FLAG_MEDIAN
    ok = (ref["flags"] & any_flag) == 0
    assert ok.mean() >= 0.99
    g = out_c.cpu().numpy()
    branch = (ref["flags"] & oracle.FLAG_BRANCH) != 0
    v = gu.plane_violations(g, ref["out"], ok)
    v_nb = gu.plane_violations(g, ref["out"], ok & ~branch)
    for p, name in enumerate(gu.PLANES):
        e = v_nb[p] if p in gu.DEPTH_PLANES else v[p]
        assert e <= 1.0, (name, e)
    assert np.array_equal(cnt_c.cpu().numpy()[ok], ref["count"][ok])


def test_compressed_scene_serves_and_counts_contribution():
    from paper_2411_00771_gb300 import binding as B
    scene, cam, _, _ = syn.tiny_scene(seed=18, n=2000, sh_degree=2)
    contrib = np.random.default_rng(19).exponential(0.1, 2000).astype(np.float32)
    comp, _, _ = _compressed(scene, contrib, method=SIMT)
    csc = B.CompressedScene(comp)
    lone, _ = csc.render(cam, save=False)
    srv = B.Server(1 << 30, max_slots=2)
    sid = srv.add_scene(csc)
    out = torch.empty_like(lone)
    t = srv.submit(sid, cam, out)
    srv.wait(t)
    torch.cuda.synchronize()
    assert torch.equal(out, lone)
    srv.close()
    s = torch.zeros(2000, device="cuda")
    csc.contribution(cam, contrib=s)
    torch.cuda.synchronize()
    assert float(s.sum()) > 0


def test_compressed_scene_is_render_only_and_checked():
    from paper_2411_00771_gb300 import binding as B
    scene, cam, _, _ = syn.tiny_scene(seed=20, n=800, sh_degree=1)
    contrib = np.random.default_rng(21).exponential(0.1, 800).astype(np.float32)
    comp, _, _ = _compressed(scene, contrib, method=SIMT)
    csc = B.CompressedScene(comp)
    out, frame = csc.render(cam)
    grads = {k: torch.zeros(1, device="cuda") for k in ("mu", "quat", "scale", "opacity", "sh")}
    with pytest.raises(B.GsError):
        csc.backward(frame, [torch.zeros((11,) + tuple(out.shape[1:]), device="cuda")], [0x7FF], grads)
    frame.release()
    bad = dict(comp)
    bad["sh_row"] = comp["sh_row"].clone()
    bad["sh_row"][5] = comp["sh_table"].shape[0]  # one past the table
    with pytest.raises(B.GsError):
        B.CompressedScene(bad)
    mis = dict(comp)
    buf = torch.zeros(800 * 4 + 1, dtype=torch.float16, device="cuda")
    mis["quat"] = buf[1:].view(800, 4)  # 2-byte offset: not 8-byte aligned
    with pytest.raises(B.GsError):
        B.CompressedScene(mis)


def test_full_size_assignment_properties():
    """The 4M-surfel city size: 1.6 M quantised vectors of degree 3 against
    8192 entries.  On 3000 sampled vectors the entry is the nearest of the
    returned codebook (up to the FP32 evaluation error), and Lloyd's
    objective does not rise."""
    from paper_2411_00771_gb300 import binding as B
    n = 4_000_000
    rng = np.random.default_rng(22)
    sh = rng.normal(0, 0.05, (n, 16, 3)).astype(np.float32)
    sh[:, 0, :] = rng.uniform(-1.0, 1.5, (n, 1)) + rng.normal(0, 0.1, (n, 3))
    contrib = rng.exponential(0.1, n).astype(np.float32)
    keep, _ = B.prune_by_contribution(_dev(contrib), 0.4)
    u = _dev(rng.random(8192, dtype=np.float32))
    cb, assign, obj, m = B.vq_kmeans(_dev(sh), 3, keep, K=8192, iters=2, init_u=u, method=TC)
    assert m == math.ceil(0.4 * n)
    o = obj.cpu().numpy()
    assert np.all(np.diff(o) <= m * 48 * (2.0 ** -11 * 4) ** 2)
    a = assign.cpu().numpy()
    q = np.nonzero(a >= 0)[0]
    assert q.size == m
    pick = rng.choice(q, 3000, replace=False)
    x = oracle.half(sh[pick].reshape(3000, 48)).astype(np.float64)
    c = cb.cpu().numpy().astype(np.float64)
    score = (c * c).sum(1)[None, :] - 2 * x @ c.T
    best = score.min(1)
    mine = score[np.arange(3000), a[pick]]
    eps = 4 * 2.0 ** -17 * ((c * c).sum(1).max() + 2 * np.abs(x) @ np.abs(c).max(0))
    assert np.all(mine - best <= eps)
