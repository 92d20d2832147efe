"""Serving loop (continuous batching over resident scenes) on the GPU.

Requests of mixed resolutions and scenes, submitted concurrently from
several client threads, must produce exactly the images a lone gs_render
produces; admission respects the memory budget; failures (a request that
can never fit, an allocator that fails) are reported per request while the
server keeps serving; a timed-out wait leaves the ticket valid.
"""
import ctypes
import math
import threading

import numpy as np
import pytest
import torch

from paper_2411_00771_gb300 import synthetic as syn
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu

RES = [(64, 48), (100, 75), (128, 128), (37, 29), (256, 144)]


def _cams(rng, count):
    cams = []
    for _ in range(count):
        W, H = RES[rng.integers(len(RES))]
        yaw = rng.uniform(-0.25, 0.25)
        pitch = rng.uniform(-0.2, 0.2)
        cy, sy, cp, sp = math.cos(yaw), math.sin(yaw), math.cos(pitch), math.sin(pitch)
        Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
        Rx = np.array([[1, 0, 0], [0, cp, -sp], [0, sp, cp]])
        R = Rx @ Ry
        cam = dict(R=R, t=np.array([rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), 0.5]),
                   fx=0.9 * W, fy=0.9 * W, cx=W / 2, cy=H / 2, width=W, height=H)
        cams.append(cam)
    return cams


@pytest.fixture(scope="module")
def scenes():
    a, _, _, _ = syn.tiny_scene(seed=501, n=4000, sh_degree=3, log_scale_range=(-4.5, -2.0))
    b, _, _, _ = syn.tiny_scene(seed=502, n=1500, sh_degree=1, log_scale_range=(-3.5, -1.5))
    return [gu.gpu_scene(a), gu.gpu_scene(b)]


def _reference(scenes, reqs):
    refs = []
    for sid, cam in reqs:
        sc = scenes[sid][0]
        cnt = torch.empty((cam["height"], cam["width"]), dtype=torch.int32, device="cuda")
        out, _ = sc.render(cam, n_contrib=cnt, save=False)
        refs.append((out, cnt))
    torch.cuda.synchronize()
    return refs


def test_served_renders_equal_single_renders(scenes):
    from paper_2411_00771_gb300 import binding as B
    rng = np.random.default_rng(7)
    cams = _cams(rng, 40)
    reqs = [(int(rng.integers(2)), c) for c in cams]
    refs = _reference(scenes, reqs)
    srv = B.Server(budget_bytes=1 << 30, max_slots=6)
    ids = [srv.add_scene(s[0]) for s in scenes]
    outs = [None] * len(reqs)

    def client(k):
        for i in range(k, len(reqs), 4):
            sid, cam = reqs[i]
            out = torch.full((12, cam["height"], cam["width"]), float("nan"), device="cuda")
            cnt = torch.full((cam["height"], cam["width"]), -1, dtype=torch.int32, device="cuda")
            t = srv.submit(ids[sid], cam, out, cnt)
            srv.wait(t, 60000)
            outs[i] = (out, cnt)

    torch.cuda.synchronize()
    th = [threading.Thread(target=client, args=(k,)) for k in range(4)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    for i, ((o, c), (ro, rc)) in enumerate(zip(outs, refs)):
        assert torch.equal(o, ro), i
        assert torch.equal(c, rc), i
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["batches"] >= 1 and st["batched_views"] == len(reqs)
    assert st["latency_p99_ms"] >= st["latency_p50_ms"] > 0
    srv.close()


def test_admission_under_a_tight_budget(scenes):
    """A budget that holds about one request's buffers: requests queue and
    complete one after another, still exact."""
    from paper_2411_00771_gb300 import binding as B
    rng = np.random.default_rng(8)
    cams = _cams(rng, 8)
    reqs = [(0, c) for c in cams]
    refs = _reference(scenes, reqs)
    srv = B.Server(budget_bytes=4 << 20, max_slots=4)
    sid = srv.add_scene(scenes[0][0])
    outs = []
    tickets = []
    for _, cam in reqs:
        out = torch.zeros((12, cam["height"], cam["width"]), device="cuda")
        outs.append(out)
        tickets.append(srv.submit(sid, cam, out))
    for t in tickets:
        srv.wait(t, 60000)
    torch.cuda.synchronize()
    for o, (ro, _) in zip(outs, refs):
        assert torch.equal(o, ro)
    assert srv.stats()["bytes_in_use"] <= 4 << 20
    srv.close()


def test_request_that_cannot_fit_fails_and_server_continues(scenes):
    from paper_2411_00771_gb300 import binding as B
    srv = B.Server(budget_bytes=256 << 10, max_slots=2)
    big = srv.add_scene(scenes[0][0])      # 4000 surfels need more than 256 KB
    small_scene, _ = gu.gpu_scene(syn.tiny_scene(seed=9, n=40, width=16, height=16, fx=16.0)[0])
    small = srv.add_scene(small_scene)
    cam = dict(R=np.eye(3), t=np.zeros(3), fx=16.0, fy=16.0, cx=8.0, cy=8.0, width=16, height=16)
    out = torch.zeros((12, 16, 16), device="cuda")
    t = srv.submit(big, cam, out)
    with pytest.raises(B.GsError) as e:
        srv.wait(t, 60000)
    assert e.value.code == -3
    ref, _ = small_scene.render(cam, save=False)
    t2 = srv.submit(small, cam, out)
    srv.wait(t2, 60000)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert srv.stats()["failed"] == 1
    srv.close()


def test_allocator_failure_is_reported_per_request(scenes):
    """Fault injection on the host: the allocator refuses the third
    allocation; that request fails with GS_ERR_OOM, later ones succeed."""
    from paper_2411_00771_gb300 import binding as B
    state = {"calls": 0, "fail_at": 3, "live": {}}

    def alloc(size, ctx, stream):
        state["calls"] += 1
        if state["calls"] == state["fail_at"]:
            return None
        t = torch.empty(int(size), dtype=torch.uint8, device="cuda")
        state["live"][t.data_ptr()] = t
        return t.data_ptr()

    def free(ptr, size, ctx, stream):
        torch.cuda.synchronize()
        state["live"].pop(ptr, None)

    al = B.gs_allocator(B.ALLOC_FN(alloc), B.FREE_FN(free), None)
    srv = B.Server(budget_bytes=1 << 30, max_slots=1, allocator=al)
    sid = srv.add_scene(scenes[1][0])
    cam = _cams(np.random.default_rng(3), 1)[0]
    ref, _ = scenes[1][0].render(cam, save=False)
    out = torch.zeros_like(ref)
    t = srv.submit(sid, cam, out)
    with pytest.raises(B.GsError) as e:
        srv.wait(t, 60000)
    assert e.value.code == -2
    t = srv.submit(sid, cam, out)
    srv.wait(t, 60000)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    srv.close()


def test_wait_timeout_keeps_the_ticket(scenes):
    from paper_2411_00771_gb300 import binding as B
    srv = B.Server(budget_bytes=1 << 30, max_slots=2)
    sid = srv.add_scene(scenes[0][0])
    cams = _cams(np.random.default_rng(4), 6)
    outs = [torch.zeros((12, c["height"], c["width"]), device="cuda") for c in cams]
    ts = [srv.submit(sid, c, o) for c, o in zip(cams, outs)]
    last = ts[-1]
    try:
        srv.wait(last, 0)
        timed_out = False
    except B.GsError as e:
        assert e.code == -5
        timed_out = True
    if timed_out:
        srv.wait(last, 60000)
    for t in ts[:-1]:
        srv.wait(t, 60000)
    with pytest.raises(B.GsError):
        srv.wait(last, 0)  # consumed
    srv.close()


def test_served_small_view_with_long_lists_equals_single_render():
    """A view with few tiles and long lists is composited in segments by both
    paths; the served image equals the lone render bit for bit."""
    from paper_2411_00771_gb300 import binding as B
    scene, cam, _, _ = syn.tiny_scene(seed=77, n=30000, width=64, height=64, fx=64.0, sh_degree=1,
                                      log_scale_range=(-4.0, -2.5))
    sc, _ = gu.gpu_scene(scene)
    cnt_ref = torch.empty((64, 64), dtype=torch.int32, device="cuda")
    ref, _ = sc.render(cam, n_contrib=cnt_ref, save=False)
    srv = B.Server(budget_bytes=1 << 30, max_slots=2)
    sid = srv.add_scene(sc)
    out = torch.full((12, 64, 64), float("nan"), device="cuda")
    cnt = torch.full((64, 64), -1, dtype=torch.int32, device="cuda")
    srv.wait(srv.submit(sid, cam, out, cnt), 60000)
    torch.cuda.synchronize()
    assert torch.equal(out, ref) and torch.equal(cnt, cnt_ref)
    srv.close()
