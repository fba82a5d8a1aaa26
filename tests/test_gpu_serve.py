"""The serving loop: each request's result is the same alone and in a mix whose
requests overlap on the device or share launches with requests of other scenes,
admission keeps the working sets within the HBM budget, and the plain loop
serves in arrival order.

Results are compared within the tolerances of the parity tests (the reverse
pass adds with float atomics, so runs agree to rounding, not bit for bit).
"""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def scenes():
    from paper_2602_00395_gb300.serve import Scene
    return [Scene(0, 20000, 256, 256, n_views=4), Scene(1, 30000, 320, 240, n_views=4),
            Scene(2, 15000, 256, 192, n_views=4), Scene(3, 9000, 256, 256, n_views=4)]


def _snapshot(sc):
    return [b.clone() for b in (sc.x, sc.g_ema, sc.d_ema)], sc.t


def _restore(sc, snap):
    bufs, t = snap
    for b, v in zip((sc.x, sc.g_ema, sc.d_ema), bufs):
        b.copy_(v)
    sc.t = t
    torch.cuda.synchronize()


def _close(a, b, rel):
    scale = float(b.abs().max()) + 1e-30
    assert float((a - b).abs().max()) <= rel * scale


def test_results_equal_alone_and_in_the_mix(scenes):
    from paper_2602_00395_gb300.serve import Server
    snaps = [_snapshot(sc) for sc in scenes]
    mine = [(0.0, "train", 0, 1), (0.0, "train", 0, 2), (0.0, "render", 0, 3)]
    alone = Server(scenes, slots=4).run(mine, keep_results=True)
    ref_state = [b.clone() for b in (scenes[0].x, scenes[0].g_ema, scenes[0].d_ema)]
    ref_image = alone.requests[2].image.clone()
    assert set(alone.summary()["status_words"]) == {0}
    for sc, sn in zip(scenes, snaps):
        _restore(sc, sn)
    mix = [(0.0, "train", 1, 0), (0.0, "train", 0, 1), (0.0, "render", 2, 1), (0.0, "train", 2, 2),
           (0.0, "train", 0, 2), (0.0, "train", 1, 3), (0.0, "render", 0, 3), (0.0, "render", 1, 1)]
    res = Server(scenes, slots=4).run(mix, keep_results=True)
    assert set(res.summary()["status_words"]) == {0}
    # requests of different scenes were on the device together
    reqs = res.requests
    assert any(a.start < b.done and b.start < a.done for i, a in enumerate(reqs) for b in reqs[i + 1:]
               if a.scene != b.scene)
    for got, want in zip((scenes[0].x, scenes[0].g_ema, scenes[0].d_ema), ref_state):
        _close(got, want, 1e-4)
    img = [r for r in reqs if r.scene == 0 and r.kind == "render"][0].image
    assert float((img - ref_image).abs().max()) <= 1e-5
    for sc, sn in zip(scenes, snaps):
        _restore(sc, sn)


def test_requests_of_several_scenes_sharing_launches_equal_each_alone(scenes):
    """Training steps of scenes 0 and 3 (same image size, 20k and 9k Gaussians)
    waiting together start as one batch; every scene's state and every render
    equals what it gets served alone."""
    from paper_2602_00395_gb300.serve import Server
    snaps = [_snapshot(sc) for sc in scenes]
    ref = {}
    for sid in (0, 3):
        Server(scenes, slots=2).run([(0.0, "train", sid, 1), (0.0, "train", sid, 2)])
        ref[sid] = [b.clone() for b in (scenes[sid].x, scenes[sid].g_ema, scenes[sid].d_ema)]
        img = Server(scenes, slots=2).run([(0.0, "render", sid, 3)], keep_results=True).requests[0].image.clone()
        ref[sid].append(img)
    for sc, sn in zip(scenes, snaps):
        _restore(sc, sn)
    spec = [(0.0, "train", 0, 1), (0.0, "train", 3, 1), (0.0, "train", 0, 2), (0.0, "train", 3, 2),
            (0.0, "render", 0, 3), (0.0, "render", 3, 3)]
    res = Server(scenes, slots=4).run(spec, keep_results=True)
    assert set(res.summary()["status_words"]) == {0}
    assert [r.batch for r in res.requests] == [2, 2, 2, 2, 2, 2]
    for sid in (0, 3):
        for got, want in zip((scenes[sid].x, scenes[sid].g_ema, scenes[sid].d_ema), ref[sid][:3]):
            _close(got, want, 1e-4)
        img = [r for r in res.requests if r.scene == sid and r.kind == "render"][0].image
        assert float((img - ref[sid][3]).abs().max()) <= 1e-5
    for sc, sn in zip(scenes, snaps):
        _restore(sc, sn)


def test_waiting_renders_of_a_scene_start_as_one_multi_view_render(scenes):
    """Renders of one scene that wait together start as one launch sequence and
    each image equals the one the plain loop renders alone; a training step of
    that scene between them splits the batch, and the render after it starts
    only when the step is done."""
    from paper_2602_00395_gb300.serve import Server, plain_loop
    snaps = [_snapshot(sc) for sc in scenes]
    spec = [(0.0, "render", 0, 0), (0.0, "render", 1, 2), (0.0, "render", 0, 3), (0.0, "render", 0, 1),
            (0.0, "train", 0, 2), (0.0, "render", 0, 0)]
    res = Server(scenes, slots=4).run(spec, keep_results=True)
    assert set(res.summary()["status_words"]) == {0}
    assert res.requests[5].start >= res.requests[4].done >= res.requests[4].start >= res.requests[0].done
    batch = {r.rid: r.batch for r in res.requests}
    assert batch[0] == batch[2] == batch[3] == 3 and batch[1] == 1 and batch[5] == 1
    after_train = res.requests[5].image.clone()
    for sc, sn in zip(scenes, snaps):
        _restore(sc, sn)
    ref = plain_loop(scenes, spec, keep_results=True)
    for r, q in zip(res.requests, ref.requests):
        if r.kind == "render" and r.rid != 5:
            assert torch.equal(r.image.view(-1), q.image.view(-1)), r.rid
    assert float((after_train.view(-1) - ref.requests[5].image.view(-1)).abs().max()) <= 1e-5
    for sc, sn in zip(scenes, snaps):
        _restore(sc, sn)


def test_admission_keeps_working_sets_within_the_budget(scenes):
    from paper_2602_00395_gb300.serve import Server
    snaps = [_snapshot(sc) for sc in scenes]
    from paper_2602_00395_gb300.serve import Request
    probe = Server(scenes, slots=1)
    sizes = sorted(probe.batch_bytes([Request(0, 0.0, "train", s, 0)]) for s in range(3))
    budget = sizes[-1] + sizes[0] // 2  # the largest fits, never two of the larger ones together
    spec = [(0.0, "train", s, v) for v in range(2) for s in range(3)]
    res = Server(scenes, slots=4, budget_bytes=budget).run(spec)
    assert res.peak_inflight_bytes <= budget
    assert all(r.done >= r.start >= r.arrival for r in res.requests)
    assert set(res.summary()["status_words"]) == {0}
    for sc, sn in zip(scenes, snaps):
        _restore(sc, sn)


def test_plain_loop_serves_in_arrival_order(scenes):
    from paper_2602_00395_gb300.serve import plain_loop
    snaps = [_snapshot(sc) for sc in scenes]
    spec = [(0.001 * k, "train" if k % 3 else "render", k % 3, k % 4) for k in range(9)]
    res = plain_loop(scenes, spec)
    starts = [r.start for r in res.requests]
    assert starts == sorted(starts)
    assert all(a.done <= b.start for a, b in zip(res.requests, res.requests[1:]))
    assert set(res.summary()["status_words"]) == {0}
    for sc, sn in zip(scenes, snaps):
        _restore(sc, sn)
