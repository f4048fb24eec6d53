"""Serving loop through the C ABI: requests with host buffers, mixed shape
buckets and scenes, several lanes in flight.  Each request's image must equal
glassnet_render_host of the same inputs alone, bit for bit, whatever the mix,
the admission budget or the lane it ran on."""
import numpy as np
import pytest
import torch

from gen import synth
from paper_2405_19056_gb300 import glassnet as gl

pytestmark = pytest.mark.gpu


def _pin(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory()


@pytest.fixture(scope="module")
def model(cuda_lib):
    return gl.Model(synth.make_weights(synth.DOUBLED_WIDTHS, seed=0), gl.GN_BF16_FUSED)


SHAPES = [(64, 64), (128, 128), (96, 80), (33, 47)]


def _requests(n, seed, n_scenes):
    rng = np.random.default_rng([seed, 6])
    reqs = []
    for i in range(n):
        h, w = SHAPES[int(rng.integers(len(SHAPES)))]
        K = int(rng.integers(1, 9))
        f = synth.make_frame(h, w, K, counts="uniform", seed=700 + seed * 100 + i)
        reqs.append(dict(scene=i % n_scenes, h=h, w=w, K=K, g=_pin(f.gbuf), t=_pin(f.tbuf),
                         c=_pin(f.counts), out=torch.full((3, h, w), float("nan")).pin_memory()))
    return reqs


def _alone(model, lat, r):
    out = torch.full((3, r["h"], r["w"]), float("nan")).pin_memory()
    gl.glassnet_render_host(model.handle, lat.handle, r["g"], r["t"], r["c"], r["K"], r["h"],
                            r["w"], out)
    return out.numpy().copy()


def _serve(model, reqs, scene_ids, **cfg):
    srv = gl.glassnet_server_create(model.handle, **cfg)
    try:
        ids = [gl.glassnet_server_add_scene(srv, synth.make_scene(s)) for s in scene_ids]
        tickets = [gl.glassnet_server_submit(srv, ids[r["scene"]], r["g"], r["t"], r["c"], r["K"],
                                             r["h"], r["w"], r["out"]) for r in reqs]
        lat = [gl.glassnet_server_wait(srv, t) for t in tickets]
        stats = gl.glassnet_server_stats(srv)
    finally:
        gl.glassnet_server_destroy(srv)
    return lat, stats


def test_mixed_requests_equal_alone(model):
    scenes = [11, 12, 13]
    reqs = _requests(24, seed=1, n_scenes=len(scenes))
    lats, stats = _serve(model, reqs, scenes, n_streams=4, max_scenes=4, max_h=128, max_w=128,
                         max_K=8)
    model.check()
    assert stats["submitted"] == 24 and stats["completed"] == 24
    assert stats["pixels"] == sum(r["h"] * r["w"] for r in reqs)
    assert 0 < stats["p50_ms"] <= stats["p99_ms"] <= stats["max_ms"]
    assert all(l > 0 for l in lats)
    latents = [model.encode(synth.make_scene(s)) for s in scenes]
    for i, r in enumerate(reqs):
        assert np.array_equal(r["out"].numpy(), _alone(model, latents[r["scene"]], r)), i


def test_many_requests_in_flight_each_equal_alone(model):
    """300 requests of one size submitted at once, K alternating 8 and 1, four
    lanes: a lane's arena then holds a K = 8 layer buffer where the next
    K = 1 request keeps its counts, so a lane handed a new request before its
    previous one had finished would mix them (and report a count above K).
    A lane is free again only after its own request's event completed: every
    image equals its request rendered alone and no device error is set."""
    scene = 21
    reqs = []
    for i in range(300):
        K = 8 if i % 2 == 0 else 1
        f = synth.make_frame(96, 96, K, counts="all", seed=900 + i % 6)
        reqs.append(dict(scene=0, h=96, w=96, K=K, g=_pin(f.gbuf), t=_pin(f.tbuf), c=_pin(f.counts),
                         out=torch.full((3, 96, 96), float("nan")).pin_memory()))
    lats, stats = _serve(model, reqs, [scene], n_streams=4, max_scenes=2, max_h=96, max_w=96,
                         max_K=8)
    model.check()
    assert stats["completed"] == 300
    lat = model.encode(synth.make_scene(scene))
    alone = {}
    for i, r in enumerate(reqs):
        key = (r["K"], i % 6)
        if key not in alone:
            alone[key] = _alone(model, lat, r)
        assert np.array_equal(r["out"].numpy(), alone[key]), i


def test_budget_of_one_request_serialises_admission(model):
    reqs = _requests(10, seed=2, n_scenes=1)
    one = 128 * 128 * (14 * 4 + 12 * 4 * 8 + 1 + 3 * 4) + 4 * 256  # the largest request, padded
    lats, stats = _serve(model, reqs, [21], n_streams=4, max_scenes=1, max_h=128, max_w=128,
                         max_K=8, budget_bytes=one)
    assert stats["completed"] == 10
    lat = model.encode(synth.make_scene(21))
    for r in reqs:
        assert np.array_equal(r["out"].numpy(), _alone(model, lat, r))


def test_least_recently_used_scene_is_replaced(model):
    srv = gl.glassnet_server_create(model.handle, n_streams=2, max_scenes=2, max_h=64, max_w=64,
                                    max_K=4)
    try:
        a = gl.glassnet_server_add_scene(srv, synth.make_scene(31))
        b = gl.glassnet_server_add_scene(srv, synth.make_scene(32))
        c = gl.glassnet_server_add_scene(srv, synth.make_scene(33))  # replaces a
        assert len({a, b, c}) == 3
        f = synth.make_frame(64, 64, 4, counts="uniform", seed=9)
        r = dict(h=64, w=64, K=4, g=_pin(f.gbuf), t=_pin(f.tbuf), c=_pin(f.counts),
                 out=torch.empty((3, 64, 64)).pin_memory())
        with pytest.raises(gl.GlassNetError) as ei:
            gl.glassnet_server_submit(srv, a, r["g"], r["t"], r["c"], 4, 64, 64, r["out"])
        assert ei.value.code == gl.GN_EINVAL
        t = gl.glassnet_server_submit(srv, c, r["g"], r["t"], r["c"], 4, 64, 64, r["out"])
        gl.glassnet_server_wait(srv, t)
        assert np.array_equal(r["out"].numpy(), _alone(model, model.encode(synth.make_scene(33)), r))
        with pytest.raises(gl.GlassNetError):  # larger than the server's maximum
            gl.glassnet_server_submit(srv, c, r["g"], r["t"], r["c"], 8, 64, 64, r["out"])
    finally:
        gl.glassnet_server_destroy(srv)


@pytest.mark.parametrize("form", ["sum", "r3", "pe", "pe128"])
def test_model_options_served_equal_alone(cuda_lib, form):
    """The serving loop with the model options (sum pooling, a 3x3 R whose
    per-lane graphs hold a neural buffer, positional encoding at H = 64 and
    at H = 128, where the per-pixel weights stream): each request equals its
    render alone, bit for bit."""
    if form == "pe":
        w = synth.make_weights(synth.Widths(64, 128, 4), seed=2, bias="uniform")
    elif form == "pe128":
        w = synth.make_weights(synth.Widths(128, 256, 3), seed=2, bias="uniform")
    else:
        w = synth.make_weights(synth.Widths(128, 256, 0, 3 if form == "r3" else 1), seed=2, bias="uniform")
    m = gl.Model(w, gl.GN_BF16_FUSED, gl.GN_POOL_SUM if form == "sum" else gl.GN_POOL_MAX_MEAN)
    scenes = [21, 22]
    reqs = _requests(10, seed=3, n_scenes=len(scenes))
    _serve(m, reqs, scenes, n_streams=2, max_scenes=2, max_h=128, max_w=128, max_K=8)
    m.check()
    latents = [m.encode(synth.make_scene(s)) for s in scenes]
    for i, r in enumerate(reqs):
        assert np.array_equal(r["out"].numpy(), _alone(m, latents[r["scene"]], r)), (form, i)


def test_concurrent_add_scene_takes_distinct_slots(model):
    """Scenes added from several threads at once: every call gets its own
    slot and id, and every id stays resident and renders its own scene."""
    import threading
    srv = gl.glassnet_server_create(model.handle, n_streams=2, max_scenes=8, max_h=32, max_w=32,
                                    max_K=2)
    try:
        ids, errs = {}, []

        def add(s):
            try:
                ids[s] = gl.glassnet_server_add_scene(srv, synth.make_scene(s))
            except Exception as e:  # noqa: BLE001 - reported below
                errs.append(e)
        threads = [threading.Thread(target=add, args=(40 + i,)) for i in range(8)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errs, errs
        assert len(set(ids.values())) == 8
        f = synth.make_frame(32, 32, 2, counts="uniform", seed=19)
        r = dict(h=32, w=32, K=2, g=_pin(f.gbuf), t=_pin(f.tbuf), c=_pin(f.counts))
        for s, sid in ids.items():
            out = torch.full((3, 32, 32), float("nan")).pin_memory()
            gl.glassnet_server_wait(srv, gl.glassnet_server_submit(srv, sid, r["g"], r["t"], r["c"],
                                                                   2, 32, 32, out))
            assert np.array_equal(out.numpy(), _alone(model, model.encode(synth.make_scene(s)),
                                                      dict(r, out=out))), s
    finally:
        gl.glassnet_server_destroy(srv)


def test_prepared_buckets_serve_equal_alone(model):
    """glassnet_server_prepare captures a bucket's graph on every lane; a
    bucket beyond the server's maximum is refused; requests of prepared
    buckets equal the same inputs rendered alone."""
    srv = gl.glassnet_server_create(model.handle, n_streams=3, max_scenes=1, max_h=64, max_w=64,
                                    max_K=4)
    try:
        sid = gl.glassnet_server_add_scene(srv, synth.make_scene(50))
        for K in (1, 4):
            gl.glassnet_server_prepare(srv, 64, 64, K)
        with pytest.raises(gl.GlassNetError) as ei:
            gl.glassnet_server_prepare(srv, 64, 64, 5)  # K above the server's maximum
        assert ei.value.code == gl.GN_EINVAL
        lat = model.encode(synth.make_scene(50))
        reqs = []
        for i, K in enumerate((1, 4, 4, 1, 4, 1)):
            f = synth.make_frame(64, 64, K, counts="uniform", seed=80 + i)
            reqs.append(dict(h=64, w=64, K=K, g=_pin(f.gbuf), t=_pin(f.tbuf), c=_pin(f.counts),
                             out=torch.full((3, 64, 64), float("nan")).pin_memory()))
        tickets = [gl.glassnet_server_submit(srv, sid, r["g"], r["t"], r["c"], r["K"], 64, 64, r["out"])
                   for r in reqs]
        for t in tickets:
            gl.glassnet_server_wait(srv, t)
        for r in reqs:
            assert np.array_equal(r["out"].numpy(), _alone(model, lat, r))
    finally:
        gl.glassnet_server_destroy(srv)
