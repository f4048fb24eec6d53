"""Streaming (incremental) rendering through the C ABI: the pooled set
representation of Eq. 5 built one transparency layer at a time
(glassnet_accumulate_layer) and resolved once (glassnet_resolve).

The pooling is exact and order-independent, so for any frame and any order of
its layers the streamed result must equal glassnet_render of the frame, bit
for bit; through that, and directly on a small frame, it meets the FP64
oracle within the BF16 tolerance.  Layer k of a frame covers the pixels whose
count exceeds k.
"""
import numpy as np
import pytest
import torch

import oracle
from gen import synth
from paper_2405_19056_gb300 import glassnet as gl

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
BF16_MAX = 2e-2
BF16_MEAN = 3e-3


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def net(cuda_lib):
    w = synth.make_weights(synth.DOUBLED_WIDTHS, seed=0, bias="uniform")
    m = gl.Model(w, gl.GN_BF16_FUSED)
    return w, m, m.encode(synth.make_scene(3))


def _render(m, lat, f):
    out = torch.full((3, f.h, f.w), float("nan"), device=DEV)
    m.render(lat, _dev(f.gbuf), _dev(f.tbuf) if f.tbuf.shape[0] else None, _dev(f.counts), out)
    m.check()
    return out.cpu().numpy()


def _stream(m, lat, f, order, pool=None):
    own = pool is None
    if own:
        pool = gl.glassnet_pool_create(m.handle, f.h, f.w)
    try:
        tb = _dev(f.tbuf)
        cnt = _dev(f.counts)
        for k in order:
            cov = (cnt > k).to(torch.uint8)
            gl.glassnet_accumulate_layer(m.handle, lat.handle, pool, tb[k], cov)
        out = torch.full((3, f.h, f.w), float("nan"), device=DEV)
        gl.glassnet_resolve(m.handle, lat.handle, pool, _dev(f.gbuf), out)
        m.check()
        return out.cpu().numpy()
    finally:
        if own:
            gl.glassnet_pool_free(pool)


# 512x512 K=8 Poisson(3): the benchmark's frame; layer 7 covers ~1 % of the
# pixels, so most of its tiles have no covered pixel
CASES = [(96, 80, 8, "poisson3", 1), (33, 47, 4, "uniform", 2), (256, 256, 8, "poisson3", 3),
         (128, 128, 3, "all", 4), (512, 512, 8, "poisson3", 5)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-K{c[2]}-{c[3]}")
def test_streamed_layers_equal_render(net, case):
    _, m, lat = net
    h, w, K, cd, seed = case
    f = synth.make_frame(h, w, K, counts=cd, seed=40 + seed)
    ref = _render(m, lat, f)
    assert np.array_equal(_stream(m, lat, f, range(K)), ref)


def test_layer_order_does_not_matter(net):
    _, m, lat = net
    f = synth.make_frame(64, 64, 6, counts="uniform", seed=50)
    ref = _render(m, lat, f)
    rng = np.random.default_rng(7)
    for _ in range(3):
        assert np.array_equal(_stream(m, lat, f, rng.permutation(6)), ref)


def test_streamed_frame_meets_oracle(net):
    wts, m, lat = net
    f = synth.make_frame(40, 36, 5, counts="uniform", seed=51)
    got = _stream(m, lat, f, range(5)).astype(np.float64)
    exp = oracle.render_frame(wts, synth.make_scene(3), f.gbuf, f.tbuf, f.counts)
    err = np.abs(got - exp)
    assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (err.max(), err.mean())


def test_empty_pool_is_opaque_only(net):
    wts, m, lat = net
    f = synth.make_frame(24, 20, 2, counts="all", seed=52)
    pool = gl.glassnet_pool_create(m.handle, 24, 20)
    try:
        out = torch.full((3, 24, 20), float("nan"), device=DEV)
        gl.glassnet_resolve(m.handle, lat.handle, pool, _dev(f.gbuf), out)
        m.check()
        got = out.cpu().numpy()
    finally:
        gl.glassnet_pool_free(pool)
    zero = np.zeros_like(f.counts)
    assert np.array_equal(got, _render(m, lat, synth.Frame(gbuf=f.gbuf, tbuf=f.tbuf, counts=zero)))
    sigma = oracle.scene_encoder(wts, synth.make_scene(3))
    exp = oracle.render_opaque_only(wts, sigma, f.gbuf.reshape(14, -1).T).T.reshape(3, 24, 20)
    assert np.abs(got - exp).max() <= BF16_MAX


def test_null_coverage_covers_every_pixel(net):
    _, m, lat = net
    f = synth.make_frame(48, 40, 1, counts="all", seed=53)
    ref = _render(m, lat, f)
    pool = gl.glassnet_pool_create(m.handle, 48, 40)
    try:
        gl.glassnet_accumulate_layer(m.handle, lat.handle, pool, _dev(f.tbuf)[0], None)
        out = torch.full((3, 48, 40), float("nan"), device=DEV)
        gl.glassnet_resolve(m.handle, lat.handle, pool, _dev(f.gbuf), out)
        m.check()
        assert np.array_equal(out.cpu().numpy(), ref)
    finally:
        gl.glassnet_pool_free(pool)


def test_layer_limit_and_reset(net):
    _, m, lat = net
    f = synth.make_frame(32, 32, 8, counts="all", seed=54)
    pool = gl.glassnet_pool_create(m.handle, 32, 32)
    try:
        layer = _dev(f.tbuf)[0]
        for _ in range(8):
            gl.glassnet_accumulate_layer(m.handle, lat.handle, pool, layer, None)
        with pytest.raises(gl.GlassNetError) as ei:
            gl.glassnet_accumulate_layer(m.handle, lat.handle, pool, layer, None)
        assert ei.value.code == gl.GN_EINVAL
        # reset empties it: the streamed frame then equals the one-shot render
        gl.glassnet_pool_reset(pool)
        assert np.array_equal(_stream(m, lat, f, range(8), pool=pool), _render(m, lat, f))
    finally:
        gl.glassnet_pool_free(pool)


def test_accumulates_over_alternating_empty_tiles(net):
    """Accumulate launches whose tiles alternate between a few covered pixels
    and none (the tiles without covered pixels involve no MMA): 30 streamed
    frames of 8 layers at 512x512, each resolved and checked.  The loaders'
    pacing barrier must never complete two phases ahead of their wait, however
    fast the empty tiles go by (a device wait that gives up is reported as
    GN_ETIMEOUT by the check); every frame equals the one-shot render."""
    _, m, lat = net
    h = w = 512
    f = synth.make_frame(h, w, 8, counts="all", seed=56)
    cnt = np.zeros((h, w), dtype=np.uint8)
    flat = cnt.reshape(-1)
    for t0 in range(0, h * w, 256):  # even 128-pixel tiles: 3 covered pixels, odd tiles: none
        flat[t0 + 5] = flat[t0 + 60] = flat[t0 + 127] = 8
    f = synth.Frame(gbuf=f.gbuf, tbuf=f.tbuf, counts=cnt)
    want = _render(m, lat, f)
    pool = gl.glassnet_pool_create(m.handle, h, w)
    try:
        for _ in range(30):
            gl.glassnet_pool_reset(pool)
            assert np.array_equal(_stream(m, lat, f, range(8), pool=pool), want)
    finally:
        gl.glassnet_pool_free(pool)


def test_coverage_above_one_is_reported(net):
    _, m, lat = net
    f = synth.make_frame(16, 16, 1, counts="all", seed=55)
    pool = gl.glassnet_pool_create(m.handle, 16, 16)
    try:
        cov = torch.ones((16, 16), dtype=torch.uint8, device=DEV)
        cov[3, 5] = 2
        gl.glassnet_accumulate_layer(m.handle, lat.handle, pool, _dev(f.tbuf)[0], cov)
        with pytest.raises(gl.GlassNetError) as ei:
            m.check()
        assert ei.value.code == gl.GN_EINVAL
    finally:
        gl.glassnet_pool_free(pool)


def test_streaming_needs_bf16_model(cuda_lib):
    m = gl.Model(synth.make_weights(synth.BASE_WIDTHS, seed=0), gl.GN_FP32_PLAIN)
    with pytest.raises(gl.GlassNetError) as ei:
        gl.glassnet_pool_create(m.handle, 8, 8)
    assert ei.value.code == gl.GN_EUNSUPPORTED
