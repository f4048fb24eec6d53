"""Positional encoding of the inputs (Sec. 3.4) on the GPU, through the C ABI:
models loaded with gn_model_config.pe_freqs = L, every input (scene vector,
transparency layers, G-buffer) entering its first layer as
[x ; sin(2^f pi x) ; cos(2^f pi x) for f < L].

Tolerances (RGB in [0, 1]), the same as without encoding:
  FP32 plain vs oracle:  max |err| <= 1e-4   (L = 1, 4 and 10)
  BF16 fused vs oracle:  max |err| <= 2e-2, mean |err| <= 3e-3   (H = 64 and
  H = 128, L = 1 .. 4; at H = 128 the per-pixel weights stream through the
  kernel's shared-memory ring, with the same arithmetic)
A CPU emulation of the BF16 kernel's rounding points with every encoded band
rounded to BF16 gives at most 6.4e-3 max and 7e-4 mean error against the
oracle on these weights.  BF16 under any permutation of each pixel's valid
layers: bit-identical.
"""
import numpy as np
import pytest
import torch

import oracle
from gen import synth
from paper_2405_19056_gb300 import glassnet as gl

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FP32_MAX = 1e-4
BF16_MAX = 2e-2
BF16_MEAN = 3e-3


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


_NETS = {}


def net(L, seed=3, bias="uniform", H=64, Z=128):
    key = (L, seed, bias, H, Z)
    if key not in _NETS:
        _NETS[key] = (synth.make_weights(synth.Widths(H, Z, L), seed=seed, bias=bias), {})
    return _NETS[key]


def model(L, precision=gl.GN_BF16_FUSED, pooling=gl.GN_POOL_MAX_MEAN, **kw):
    w, models = net(L, **kw)
    if (precision, pooling) not in models:
        models[(precision, pooling)] = gl.Model(w, precision, pooling)
    return w, models[(precision, pooling)]


def render(m, scene, f, tbuf=None):
    lat = m.encode(scene)
    t = f.tbuf if tbuf is None else tbuf
    out = torch.full((3, f.h, f.w), float("nan"), device=DEV)
    m.render(lat, _dev(f.gbuf), _dev(t) if t.shape[0] else None, _dev(f.counts), out)
    m.check()
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def ref(w, scene, f, pooling="max_mean"):
    return oracle.render_frame(w, scene, f.gbuf, f.tbuf, f.counts, pooling=pooling)


def test_model_reports_its_encoding(cuda_lib):
    _, m = model(2)
    assert m.pe_freqs == 2 and m.pooling == gl.GN_POOL_MAX_MEAN and m.hidden == 64


@pytest.mark.parametrize("L", [1, 4, 10])
def test_fp32_plain_pe_vs_oracle(cuda_lib, L):
    w, m = model(L, gl.GN_FP32_PLAIN)
    scene = synth.make_scene(1)
    f = synth.make_frame(40, 72, 4, counts="uniform", seed=1)
    err = np.abs(render(m, scene, f) - ref(w, scene, f))
    assert err.max() <= FP32_MAX, err.max()


CASES = [
    # (L, h, w, K, counts, pooling): several tiles and a ragged tail
    (1, 64, 64, 2, "all", "max_mean"),
    (2, 96, 80, 3, "uniform", "max_mean"),
    (4, 64, 72, 8, "poisson3", "max_mean"),
    (4, 33, 47, 8, "all", "sum"),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"L{c[0]}-{c[1]}x{c[2]}-K{c[3]}-{c[4]}-{c[5]}")
def test_bf16_fused_pe_vs_oracle(cuda_lib, case):
    L, h, w_, K, counts, pooling = case
    pl = gl.GN_POOL_SUM if pooling == "sum" else gl.GN_POOL_MAX_MEAN
    w, m = model(L, gl.GN_BF16_FUSED, pl)
    scene = synth.make_scene(1)
    f = synth.make_frame(h, w_, K, counts=counts, seed=1)
    got = render(m, scene, f)
    err = np.abs(got - ref(w, scene, f, pooling))
    assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (err.max(), err.mean())
    # the FP32 plain path of the same encoded network agrees within BF16 rounding
    _, mp = model(L, gl.GN_FP32_PLAIN, pl)
    assert np.abs(got - render(mp, scene, f)).max() <= BF16_MAX


def test_encoding_changes_the_result(cuda_lib):
    """An L = 4 model whose sin / cos weight columns are zero renders the
    plain model's frame (the raw block comes first); with the columns set, the
    result moves far beyond the BF16 tolerance."""
    plain = synth.make_weights(synth.BASE_WIDTHS, seed=5, bias="uniform")
    L = 4
    pe = dict(plain)
    rng = np.random.default_rng(9)
    for name, n_raw in (("F1", synth.SCENE_DIM), ("phi1", 12), ("B1", 14)):
        W, b = plain[name]
        Wz = np.zeros((W.shape[0], W.shape[1] + 2 * L * n_raw), np.float32)
        Wz[:, :n_raw] = W[:, :n_raw]
        Wz[:, n_raw * (1 + 2 * L):] = W[:, n_raw:]
        pe[name] = (Wz, b)
    pe["pe_freqs"] = L
    scene = synth.make_scene(2)
    f = synth.make_frame(64, 64, 6, counts="uniform", seed=2)
    a = render(gl.Model(plain, gl.GN_BF16_FUSED), scene, f)
    b = render(gl.Model(pe, gl.GN_BF16_FUSED), scene, f)
    assert np.abs(a - b).max() <= BF16_MAX  # same network; the zero columns add exact zeros
    np.testing.assert_allclose(b, ref(plain, scene, f), atol=BF16_MAX)
    live = dict(pe)
    for name, n_raw in (("phi1", 12), ("B1", 14)):
        W, bb = pe[name]
        W = W.copy()
        W[:, n_raw:n_raw * (1 + 2 * L)] = rng.standard_normal((W.shape[0], 2 * L * n_raw)) * 0.2
        live[name] = (W, bb)
    c = render(gl.Model(live, gl.GN_BF16_FUSED), scene, f)
    assert np.abs(c - b).max() > 5 * BF16_MAX
    err = np.abs(c - ref(live, scene, f))
    assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (err.max(), err.mean())


def test_pe_bit_identical_under_permutations(cuda_lib):
    _, m = model(4)
    scene = synth.make_scene(2)
    f = synth.make_frame(128, 96, 8, counts="uniform", seed=7)
    base = render(m, scene, f)
    for s in range(1, 5):
        assert np.array_equal(render(m, scene, synth.permute_layers(f, seed=s)), base), s


def test_pe_empty_sets_and_no_layers(cuda_lib):
    w, m = model(3)
    scene = synth.make_scene(4)
    f0 = synth.make_frame(40, 56, 0, seed=5)
    err = np.abs(render(m, scene, f0) - ref(w, scene, f0))
    assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (err.max(), err.mean())
    sigma = oracle.scene_encoder(w, scene)
    exp = oracle.render_opaque_only(w, sigma, f0.gbuf.reshape(14, -1).T).T.reshape(3, 40, 56)
    assert np.abs(render(m, scene, f0) - exp).max() <= BF16_MAX


def test_pe_batch_graph_and_streaming_equal_render(cuda_lib):
    _, m = model(4)
    specs = [(33, 47, 3, "uniform", 1), (128, 64, 8, "poisson3", 2), (5, 300, 1, "all", 3)]
    frames, singles, outs, lats = [], [], [], []
    for (h, w, K, cd, s) in specs:
        f = synth.make_frame(h, w, K, counts=cd, seed=20 + s)
        singles.append(render(m, synth.make_scene(s), f))
        lat = m.encode(synth.make_scene(s))
        lats.append(lat)
        out = torch.full((3, h, w), float("nan"), device=DEV)
        outs.append(out)
        frames.append(dict(latent=lat.handle, gbuf=_dev(f.gbuf), tbuf=_dev(f.tbuf),
                           layer_count=_dev(f.counts), K=K, h=h, w=w, out=out))
    gl.glassnet_render_batch(m.handle, frames)
    m.check()
    for out, single in zip(outs, singles):
        assert np.array_equal(out.cpu().numpy().astype(np.float64), single)
        out.fill_(float("nan"))
    g = gl.glassnet_graph_create(m.handle, frames)
    try:
        gl.glassnet_graph_launch(g)
        m.check()
        for out, single in zip(outs, singles):
            assert np.array_equal(out.cpu().numpy().astype(np.float64), single)
    finally:
        gl.glassnet_graph_free(g)
    # streamed: one layer at a time, resolved once
    scene = synth.make_scene(3)
    f = synth.make_frame(160, 96, 8, counts="poisson3", seed=6)
    want = render(m, scene, f)
    lat = m.encode(scene)
    pool = gl.glassnet_pool_create(m.handle, f.h, f.w)
    try:
        tb, cnt = _dev(f.tbuf), _dev(f.counts)
        for k in [5, 0, 7, 3, 1, 6, 2, 4]:
            gl.glassnet_accumulate_layer(m.handle, lat.handle, pool, tb[k], (cnt > k).to(torch.uint8))
        out = torch.full((3, f.h, f.w), float("nan"), device=DEV)
        gl.glassnet_resolve(m.handle, lat.handle, pool, _dev(f.gbuf), out)
        m.check()
        assert np.array_equal(out.cpu().numpy().astype(np.float64), want)
    finally:
        gl.glassnet_pool_free(pool)


def test_full_512_K8_poisson_sampled_pe4(cuda_lib):
    """512x512, K=8, Poisson(3) counts, H=64 with L=4 in one launch; the oracle
    checks a 64x64 crop and 1024 sampled pixels."""
    w, m = model(4, seed=0, bias="zero")
    scene = synth.make_scene(0)
    f = synth.make_frame(512, 512, 8, counts="poisson3", seed=0)
    got = render(m, scene, f)
    crop = synth.Frame(gbuf=f.gbuf[:, :64, :64].copy(), tbuf=f.tbuf[:, :, :64, :64].copy(),
                       counts=f.counts[:64, :64].copy())
    err = np.abs(got[:, :64, :64] - ref(w, scene, crop))
    assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (err.max(), err.mean())
    rng = np.random.default_rng(0)
    idx = rng.choice(512 * 512, 1024, replace=False)
    ys, xs = idx // 512, idx % 512
    samp = synth.Frame(gbuf=f.gbuf[:, ys, xs][:, None, :].copy(),
                       tbuf=f.tbuf[:, :, ys, xs][:, :, None, :].copy(),
                       counts=f.counts[ys, xs][None, :].copy())
    e2 = np.abs(got[:, ys, xs] - ref(w, scene, samp)[:, 0, :])
    assert e2.max() <= BF16_MAX and e2.mean() <= BF16_MEAN, (e2.max(), e2.mean())


# ---------------------------------------------------------------- H = 128
# The doubled widths (H = 128, Z = 256): the kernel keeps phi1, phi2 and B1's
# first band resident and streams rho, B1's other bands and r block, B2, R1
# and R2 through its two-stage weight ring.

def dmodel(L, pooling=gl.GN_POOL_MAX_MEAN, seed=3, bias="uniform", r_kernel=1):
    key = (L, seed, bias, 128, 256, r_kernel)
    if key not in _NETS:
        _NETS[key] = (synth.make_weights(synth.Widths(128, 256, L, r_kernel), seed=seed, bias=bias), {})
    w, models = _NETS[key]
    if pooling not in models:
        models[pooling] = gl.Model(w, gl.GN_BF16_FUSED, pooling)
    return w, models[pooling]


D_CASES = [
    # (L, h, w, K, counts, pooling, r_kernel): several tiles and a ragged tail
    (1, 64, 64, 2, "all", "max_mean", 1),
    (2, 96, 80, 3, "uniform", "max_mean", 1),
    (3, 40, 136, 5, "uniform", "max_mean", 1),
    (4, 64, 72, 8, "poisson3", "max_mean", 1),
    (4, 33, 47, 8, "all", "sum", 1),
    (2, 48, 40, 4, "uniform", "max_mean", 3),
]


@pytest.mark.parametrize("case", D_CASES,
                         ids=lambda c: f"L{c[0]}-{c[1]}x{c[2]}-K{c[3]}-{c[4]}-{c[5]}-r{c[6]}")
def test_bf16_fused_pe_doubled_vs_oracle(cuda_lib, case):
    L, h, w_, K, counts, pooling, rk = case
    pl = gl.GN_POOL_SUM if pooling == "sum" else gl.GN_POOL_MAX_MEAN
    w, m = dmodel(L, pl, r_kernel=rk)
    assert m.pe_freqs == L and m.hidden == 128
    scene = synth.make_scene(1)
    f = synth.make_frame(h, w_, K, counts=counts, seed=1)
    got = render(m, scene, f)
    err = np.abs(got - ref(w, scene, f, pooling))
    assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (err.max(), err.mean())


def test_pe_doubled_bit_identical_under_permutations(cuda_lib):
    _, m = dmodel(4)
    scene = synth.make_scene(2)
    f = synth.make_frame(128, 96, 8, counts="uniform", seed=7)
    base = render(m, scene, f)
    for s in range(1, 5):
        assert np.array_equal(render(m, scene, synth.permute_layers(f, seed=s)), base), s


def test_pe_doubled_batch_graph_and_streaming_equal_render(cuda_lib):
    _, m = dmodel(4)
    specs = [(33, 47, 3, "uniform", 1), (128, 64, 8, "poisson3", 2), (5, 300, 1, "all", 3)]
    frames, singles, outs = [], [], []
    for (h, w, K, cd, s) in specs:
        f = synth.make_frame(h, w, K, counts=cd, seed=20 + s)
        singles.append(render(m, synth.make_scene(s), f))
        lat = m.encode(synth.make_scene(s))
        out = torch.full((3, h, w), float("nan"), device=DEV)
        outs.append(out)
        frames.append(dict(latent=lat.handle, gbuf=_dev(f.gbuf), tbuf=_dev(f.tbuf),
                           layer_count=_dev(f.counts), K=K, h=h, w=w, out=out, _lat=lat))
    gl.glassnet_render_batch(m.handle, frames)
    m.check()
    for out, single in zip(outs, singles):
        assert np.array_equal(out.cpu().numpy().astype(np.float64), single)
        out.fill_(float("nan"))
    g = gl.glassnet_graph_create(m.handle, frames)
    try:
        gl.glassnet_graph_launch(g)
        m.check()
        for out, single in zip(outs, singles):
            assert np.array_equal(out.cpu().numpy().astype(np.float64), single)
    finally:
        gl.glassnet_graph_free(g)
    scene = synth.make_scene(3)
    f = synth.make_frame(160, 96, 8, counts="poisson3", seed=6)
    want = render(m, scene, f)
    lat = m.encode(scene)
    pool = gl.glassnet_pool_create(m.handle, f.h, f.w)
    try:
        tb, cnt = _dev(f.tbuf), _dev(f.counts)
        for k in [5, 0, 7, 3, 1, 6, 2, 4]:
            gl.glassnet_accumulate_layer(m.handle, lat.handle, pool, tb[k], (cnt > k).to(torch.uint8))
        out = torch.full((3, f.h, f.w), float("nan"), device=DEV)
        gl.glassnet_resolve(m.handle, lat.handle, pool, _dev(f.gbuf), out)
        m.check()
        assert np.array_equal(out.cpu().numpy().astype(np.float64), want)
    finally:
        gl.glassnet_pool_free(pool)


def test_pe_doubled_timeout_reported_and_next_render_exact(cuda_lib):
    """The stall hook on the streamed kernel: the ring warp has copies in
    flight when the MMA warp gives up; every warp leaves through the exit
    path, the error names the kernel, and the next render is exact."""
    _, m = dmodel(2)
    scene = synth.make_scene(12)
    f = synth.make_frame(40, 52, 4, counts="uniform", seed=12)
    before = render(m, scene, f)
    lat = m.encode(scene)
    out = torch.full((3, f.h, f.w), float("nan"), device=DEV)
    gl.glassnet_debug_stall_next_render(m.handle, 20_000)
    m.render(lat, _dev(f.gbuf), _dev(f.tbuf), _dev(f.counts), out)
    assert gl.glassnet_check_code(m.handle) == gl.GN_ETIMEOUT
    assert "fused BF16 kernel, frame launch" in gl.glassnet_last_error()
    assert np.isnan(out.cpu().numpy()).all()
    assert np.array_equal(render(m, scene, f), before)


def test_full_512_K8_poisson_sampled_pe4_doubled(cuda_lib):
    """512x512, K=8, Poisson(3) counts, H=128 with L=4 in one launch; the
    oracle checks a 64x64 crop and 1024 sampled pixels."""
    w, m = dmodel(4, seed=0, bias="zero")
    scene = synth.make_scene(0)
    f = synth.make_frame(512, 512, 8, counts="poisson3", seed=0)
    got = render(m, scene, f)
    crop = synth.Frame(gbuf=f.gbuf[:, :64, :64].copy(), tbuf=f.tbuf[:, :, :64, :64].copy(),
                       counts=f.counts[:64, :64].copy())
    err = np.abs(got[:, :64, :64] - ref(w, scene, crop))
    assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (err.max(), err.mean())
    rng = np.random.default_rng(0)
    idx = rng.choice(512 * 512, 1024, replace=False)
    ys, xs = idx // 512, idx % 512
    samp = synth.Frame(gbuf=f.gbuf[:, ys, xs][:, None, :].copy(),
                       tbuf=f.tbuf[:, :, ys, xs][:, :, None, :].copy(),
                       counts=f.counts[ys, xs][None, :].copy())
    e2 = np.abs(got[:, ys, xs] - ref(w, scene, samp)[:, 0, :])
    assert e2.max() <= BF16_MAX and e2.mean() <= BF16_MEAN, (e2.max(), e2.mean())
