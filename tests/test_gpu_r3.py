"""R with a 3x3 first layer (Sec. 3.4) on the GPU, through the C ABI: models
loaded with gn_model_config.r_kernel = 3.  The fused kernel stops at the
neural buffer y (BF16 in the render's workspace); a tcgen05 kernel runs the
3x3 layer over the frame (zero outside it), R2 and the sigmoid.

Tolerances (RGB in [0, 1]), the same as with a 1x1 R:
  FP32 plain vs oracle:  max |err| <= 1e-4
  BF16 fused vs oracle:  max |err| <= 2e-2, mean |err| <= 3e-3
A CPU emulation of the BF16 rounding points (y, the 3x3 weights and q in
BF16, FP32 accumulation) gives at most 5.1e-3 max and 6e-4 mean error
against the oracle on these weights.
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


def net(H=128, Z=256, L=0, seed=3, bias="uniform"):
    key = (H, Z, L, seed, bias)
    if key not in _NETS:
        _NETS[key] = (synth.make_weights(synth.Widths(H, Z, L, 3), seed=seed, bias=bias), {})
    return _NETS[key]


def model(precision=gl.GN_BF16_FUSED, pooling=gl.GN_POOL_MAX_MEAN, **kw):
    w, models = net(**kw)
    if (precision, pooling) not in models:
        models[(precision, pooling)] = gl.Model(w, precision, pooling)
    return w, models[(precision, pooling)]


def render(m, scene, f):
    lat = m.encode(scene)
    out = torch.full((3, f.h, f.w), float("nan"), device=DEV)
    m.render(lat, _dev(f.gbuf), _dev(f.tbuf) if f.tbuf.shape[0] else None, _dev(f.counts), out)
    m.check()
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def ref(w, scene, f, pooling="max_mean"):
    return oracle.render_frame(w, scene, f.gbuf, f.tbuf, f.counts, pooling=pooling)


def test_model_reports_its_kernel(cuda_lib):
    _, m = model()
    assert m.r_kernel == 3


@pytest.mark.parametrize("H", [64, 128])
def test_fp32_plain_r3_vs_oracle(cuda_lib, H):
    w, m = model(gl.GN_FP32_PLAIN, H=H, Z=2 * H)
    scene = synth.make_scene(1)
    f = synth.make_frame(21, 37, 4, counts="uniform", seed=1)
    err = np.abs(render(m, scene, f) - ref(w, scene, f))
    assert err.max() <= FP32_MAX, err.max()


CASES = [
    # (H, L, h, w, K, counts, pooling): strips of 128 columns with a ragged
    # last strip, single rows and columns, frames narrower than a strip
    (128, 0, 40, 300, 8, "poisson3", "max_mean"),
    (128, 0, 1, 130, 4, "uniform", "max_mean"),
    (128, 0, 67, 1, 3, "all", "max_mean"),
    (64, 0, 33, 47, 8, "poisson3", "max_mean"),
    (128, 0, 24, 256, 6, "uniform", "sum"),
    (64, 4, 30, 140, 8, "poisson3", "max_mean"),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"H{c[0]}-L{c[1]}-{c[2]}x{c[3]}-K{c[4]}-{c[5]}-{c[6]}")
def test_bf16_fused_r3_vs_oracle(cuda_lib, case):
    H, L, h, w_, K, counts, pooling = case
    pl = gl.GN_POOL_SUM if pooling == "sum" else gl.GN_POOL_MAX_MEAN
    w, m = model(gl.GN_BF16_FUSED, pl, H=H, Z=2 * H, L=L)
    scene = synth.make_scene(1)
    f = synth.make_frame(h, w_, K, counts=counts, seed=2)
    got = render(m, scene, f)
    err = np.abs(got - ref(w, scene, f, pooling))
    assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (err.max(), err.mean())
    _, mp = model(gl.GN_FP32_PLAIN, pl, H=H, Z=2 * H, L=L)
    assert np.abs(got - render(mp, scene, f)).max() <= BF16_MAX


def test_centre_tap_only_equals_the_1x1_model(cuda_lib):
    """With only the centre tap set, the 3x3 R is the 1x1 R: zero taps add
    exact zeros and the centre tap's MMAs, the bias, ReLU and BF16 rounding of
    q run as in the fused kernel; R2 (128 terms) then sums in FP32 on the CUDA
    cores instead of the tensor core, so the frames agree to FP32 rounding of
    that sum (2e-6 in RGB), far inside any tap or halo mistake."""
    w1 = synth.make_weights(synth.DOUBLED_WIDTHS, seed=4, bias="uniform")
    H = 128
    K3 = np.zeros((H, H, 3, 3), np.float32)
    K3[:, :, 1, 1] = w1["R1"][0]
    w3 = dict(w1)
    w3["R1"] = (K3.reshape(H, 9 * H), w1["R1"][1])
    w3["r_kernel"] = 3
    scene = synth.make_scene(5)
    f = synth.make_frame(77, 300, 8, counts="poisson3", seed=5)
    a = render(gl.Model(w1, gl.GN_BF16_FUSED), scene, f)
    b = render(gl.Model(w3, gl.GN_BF16_FUSED), scene, f)
    assert np.abs(a - b).max() <= 2e-6, np.abs(a - b).max()


def test_r3_bit_identical_under_permutations(cuda_lib):
    _, m = model()
    scene = synth.make_scene(2)
    f = synth.make_frame(64, 200, 8, counts="uniform", seed=7)
    base = render(m, scene, f)
    for s in range(1, 4):
        assert np.array_equal(render(m, scene, synth.permute_layers(f, seed=s)), base), s


def test_r3_render_host_and_workspace(cuda_lib):
    _, m = model()
    scene = synth.make_scene(3)
    f = synth.make_frame(50, 150, 5, counts="uniform", seed=9)
    dev_out = render(m, scene, f)
    lat = m.encode(scene)
    out_h = torch.empty((3, 50, 150)).pin_memory()
    gl.glassnet_render_host(m.handle, lat.handle, torch.from_numpy(f.gbuf).pin_memory(),
                            torch.from_numpy(f.tbuf).pin_memory(), torch.from_numpy(f.counts).pin_memory(),
                            5, 50, 150, out_h)
    assert np.array_equal(out_h.numpy().astype(np.float64), dev_out)
    n3 = gl.glassnet_workspace_bytes(m.handle, 5, 50, 150)
    m1 = gl.Model(synth.make_weights(synth.DOUBLED_WIDTHS, seed=3), gl.GN_BF16_FUSED)
    n1 = gl.glassnet_workspace_bytes(m1.handle, 5, 50, 150)
    assert n3 >= n1 + 50 * 150 * 128 * 2  # the neural buffer


def test_r3_batch_and_graph_equal_single_renders(cuda_lib):
    """Frames of different sizes in one batched launch (each with its own
    neural buffer and 3x3 kernel launch), and the same batch replayed from a
    CUDA graph, reproduce the single renders bit for bit."""
    _, m = model()
    specs = [(33, 47, 3, "uniform", 1), (70, 200, 8, "poisson3", 2), (5, 300, 1, "all", 3)]
    frames, singles, outs, lats = [], [], [], []
    for (h, w, K, cd, sd) in specs:
        f = synth.make_frame(h, w, K, counts=cd, seed=20 + sd)
        singles.append(render(m, synth.make_scene(sd), f))
        lat = m.encode(synth.make_scene(sd))
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
        for _ in range(2):
            gl.glassnet_graph_launch(g)
            m.check()
            for out, single in zip(outs, singles):
                assert np.array_equal(out.cpu().numpy().astype(np.float64), single)
                out.fill_(float("nan"))
    finally:
        gl.glassnet_graph_free(g)


def test_r3_streamed_equals_render(cuda_lib):
    """Layers accumulated one at a time (any order), then the resolve writes
    the neural buffer into the pool's own and the 3x3 kernel runs: the frame
    equals glassnet_render bit for bit."""
    _, m = model()
    scene = synth.make_scene(4)
    f = synth.make_frame(90, 260, 8, counts="poisson3", seed=12)
    want = render(m, scene, f)
    lat = m.encode(scene)
    pool = gl.glassnet_pool_create(m.handle, f.h, f.w)
    try:
        tb, cnt = _dev(f.tbuf), _dev(f.counts)
        for k in [2, 7, 0, 5, 3, 1, 6, 4]:
            gl.glassnet_accumulate_layer(m.handle, lat.handle, pool, tb[k], (cnt > k).to(torch.uint8))
        out = torch.full((3, f.h, f.w), float("nan"), device=DEV)
        gl.glassnet_resolve(m.handle, lat.handle, pool, _dev(f.gbuf), out)
        m.check()
        assert np.array_equal(out.cpu().numpy().astype(np.float64), want)
    finally:
        gl.glassnet_pool_free(pool)


def test_fp8_r3_vs_oracle(cuda_lib):
    """FP8 (E4M3) fused kernel to the neural buffer (B2's output in real units
    as BF16), then the 3x3 kernel: within the FP8 bound (max 0.1, at most 1e-3 of values above 6e-2, mean
    1e-2), calibrated on a seed-1 frame with the FP32 path's 3x3 R, and
    bit-identical under permutations of the layers."""
    w, _ = net()
    m = gl.Model(w, gl.GN_FP8_FUSED)
    cal = synth.make_frame(128, 128, 8, counts="poisson3", seed=1)
    lat = m.encode(synth.make_scene(0))
    gl.glassnet_calibrate_fp8(m.handle, lat.handle, _dev(cal.gbuf), _dev(cal.tbuf), _dev(cal.counts),
                              8, 128, 128)
    scene = synth.make_scene(0)
    f = synth.make_frame(60, 150, 8, counts="poisson3", seed=14)
    got = render(m, scene, f)
    err = np.abs(got - ref(w, scene, f))
    assert err.max() <= 0.1 and err.mean() <= 1e-2, (err.max(), err.mean())
    assert np.mean(err > 6e-2) <= 1e-3, (np.mean(err > 6e-2), err.max())
    assert np.array_equal(render(m, scene, synth.permute_layers(f, seed=3)), got)


def test_full_512_K8_poisson_r3_corner_and_interior(cuda_lib):
    """512x512, K=8, Poisson(3) counts, doubled widths with the 3x3 R: the
    oracle renders two 66x66 crops (the frame's top-left corner and an
    interior block spanning a strip boundary) and the 64x64 pixels whose
    neighbourhoods lie inside each crop are compared."""
    w, m = model(seed=0, bias="zero")
    scene = synth.make_scene(0)
    f = synth.make_frame(512, 512, 8, counts="poisson3", seed=0)
    got = render(m, scene, f)
    for (y0, x0) in [(0, 0), (200, 95)]:
        ys, xs = slice(max(y0 - 1, 0), y0 + 65), slice(max(x0 - 1, 0), x0 + 65)
        crop = synth.Frame(gbuf=f.gbuf[:, ys, xs].copy(), tbuf=f.tbuf[:, :, ys, xs].copy(),
                           counts=f.counts[ys, xs].copy())
        exp = ref(w, scene, crop)
        oy, ox = y0 - ys.start, x0 - xs.start
        e = np.abs(got[:, y0:y0 + 64, x0:x0 + 64] - exp[:, oy:oy + 64, ox:ox + 64])
        assert e.max() <= BF16_MAX and e.mean() <= BF16_MEAN, ((y0, x0), e.max(), e.mean())


def test_pool_of_another_r_kernel_is_rejected(cuda_lib):
    """A pool holds state shaped by its model (a 3x3 R also owns a neural
    buffer): a model with another R kernel cannot use it."""
    _, m3 = model()
    m1 = gl.Model(synth.make_weights(synth.DOUBLED_WIDTHS, seed=3), gl.GN_BF16_FUSED)
    lat = m3.encode(synth.make_scene(0))
    f = synth.make_frame(16, 16, 1, counts="all", seed=1)
    pool = gl.glassnet_pool_create(m1.handle, 16, 16)
    try:
        out = torch.empty((3, 16, 16), device=DEV)
        with pytest.raises(gl.GlassNetError) as ei:
            gl.glassnet_resolve(m3.handle, lat.handle, pool, _dev(f.gbuf), out)
        assert ei.value.code == gl.GN_EINVAL and "R" in str(ei.value)
    finally:
        gl.glassnet_pool_free(pool)
