"""GPU parity of the CUDA path against the FP64 oracle, through the C ABI.

Tolerances (RGB in [0, 1]):
  FP32 plain vs oracle:  max |err| <= 1e-4
  BF16 fused vs oracle:  max |err| <= 2e-2, mean |err| <= 3e-3
  BF16 vs FP32 plain:    PSNR >= 45 dB
  BF16 under any permutation of each pixel's valid layers: bit-identical.
"""
import numpy as np
import pytest
import torch

import oracle
from gen import synth
from paper_2405_19056_gb300 import glassnet as gl

pytestmark = pytest.mark.gpu

FP32_MAX = 1e-4
BF16_MAX = 2e-2
BF16_MEAN = 3e-3
PSNR_MIN = 45.0

DEV = "cuda:0"


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


class Net:
    def __init__(self, widths, seed=0, bias="zero"):
        self.w = synth.make_weights(widths, seed=seed, bias=bias)
        self.blob = gl.pack_blob(self.w)
        self.models = {}

    def model(self, precision):
        if precision not in self.models:
            self.models[precision] = gl.Model(self.blob, precision)
        return self.models[precision]


@pytest.fixture(scope="module")
def base(cuda_lib):
    return Net(synth.BASE_WIDTHS, seed=0)


@pytest.fixture(scope="module")
def base_bias(cuda_lib):
    return Net(synth.BASE_WIDTHS, seed=3, bias="uniform")


@pytest.fixture(scope="module")
def doubled(cuda_lib):
    return Net(synth.DOUBLED_WIDTHS, seed=0)


def render(net, precision, scene, frame, tbuf=None, counts=None):
    m = net.model(precision)
    lat = m.encode(scene)
    t = frame.tbuf if tbuf is None else tbuf
    c = frame.counts if counts is None else counts
    out = torch.full((3, frame.h, frame.w), float("nan"), device=DEV)
    m.render(lat, _dev(frame.gbuf), _dev(t) if t.shape[0] else None, _dev(c), out)
    m.check()
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def ref(net, scene, frame):
    return oracle.render_frame(net.w, scene, frame.gbuf, frame.tbuf, frame.counts)


def psnr(a, b):
    mse = np.mean((a - b) ** 2)
    return float("inf") if mse == 0 else 10 * np.log10(1.0 / mse)


# ------------------------------------------------------------------ encoder

@pytest.mark.parametrize("which", ["base", "doubled"])
def test_encode_scene_and_fold(which, request):
    net = request.getfixturevalue(which)
    m = net.model(gl.GN_BF16_FUSED)
    scene = synth.make_scene(5)
    lat = m.encode(scene)
    H, Z = m.hidden, m.latent_width
    sig = torch.empty(Z, device=DEV)
    cphi = torch.empty(H, device=DEV)
    cb = torch.empty(H, device=DEV)
    gl.glassnet_latent_read(lat.handle, sig, cphi, cb)
    torch.cuda.synchronize()
    sigma = oracle.scene_encoder(net.w, scene)
    np.testing.assert_allclose(sig.cpu().numpy(), sigma, rtol=1e-5, atol=1e-5)
    W1, b1 = (np.float64(a) for a in net.w["phi1"])
    WB, bB = (np.float64(a) for a in net.w["B1"])
    np.testing.assert_allclose(cphi.cpu().numpy(), W1[:, 12:] @ sigma + b1, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(cb.cpu().numpy(), WB[:, 14 + H:] @ sigma + bB, rtol=1e-5, atol=1e-5)


# ------------------------------------------------------ small configurations

CASES = [
    # (name, widths fixture, h, w, K, counts)
    ("64x64 K=2 all valid (base)", "base", 64, 64, 2, "all"),
    ("256x256 K=4 uniform counts (base)", "base", 256, 256, 4, "uniform"),
    ("64x64 K=8 poisson (doubled)", "doubled", 64, 64, 8, "poisson3"),
    ("96x80 K=3 uniform, biases (base)", "base_bias", 96, 80, 3, "uniform"),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp32_plain_vs_oracle(case, request):
    _, fx, h, w, K, counts = case
    net = request.getfixturevalue(fx)
    scene = synth.make_scene(1)
    frame = synth.make_frame(h, w, K, counts=counts, seed=1)
    got = render(net, gl.GN_FP32_PLAIN, scene, frame)
    err = np.abs(got - ref(net, scene, frame))
    assert err.max() <= FP32_MAX, err.max()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_bf16_fused_vs_oracle_and_fp32(case, request):
    _, fx, h, w, K, counts = case
    net = request.getfixturevalue(fx)
    scene = synth.make_scene(1)
    frame = synth.make_frame(h, w, K, counts=counts, seed=1)
    got = render(net, gl.GN_BF16_FUSED, scene, frame)
    err = np.abs(got - ref(net, scene, frame))
    assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (err.max(), err.mean())
    plain = render(net, gl.GN_FP32_PLAIN, scene, frame)
    assert psnr(got, plain) >= PSNR_MIN, psnr(got, plain)


# ------------------------------------------------------------- invariants

def test_bf16_bit_identical_under_8_permutations(base):
    """256x256, K=4, counts U{0..4}, layers shuffled with seeds 1..8."""
    scene = synth.make_scene(0)
    frame = synth.make_frame(256, 256, 4, counts="uniform", seed=0)
    ref_out = render(base, gl.GN_BF16_FUSED, scene, frame)
    for seed in range(1, 9):
        fp = synth.permute_layers(frame, seed)
        got = render(base, gl.GN_BF16_FUSED, scene, fp)
        assert np.array_equal(got, ref_out), f"permutation seed {seed} changed the output"


def test_bf16_bit_identical_under_permutation_doubled(doubled):
    scene = synth.make_scene(2)
    frame = synth.make_frame(64, 64, 8, counts="poisson3", seed=2)
    a = render(doubled, gl.GN_BF16_FUSED, scene, frame)
    for seed in (11, 12):
        b = render(doubled, gl.GN_BF16_FUSED, scene, synth.permute_layers(frame, seed))
        assert np.array_equal(a, b)


@pytest.mark.parametrize("precision", [gl.GN_BF16_FUSED, gl.GN_FP32_PLAIN])
def test_empty_set_matches_opaque_only(base_bias, precision):
    scene = synth.make_scene(3)
    frame = synth.make_frame(40, 33, 4, counts="all", seed=3)
    zero = np.zeros_like(frame.counts)
    got = render(base_bias, precision, scene, frame, counts=zero)
    sigma = oracle.scene_encoder(base_bias.w, scene)
    rows = frame.gbuf.reshape(14, -1).T
    exp = oracle.render_opaque_only(base_bias.w, sigma, rows).T.reshape(3, frame.h, frame.w)
    tol = FP32_MAX if precision == gl.GN_FP32_PLAIN else BF16_MAX
    assert np.abs(got - exp).max() <= tol
    # K = 0 (no tbuf at all) gives the same bits as every count 0
    f0 = synth.Frame(gbuf=frame.gbuf, tbuf=np.zeros((0, 12, frame.h, frame.w), np.float32),
                     counts=zero)
    got0 = render(base_bias, precision, scene, f0)
    assert np.array_equal(got, got0)


def test_invalid_slots_never_read(base):
    scene = synth.make_scene(4)
    frame = synth.make_frame(50, 70, 5, counts="uniform", seed=4)
    a = render(base, gl.GN_BF16_FUSED, scene, frame)
    t2 = frame.tbuf.copy().reshape(5, 12, -1)
    c = frame.counts.reshape(-1)
    for k in range(5):
        t2[k][:, c <= k] = np.float32(-3.0e38)
    b = render(base, gl.GN_BF16_FUSED, scene, frame, tbuf=t2.reshape(frame.tbuf.shape))
    assert np.array_equal(a, b)
    assert np.all(np.isfinite(a))


@pytest.mark.parametrize("hw", [(1, 1), (1, 128), (129, 1), (3, 127), (130, 130)])
@pytest.mark.parametrize("K", [1, 3, 8])
def test_ragged_sizes(base, hw, K):
    h, w = hw
    scene = synth.make_scene(6)
    frame = synth.make_frame(h, w, K, counts="uniform", seed=6)
    got = render(base, gl.GN_BF16_FUSED, scene, frame)
    err = np.abs(got - ref(base, scene, frame))
    assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN


def test_result_independent_of_tile_position(base):
    """A pixel's output does not depend on where it sits in a 128-pixel tile."""
    scene = synth.make_scene(7)
    frame = synth.make_frame(16, 100, 3, counts="uniform", seed=7)
    a = render(base, gl.GN_BF16_FUSED, scene, frame)
    sh = synth.Frame(gbuf=np.roll(frame.gbuf, 37, axis=2), tbuf=np.roll(frame.tbuf, 37, axis=3),
                     counts=np.roll(frame.counts, 37, axis=1))
    b = render(base, gl.GN_BF16_FUSED, scene, sh)
    assert np.array_equal(np.roll(a, 37, axis=2), b)


@pytest.mark.parametrize("hw,bad", [(8, 5), (64, 255)], ids=["8x8-count5", "64x64-count255"])
def test_count_above_K_reported(base, hw, bad):
    """A count above K sets GN_EINVAL; the pixel is still rendered (with K
    layers), so every output is written."""
    m = base.model(gl.GN_BF16_FUSED)
    scene = synth.make_scene(8)
    frame = synth.make_frame(hw, hw, 2, counts="all", seed=8)
    lat = m.encode(scene)
    cnt = frame.counts.copy()
    cnt[3, 3] = bad
    out = torch.full((3, hw, hw), float("nan"), device=DEV)
    m.render(lat, _dev(frame.gbuf), _dev(frame.tbuf), _dev(cnt), out)
    assert gl.glassnet_check_code(m.handle) == gl.GN_EINVAL
    assert gl.glassnet_check_code(m.handle) == gl.GN_OK  # cleared
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    assert np.array_equal(got, render(base, gl.GN_BF16_FUSED, scene, frame))


def test_exact_sum_range_reported(cuda_lib):
    """Activations scaled far beyond the fixed-point range set GN_ERANGE."""
    w = synth.make_weights(synth.BASE_WIDTHS, seed=9)
    w["phi2"] = (w["phi2"][0] * 5000.0, w["phi2"][1])
    m = gl.Model(w, gl.GN_BF16_FUSED)
    frame = synth.make_frame(8, 8, 8, counts="all", seed=9)
    lat = m.encode(synth.make_scene(9))
    out = torch.empty((3, 8, 8), device=DEV)
    m.render(lat, _dev(frame.gbuf), _dev(frame.tbuf), _dev(frame.counts), out)
    assert gl.glassnet_check_code(m.handle) == gl.GN_ERANGE


@pytest.mark.parametrize("widths", ["base", "doubled"])
def test_timeout_reported_and_next_render_exact(widths, request):
    """A device wait that gives up (the stall hook: the MMA warp waits 20 us on
    a barrier nothing arrives on) is reported as GN_ETIMEOUT, the frame is left
    unwritten, and the next render of the same model is bit-identical to one
    taken before the stall."""
    net = request.getfixturevalue(widths)
    m = net.model(gl.GN_BF16_FUSED)
    scene = synth.make_scene(12)
    frame = synth.make_frame(40, 52, 4, counts="uniform", seed=12)
    before = render(net, gl.GN_BF16_FUSED, scene, frame)
    lat = m.encode(scene)
    out = torch.full((3, frame.h, frame.w), float("nan"), device=DEV)
    gl.glassnet_debug_stall_next_render(m.handle, 20_000)
    m.render(lat, _dev(frame.gbuf), _dev(frame.tbuf), _dev(frame.counts), out)
    assert gl.glassnet_check_code(m.handle) == gl.GN_ETIMEOUT
    # the report names the kernel, its launch mode and the barrier that gave up
    # (the stall hook's slot)
    assert "fused BF16 kernel, frame launch, mbarrier slot 26)" in gl.glassnet_last_error()
    assert gl.glassnet_check_code(m.handle) == gl.GN_OK  # cleared
    assert np.isnan(out.cpu().numpy()).all()  # no tile ran
    after = render(net, gl.GN_BF16_FUSED, scene, frame)
    assert np.array_equal(before, after)


def test_render_batch_equals_single_renders(base):
    m = base.model(gl.GN_BF16_FUSED)
    specs = [(33, 47, 3, "uniform", 1), (128, 64, 8, "poisson3", 2), (5, 300, 1, "all", 3)]
    frames, singles, outs, lats = [], [], [], []
    for (h, w, K, cd, s) in specs:
        f = synth.make_frame(h, w, K, counts=cd, seed=20 + s)
        lat = m.encode(synth.make_scene(s))
        lats.append(lat)
        singles.append(render(base, gl.GN_BF16_FUSED, synth.make_scene(s), f))
        out = torch.full((3, h, w), float("nan"), device=DEV)
        outs.append(out)
        frames.append(dict(latent=lat.handle, gbuf=_dev(f.gbuf), tbuf=_dev(f.tbuf),
                           layer_count=_dev(f.counts), K=K, h=h, w=w, out=out))
    gl.glassnet_render_batch(m.handle, frames)
    m.check()
    for out, single in zip(outs, singles):
        assert np.array_equal(out.cpu().numpy().astype(np.float64), single)


def test_render_host_matches_device(base):
    m = base.model(gl.GN_BF16_FUSED)
    scene = synth.make_scene(10)
    f = synth.make_frame(70, 90, 4, counts="uniform", seed=10)
    lat = m.encode(scene)
    dev_out = render(base, gl.GN_BF16_FUSED, scene, f)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    out_h = torch.empty((3, 70, 90)).pin_memory()
    gl.glassnet_render_host(m.handle, lat.handle, pin(f.gbuf), pin(f.tbuf), pin(f.counts), 4, 70,
                            90, out_h)
    assert np.array_equal(out_h.numpy().astype(np.float64), dev_out)


# ------------------------------------------------------------- full size

def test_full_512_K8_poisson_sampled(doubled):
    """The benchmark workload (512x512, K=8, Poisson(3) counts, doubled widths)
    rendered in one launch; the oracle checks the 64x64 crop at rows/cols
    0..63 and 1024 sampled pixels."""
    scene = synth.make_scene(0)
    frame = synth.make_frame(512, 512, 8, counts="poisson3", seed=0)
    got = render(doubled, gl.GN_BF16_FUSED, scene, frame)
    crop = synth.Frame(gbuf=frame.gbuf[:, :64, :64].copy(), tbuf=frame.tbuf[:, :, :64, :64].copy(),
                       counts=frame.counts[:64, :64].copy())
    err = np.abs(got[:, :64, :64] - ref(doubled, scene, crop))
    assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (err.max(), err.mean())
    rng = np.random.default_rng(0)
    idx = rng.choice(512 * 512, 1024, replace=False)
    ys, xs = idx // 512, idx % 512
    samp = synth.Frame(gbuf=frame.gbuf[:, ys, xs][:, None, :].copy(),
                       tbuf=frame.tbuf[:, :, ys, xs][:, :, None, :].copy(),
                       counts=frame.counts[ys, xs][None, :].copy())
    exp = ref(doubled, scene, samp)[:, 0, :]
    e2 = np.abs(got[:, ys, xs] - exp)
    assert e2.max() <= BF16_MAX and e2.mean() <= BF16_MEAN, (e2.max(), e2.mean())
