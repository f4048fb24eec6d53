"""The compacted ragged-layer schedule (GN_SCHEDULE_COMPACT, fused_compact.cu)
against the count-sorted kernel and the FP64 oracle, through the C ABI.

Bar: bit-identical to the sorted kernel's frame on every case (both pool the
same BF16 values exactly, Eq. 5), and within the BF16 bound of the oracle
(max |err| <= 2e-2, mean <= 3e-3) on the frames the oracle renders whole.
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


class Pair:
    """One weight set loaded twice: the sorted and the compacted schedule."""

    def __init__(self, widths, seed=0, bias="zero", pooling=gl.GN_POOL_MAX_MEAN):
        self.w = synth.make_weights(widths, seed=seed, bias=bias)
        blob = gl.pack_blob(self.w)
        self.sorted = gl.Model(blob, gl.GN_BF16_FUSED, pooling=pooling)
        self.compact = gl.Model(blob, gl.GN_BF16_FUSED, pooling=pooling)
        gl.glassnet_set_layer_schedule(self.compact.handle, gl.GN_SCHEDULE_COMPACT)


@pytest.fixture(scope="module")
def pair(cuda_lib):
    return Pair(synth.BASE_WIDTHS, seed=0)


@pytest.fixture(scope="module")
def pair_bias(cuda_lib):
    return Pair(synth.BASE_WIDTHS, seed=3, bias="uniform")


@pytest.fixture(scope="module")
def pair_sum(cuda_lib):
    return Pair(synth.BASE_WIDTHS, seed=4, pooling=gl.GN_POOL_SUM)


def render(m, scene, frame, tbuf=None):
    lat = m.encode(scene)
    t = frame.tbuf if tbuf is None else tbuf
    out = torch.full((3, frame.h, frame.w), float("nan"), device=DEV)
    m.render(lat, _dev(frame.gbuf), _dev(t) if t.shape[0] else None, _dev(frame.counts), out)
    m.check()
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def both(p, scene, frame):
    return render(p.sorted, scene, frame), render(p.compact, scene, frame)


CASES = [
    # (h, w, K, counts): several blocks, ragged tails, empty sets, K = 0
    (64, 64, 8, "poisson3"),
    (96, 80, 3, "uniform"),
    (256, 256, 4, "uniform"),
    (33, 17, 5, "poisson3"),
    (1, 1, 1, "all"),
    (129, 1, 8, "all"),
    (3, 127, 2, "uniform"),
    (130, 130, 8, "poisson3"),
    (40, 52, 0, "all"),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{h}x{w}-K{K}-{c}" for h, w, K, c in CASES])
def test_compact_bit_identical_to_sorted(pair, case):
    h, w, K, counts = case
    scene = synth.make_scene(2)
    frame = synth.make_frame(h, w, K, counts=counts, seed=h * 1000 + w + K)
    a, b = both(pair, scene, frame)
    assert np.isfinite(b).all()
    assert np.array_equal(a, b)


@pytest.mark.parametrize("case", [(64, 64, 8, "poisson3"), (96, 80, 3, "uniform")],
                         ids=["64x64-K8-poisson", "96x80-K3-uniform"])
def test_compact_vs_oracle_with_biases(pair_bias, case):
    h, w, K, counts = case
    scene = synth.make_scene(5)
    frame = synth.make_frame(h, w, K, counts=counts, seed=5)
    a, b = both(pair_bias, scene, frame)
    assert np.array_equal(a, b)
    err = np.abs(b - oracle.render_frame(pair_bias.w, scene, frame.gbuf, frame.tbuf, frame.counts))
    assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (err.max(), err.mean())


def test_compact_sum_pooling_bit_identical(pair_sum):
    scene = synth.make_scene(6)
    for (h, w, K, c) in [(64, 64, 8, "poisson3"), (33, 17, 5, "uniform"), (8, 8, 0, "all")]:
        frame = synth.make_frame(h, w, K, counts=c, seed=60 + K)
        a, b = both(pair_sum, scene, frame)
        assert np.array_equal(a, b)


def test_compact_under_permutations(pair):
    """Each pixel's valid layers shuffled (seeds 1..4): the same bits."""
    scene = synth.make_scene(0)
    frame = synth.make_frame(128, 96, 6, counts="uniform", seed=0)
    base = render(pair.compact, scene, frame)
    for s in range(1, 5):
        perm = synth.permute_layers(frame, s)
        assert np.array_equal(render(pair.compact, scene, perm), base)


def test_compact_batch_of_frames_and_scenes(pair):
    """A batch of frames of different sizes, counts and scenes (the folded
    biases change between blocks) equals the sorted kernel's batch."""
    specs = [(33, 47, 3, "uniform", 1), (128, 64, 8, "poisson3", 2), (5, 300, 1, "all", 3),
             (200, 3, 0, "all", 4), (64, 64, 8, "all", 5)]
    outs = {}
    for name in ("sorted", "compact"):
        m = getattr(pair, name)
        frames, res, keep = [], [], []
        for (h, w, K, cd, s) in specs:
            f = synth.make_frame(h, w, K, counts=cd, seed=30 + s)
            lat = m.encode(synth.make_scene(s))
            out = torch.full((3, h, w), float("nan"), device=DEV)
            keep.append((lat, f))
            res.append(out)
            frames.append(dict(latent=lat.handle, gbuf=_dev(f.gbuf),
                               tbuf=_dev(f.tbuf) if K else None,
                               layer_count=_dev(f.counts), K=K, h=h, w=w, out=out))
        gl.glassnet_render_batch(m.handle, frames)
        m.check()
        outs[name] = [o.cpu().numpy() for o in res]
    for a, b in zip(outs["sorted"], outs["compact"]):
        assert np.isfinite(b).all()
        assert np.array_equal(a, b)


def test_compact_count_above_K_reported(pair):
    scene = synth.make_scene(8)
    frame = synth.make_frame(64, 64, 2, counts="all", seed=8)
    cnt = frame.counts.copy()
    cnt[3, 3] = 255
    m = pair.compact
    lat = m.encode(scene)
    out = torch.full((3, 64, 64), float("nan"), device=DEV)
    m.render(lat, _dev(frame.gbuf), _dev(frame.tbuf), _dev(cnt), out)
    assert gl.glassnet_check_code(m.handle) == gl.GN_EINVAL
    assert gl.glassnet_check_code(m.handle) == gl.GN_OK
    assert np.array_equal(out.cpu().numpy().astype(np.float64), render(pair.sorted, scene, frame))


def test_compact_timeout_reported_and_next_render_exact(pair):
    m = pair.compact
    scene = synth.make_scene(12)
    frame = synth.make_frame(40, 52, 4, counts="uniform", seed=12)
    before = render(m, scene, frame)
    lat = m.encode(scene)
    out = torch.full((3, frame.h, frame.w), float("nan"), device=DEV)
    gl.glassnet_debug_stall_next_render(m.handle, 20_000)
    m.render(lat, _dev(frame.gbuf), _dev(frame.tbuf), _dev(frame.counts), out)
    assert gl.glassnet_check_code(m.handle) == gl.GN_ETIMEOUT
    # the report names the kernel, its launch mode and the barrier that gave up
    # (the stall hook's slot)
    assert "compacted kernel, frame launch, mbarrier slot 28)" in gl.glassnet_last_error()
    assert gl.glassnet_check_code(m.handle) == gl.GN_OK
    assert np.isnan(out.cpu().numpy()).all()
    assert np.array_equal(render(m, scene, frame), before)


def test_compact_full_512_K8_poisson(cuda_lib):
    """512x512, K = 8, Poisson(3) counts at the base widths: bit-identical to
    the sorted kernel over the whole frame."""
    p = Pair(synth.BASE_WIDTHS, seed=0)
    scene = synth.make_scene(0)
    frame = synth.make_frame(512, 512, 8, counts="poisson3", seed=0)
    a, b = both(p, scene, frame)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("kind", ["doubled", "fp32", "pe", "r3"])
def test_compact_unsupported_forms_refused(cuda_lib, kind):
    if kind == "doubled":
        m = gl.Model(synth.make_weights(synth.DOUBLED_WIDTHS, seed=0), gl.GN_BF16_FUSED)
    elif kind == "fp32":
        m = gl.Model(synth.make_weights(synth.BASE_WIDTHS, seed=0), gl.GN_FP32_PLAIN)
    elif kind == "pe":
        m = gl.Model(synth.make_weights(synth.BASE_PE_WIDTHS, seed=0), gl.GN_BF16_FUSED)
    else:
        m = gl.Model(synth.make_weights(synth.Widths(hidden=64, latent=128, r_kernel=3), seed=0), gl.GN_BF16_FUSED)
    rc = gl._lib().glassnet_set_layer_schedule(m.handle, gl.GN_SCHEDULE_COMPACT)
    assert rc == gl.GN_EUNSUPPORTED
    assert gl._lib().glassnet_set_layer_schedule(m.handle, 7) == gl.GN_EINVAL
