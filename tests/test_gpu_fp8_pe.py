"""FP8 (E4M3) fused path with positionally encoded inputs (Sec. 3.4), through
the C ABI, against the FP64 oracle.

The encoded bands enter as E4M3 codes: band 0 with its channel's calibrated
scale, the sine and cosine bands as 256 v (|v| <= 1).  Tolerance: the FP8
bound of the plain inputs (mean |err| <= 1e-2, max |err| <= 0.1, at most 1 in
10^3 values above 6e-2, the module docstring of test_gpu_fp8.py gives the
reasoning); the exact pooling keeps the output bit-identical under any
permutation of a pixel's valid layers.
"""
import numpy as np
import pytest
import torch

import oracle
from gen import synth
from paper_2405_19056_gb300 import glassnet as gl

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FP8_MAX = 0.1
FP8_MEAN = 1e-2
FP8_TAIL = (6e-2, 1e-3)
CAL = dict(h=128, w=128, K=8, counts="poisson3", seed=1)


def assert_fp8_close(err):
    assert err.max() <= FP8_MAX and err.mean() <= FP8_MEAN, (err.max(), err.mean())
    assert np.mean(err > FP8_TAIL[0]) <= FP8_TAIL[1], (np.mean(err > FP8_TAIL[0]), err.max())


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


class Fp8PeNet:
    def __init__(self, widths, seed=0, bias="zero", pooling=gl.GN_POOL_MAX_MEAN):
        self.w = synth.make_weights(widths, seed=seed, bias=bias)
        self.pooling = "sum" if pooling == gl.GN_POOL_SUM else "max_mean"
        self.model = gl.Model(self.w, gl.GN_FP8_FUSED, pooling)
        cal = synth.make_frame(CAL["h"], CAL["w"], CAL["K"], counts=CAL["counts"], seed=CAL["seed"])
        lat = self.model.encode(synth.make_scene(0))
        gl.glassnet_calibrate_fp8(self.model.handle, lat.handle, _dev(cal.gbuf), _dev(cal.tbuf),
                                  _dev(cal.counts), CAL["K"], CAL["h"], CAL["w"])
        self.lats = {}

    def latent(self, s):
        if s not in self.lats:
            self.lats[s] = self.model.encode(synth.make_scene(s))
        return self.lats[s]

    def render(self, frame, scene_seed=0):
        out = torch.full((3, frame.h, frame.w), float("nan"), device=DEV)
        self.model.render(self.latent(scene_seed), _dev(frame.gbuf),
                          _dev(frame.tbuf) if frame.K else None, _dev(frame.counts), out)
        self.model.check()
        torch.cuda.synchronize()
        return out.cpu().numpy().astype(np.float64)

    def ref(self, frame, scene_seed=0):
        return oracle.render_frame(self.w, synth.make_scene(scene_seed), frame.gbuf, frame.tbuf,
                                   frame.counts, pooling=self.pooling)


@pytest.fixture(scope="module")
def doubled_pe4(cuda_lib):
    return Fp8PeNet(synth.Widths(hidden=128, latent=256, pe_freqs=4), seed=0)


@pytest.fixture(scope="module")
def base_pe2(cuda_lib):
    return Fp8PeNet(synth.Widths(hidden=64, latent=128, pe_freqs=2), seed=1, bias="uniform")


@pytest.fixture(scope="module")
def doubled_pe4_sum(cuda_lib):
    return Fp8PeNet(synth.Widths(hidden=128, latent=256, pe_freqs=4), seed=2,
                    pooling=gl.GN_POOL_SUM)


CASES = [(64, 64, 8, "poisson3", 2), (96, 80, 3, "uniform", 3), (33, 47, 1, "all", 4),
         (40, 52, 0, "all", 5)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}-K{c[2]}-{c[3]}")
@pytest.mark.parametrize("net", ["doubled_pe4", "base_pe2"])
def test_fp8_pe_vs_oracle(net, case, request):
    n = request.getfixturevalue(net)
    h, w, K, counts, seed = case
    frame = synth.make_frame(h, w, K, counts=counts, seed=seed)
    assert_fp8_close(np.abs(n.render(frame, scene_seed=seed) - n.ref(frame, scene_seed=seed)))


@pytest.mark.parametrize("case", CASES[:2], ids=lambda c: f"{c[0]}x{c[1]}-K{c[2]}-{c[3]}")
def test_fp8_pe_sum_pooling_vs_oracle(doubled_pe4_sum, case):
    h, w, K, counts, seed = case
    frame = synth.make_frame(h, w, K, counts=counts, seed=seed)
    got = doubled_pe4_sum.render(frame, scene_seed=seed)
    assert_fp8_close(np.abs(got - doubled_pe4_sum.ref(frame, scene_seed=seed)))


def test_fp8_pe_bit_identical_under_permutations(doubled_pe4):
    frame = synth.make_frame(96, 64, 6, counts="uniform", seed=7)
    base = doubled_pe4.render(frame, scene_seed=7)
    for s in range(1, 5):
        assert np.array_equal(doubled_pe4.render(synth.permute_layers(frame, s), scene_seed=7), base)


def test_fp8_pe_full_512_K8_poisson_sampled(doubled_pe4):
    """512x512, K = 8, Poisson(3) counts, H = 128 with every input encoded at
    L = 4: the 64x64 crop at rows and columns 0..63 and 1024 sampled pixels
    against the oracle."""
    frame = synth.make_frame(512, 512, 8, counts="poisson3", seed=0)
    got = doubled_pe4.render(frame, scene_seed=0)
    crop = synth.Frame(gbuf=frame.gbuf[:, :64, :64].copy(), tbuf=frame.tbuf[:, :, :64, :64].copy(),
                       counts=frame.counts[:64, :64].copy())
    assert_fp8_close(np.abs(got[:, :64, :64] - doubled_pe4.ref(crop, scene_seed=0)))
    rng = np.random.default_rng(0)
    idx = rng.choice(512 * 512, 1024, replace=False)
    ys, xs = idx // 512, idx % 512
    samp = synth.Frame(gbuf=frame.gbuf[:, ys, xs][:, None, :].copy(),
                       tbuf=frame.tbuf[:, :, ys, xs][:, :, None, :].copy(),
                       counts=frame.counts[ys, xs][None, :].copy())
    exp = doubled_pe4.ref(samp, scene_seed=0)[:, 0, :]
    assert_fp8_close(np.abs(got[:, ys, xs] - exp))


@pytest.mark.parametrize("form", [dict(pe_freqs=5, r_kernel=1), dict(pe_freqs=2, r_kernel=3)],
                         ids=["L5", "L2-r3x3"])
def test_fp8_pe_forms_not_built_refused(cuda_lib, form):
    w = synth.make_weights(synth.Widths(hidden=64, latent=128, **form), seed=0)
    with pytest.raises(gl.GlassNetError) as ei:
        gl.Model(w, gl.GN_FP8_FUSED)
    assert ei.value.code == gl.GN_EUNSUPPORTED
