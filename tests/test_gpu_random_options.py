"""Seeded random cases over every model option and ragged frame shapes,
through the C ABI: pooling ([max ; mean] or the sum form), positional
encoding (both widths), R's first layer (1x1 or 3x3), widths, frame sizes from a
single pixel to several 128-column strips, K from 0 to 8 and every count
distribution.  Each case renders with the BF16 fused path and the FP32 plain
path and checks both against the FP64 oracle (BF16: max |err| <= 2e-2, mean
<= 3e-3; FP32: max |err| <= 1e-4).
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


def _case(seed):
    rng = np.random.default_rng([seed, 77])
    H = int(rng.choice([64, 128]))
    pe = int(rng.choice([0, 0, 2, 4]))
    rk = int(rng.choice([1, 1, 3]))
    pooling = str(rng.choice(["max_mean", "sum"]))
    h = int(rng.integers(1, 48))
    w = int(rng.integers(1, 300))
    K = int(rng.integers(0, 9))
    counts = str(rng.choice(["all", "uniform", "poisson3"]))
    return dict(H=H, pe=pe, rk=rk, pooling=pooling, h=h, w=w, K=K, counts=counts, seed=seed)


CASES = [_case(s) for s in range(18)]


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _render(m, scene, f):
    lat = m.encode(scene)
    out = torch.full((3, f.h, f.w), float("nan"), device=DEV)
    m.render(lat, _dev(f.gbuf), _dev(f.tbuf) if f.tbuf.shape[0] else None, _dev(f.counts), out)
    m.check()
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "H{H}-L{pe}-R{rk}-{pooling}-{h}x{w}-K{K}-{counts}".format(**c))
def test_random_option_case(cuda_lib, case):
    w = synth.make_weights(synth.Widths(case["H"], 2 * case["H"], case["pe"], case["rk"]),
                           seed=case["seed"], bias="uniform")
    pl = gl.GN_POOL_SUM if case["pooling"] == "sum" else gl.GN_POOL_MAX_MEAN
    scene = synth.make_scene(case["seed"])
    f = synth.make_frame(case["h"], case["w"], case["K"], counts=case["counts"], seed=case["seed"])
    exp = oracle.render_frame(w, scene, f.gbuf, f.tbuf, f.counts, pooling=case["pooling"])
    got = _render(gl.Model(w, gl.GN_BF16_FUSED, pl), scene, f)
    err = np.abs(got - exp)
    assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (err.max(), err.mean())
    plain = _render(gl.Model(w, gl.GN_FP32_PLAIN, pl), scene, f)
    assert np.abs(plain - exp).max() <= FP32_MAX, np.abs(plain - exp).max()
