"""The largest frames the C ABI accepts, and the first ones it refuses.

glassnet_render takes a frame when 12 max(K, 1) h w < 2^31.  At the edge the
fused kernel's 32-bit plane offsets reach their largest values: at K = 8 the
last slot's last channel plane ends just below 2^31 floats, and at K = 0 the
G-buffer's 14 planes hold 2.5 x 10^9 floats, past the signed 32-bit range.

Each accepted frame is a small seeded synthetic frame repeated down the rows
(on the device).  Every pixel of the large frame must come out bit-identical
to the same pixel rendered in the small frame by itself (per-pixel results do
not depend on where the tile falls, nor on the frame size), and the small
frame's render is compared with the FP64 oracle: BF16 max |err| <= 2e-2,
mean <= 3e-3; FP8 (calibrated on a seed-1 128x128 K=8 frame) max <= 0.1,
mean <= 1e-2 and at most 1 in 10^4 values above 6e-2.

The FP8 bound for these populations (52,030 and 93,639 distinct pixels, where
the 64x64 crops of test_gpu_fp8.py hold 4,096) comes from E4M3's rounding,
with no saturation: the input channels have per-channel scales at 8x and the
hidden activations 4x their calibrated range, and a CPU emulation of every
quantisation point of the kernel (E4M3 round-to-nearest-even of each
operand, per-channel weight scales, exact pooling of BF16-rounded phi
outputs) gives at most 0.053 (K = 8) and 0.060 (K = 0) on these frames, at
mean 0.0031 and 0.0030, with no value above 6e-2 at K = 8 and 1 in 2.8 x 10^5
at K = 0.  The kernel measured up to 1.3x its emulation's largest error
before (0.085 against 0.066 with the per-tensor scales): the bound takes
that factor with some room, 0.1.  E4M3 keeps 3 mantissa bits (a relative
step of 2^-3) in every operand of seven GEMMs, so the largest error of a
population grows with its size while the mean does not.
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
# max, mean, and (threshold, largest fraction of values above it)
TOL = {"bf16": (BF16_MAX, BF16_MEAN, None), "fp8": (0.1, 1e-2, (6e-2, 1e-4))}

# (K, h, w, rows of the repeated small frame): 12 max(K, 1) h w < 2^31, and
# one more column reaches it (checked on the CPU in test_abi_cpu.py)
EDGE_CASES = [(8, 4729, 4730, 11), (0, 13377, 13377, 7)]


@pytest.fixture(scope="module")
def doubled(cuda_lib):
    w = synth.make_weights(synth.DOUBLED_WIDTHS, seed=9, bias="uniform")
    return w, gl.Model(w, gl.GN_BF16_FUSED)


@pytest.fixture(scope="module")
def doubled_fp8(doubled):
    w, _ = doubled
    m = gl.Model(w, gl.GN_FP8_FUSED)
    cal = synth.make_frame(128, 128, 8, counts="poisson3", seed=1)
    lat = m.encode(synth.make_scene(0))

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)

    gl.glassnet_calibrate_fp8(m.handle, lat.handle, dev(cal.gbuf), dev(cal.tbuf), dev(cal.counts),
                              8, 128, 128)
    return w, m


@pytest.mark.parametrize("K,h,w,rows", EDGE_CASES, ids=["K8", "K0"])
def test_one_column_more_is_refused(doubled, K, h, w, rows):
    """Refused before any launch: the buffers passed are far too small to be
    read at all."""
    _, m = doubled
    lat = m.encode(synth.make_scene(2))
    g = torch.zeros(16, device=DEV)
    t = torch.zeros(16, device=DEV) if K else None
    c = torch.zeros(16, dtype=torch.uint8, device=DEV)
    out = torch.zeros(16, device=DEV)
    with pytest.raises(gl.GlassNetError) as e:
        gl.glassnet_render(m.handle, lat.handle, g, t, c, K, h, w + 1, out)
    assert e.value.code == gl.GN_EINVAL
    m.check()


@pytest.mark.parametrize("precision", ["bf16", "fp8"])
@pytest.mark.parametrize("K,h,w,rows", EDGE_CASES, ids=["K8", "K0"])
def test_largest_frame_matches_the_oracle(request, K, h, w, rows, precision):
    weights, m = request.getfixturevalue("doubled" if precision == "bf16" else "doubled_fp8")
    scene = synth.make_scene(2)
    f = synth.make_frame(rows, w, K, counts="poisson3", seed=21)
    exp = oracle.render_frame(weights, scene, f.gbuf, f.tbuf, f.counts)  # [3][rows][w]
    idx = torch.arange(h, device=DEV) % rows  # row y of the frame is row y mod rows
    g = torch.from_numpy(f.gbuf).to(DEV).index_select(1, idx)
    t = torch.from_numpy(f.tbuf).to(DEV).index_select(2, idx) if K else None
    c = torch.from_numpy(f.counts).to(DEV).index_select(0, idx)
    out = torch.full((3, h, w), float("nan"), device=DEV)
    lat = m.encode(scene)
    m.render(lat, g, t, c, out)
    small = torch.full((3, rows, w), float("nan"), device=DEV)
    m.render(lat, torch.from_numpy(f.gbuf).to(DEV), torch.from_numpy(f.tbuf).to(DEV) if K else None,
             torch.from_numpy(f.counts).to(DEV), small)
    m.check()
    torch.cuda.synchronize()
    del g, t, c
    assert bool(torch.isfinite(out).all())
    # every pixel of the large frame == the same pixel of the small frame
    for y0 in range(0, h, 1024):  # in bands, to bound the temporaries
        assert torch.equal(out[:, y0:y0 + 1024], small.index_select(1, idx[y0:y0 + 1024])), y0
    del out
    torch.cuda.empty_cache()
    err = np.abs(small.cpu().numpy().astype(np.float64) - exp)
    tol_max, tol_mean, tail = TOL[precision]
    assert err.max() <= tol_max and err.mean() <= tol_mean, (err.max(), err.mean())
    if tail:
        worst = np.unravel_index(np.argmax(err), err.shape)
        assert np.mean(err > tail[0]) <= tail[1], (np.mean(err > tail[0]), err.max(), worst)


def _stack_rows(f, rows_idx):
    """The frame whose row j is row rows_idx[j] of f."""
    return synth.Frame(gbuf=np.ascontiguousarray(f.gbuf[:, rows_idx]),
                       tbuf=np.ascontiguousarray(f.tbuf[:, :, rows_idx]),
                       counts=np.ascontiguousarray(f.counts[rows_idx]))


@pytest.mark.parametrize("K,h,w,rows", [(8, 4729, 4730, 5), (0, 13377, 13377, 7)], ids=["K8", "K0"])
def test_largest_frame_with_the_3x3_R(cuda_lib, K, h, w, rows):
    """The 3x3 R at the edge sizes: the neural buffer is 5.7 GB (K = 8) or
    45.8 GB (K = 0), past 32-bit byte offsets.  With the rows repeating,
    a pixel away from the top and bottom edges sees a periodic 3x3
    neighbourhood, i.e. the middle block of three stacked copies; the top and
    bottom rows see the zero padding."""
    weights = synth.make_weights(synth.Widths(128, 256, 0, 3), seed=4, bias="uniform")
    m = gl.Model(weights, gl.GN_BF16_FUSED)
    scene = synth.make_scene(3)
    f = synth.make_frame(rows, w, K, counts="poisson3", seed=22)
    r = np.arange(rows)
    mid = oracle.render_frame(weights, scene, *_fields(_stack_rows(f, np.concatenate([r, r, r]))))
    top = oracle.render_frame(weights, scene, *_fields(f))[:, 0]
    rb = (h - 1) % rows
    bot = oracle.render_frame(weights, scene, *_fields(_stack_rows(f, np.array([(rb - 1) % rows, rb]))))[:, 1]
    idx = torch.arange(h, device=DEV) % rows
    g = torch.from_numpy(f.gbuf).to(DEV).index_select(1, idx)
    t = torch.from_numpy(f.tbuf).to(DEV).index_select(2, idx) if K else None
    c = torch.from_numpy(f.counts).to(DEV).index_select(0, idx)
    out = torch.full((3, h, w), float("nan"), device=DEV)
    lat = m.encode(scene)
    m.render(lat, g, t, c, out)
    m.check()
    torch.cuda.synchronize()
    del g, t, c
    m.close()  # frees the neural buffer
    assert bool(torch.isfinite(out).all())
    assert torch.equal(out[:, 1 + rows:h - 1], out[:, 1:h - 1 - rows])
    ref = torch.from_numpy(mid[:, rows:2 * rows].astype(np.float32)).to(DEV)
    err_max, err_sum = 0.0, 0.0
    for y0 in range(1, h - 1, 1024):
        y1 = min(y0 + 1024, h - 1)
        d = (out[:, y0:y1] - ref.index_select(1, idx[y0:y1])).abs()
        err_max = max(err_max, float(d.max()))
        err_sum += float(d.double().sum())
    for y, e in ((0, top), (h - 1, bot)):
        d = (out[:, y].double().cpu().numpy() - e)
        err_max = max(err_max, float(np.abs(d).max()))
        err_sum += float(np.abs(d).sum())
    err_mean = err_sum / (3 * h * w)
    assert err_max <= BF16_MAX and err_mean <= BF16_MEAN, (err_max, err_mean)
    del out
    torch.cuda.empty_cache()


def _fields(f):
    return f.gbuf, f.tbuf, f.counts
