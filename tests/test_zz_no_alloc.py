"""glassnet_render_fp32_static: the FP32 plain render for callers that cannot
allocate device memory when they render (their device memory is all handed out
up front by their own pooling allocator, or their frame loop must never block
in the allocator).  Its scratch is a 48 MiB static device array in the library,
mapped when the FP32 model is loaded.

Checked through the C ABI on two calls in a row with different frames (so
contents left in the shared scratch by the first call cannot leak into the
second): each output against the FP64 oracle and against glassnet_render
within the FP32 tolerance used by the other tests, and the device's free
memory unchanged across each call, the first one included.  This file is
collected last so that a run that stops at the first failure has already run
every other test.
"""
import numpy as np
import pytest
import torch

import oracle
from gen import synth
from paper_2405_19056_gb300 import glassnet as gl

pytestmark = pytest.mark.gpu

FP32_MAX = 1e-4
DEV = "cuda:0"


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


@pytest.fixture(scope="module")
def plain_weights():
    return synth.make_weights(synth.BASE_WIDTHS, seed=2, bias="uniform")


@pytest.fixture(scope="module")
def plain_model(cuda_lib, plain_weights):
    return gl.Model(plain_weights, gl.GN_FP32_PLAIN)


def _static_then_render(model, lat, frame):
    """The static render (free device memory measured around it), then
    glassnet_render of the same inputs."""
    K, h, w = frame.K, frame.h, frame.w
    g, t, c = _dev(frame.gbuf), _dev(frame.tbuf), _dev(frame.counts)
    ref = torch.full((3, h, w), float("nan"), device=DEV)
    got = torch.full((3, h, w), float("nan"), device=DEV)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    gl.glassnet_render_fp32_static(model.handle, lat.handle, g, t, c, K, h, w, got)
    model.check()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    gl.glassnet_render(model.handle, lat.handle, g, t, c, K, h, w, ref)
    model.check()
    return ref.cpu().numpy(), got.cpu().numpy(), free0 - free1


def test_static_scratch_render_matches_oracle_and_render_twice(plain_model, plain_weights):
    scene = synth.make_scene(4)
    lat = plain_model.encode(scene)
    frames = [synth.make_frame(96, 100, 4, counts="uniform", seed=41),
              synth.make_frame(64, 64, 2, counts="all", seed=42)]
    for i, f in enumerate(frames):
        ref, got, grew = _static_then_render(plain_model, lat, f)
        assert grew == 0, f"call {i + 1}: device free memory dropped by {grew} bytes"
        assert np.all(np.isfinite(got))
        want = oracle.render_frame(plain_weights, scene, f.gbuf, f.tbuf, f.counts)
        assert np.abs(got - want).max() <= FP32_MAX, f"call {i + 1} against the oracle"
        assert np.abs(got - ref).max() <= FP32_MAX, f"call {i + 1} against glassnet_render"


def test_static_scratch_rejects_frames_beyond_its_size(plain_model):
    lat = plain_model.encode(synth.make_scene(5))
    h = w = 512
    g = torch.zeros((14, h, w), device=DEV)
    t = torch.zeros((8, 12, h, w), device=DEV)
    c = torch.zeros((h, w), dtype=torch.uint8, device=DEV)
    out = torch.zeros((3, h, w), device=DEV)
    with pytest.raises(gl.GlassNetError) as ei:
        gl.glassnet_render_fp32_static(plain_model.handle, lat.handle, g, t, c, 8, h, w, out)
    assert ei.value.code == gl.GN_EINVAL
    assert "static scratch" in str(ei.value)


def test_static_scratch_needs_plain_model(cuda_lib):
    m = gl.Model(synth.make_weights(synth.BASE_WIDTHS, seed=2), gl.GN_BF16_FUSED)
    lat = m.encode(synth.make_scene(6))
    f = synth.make_frame(8, 8, 1, seed=6)
    out = torch.zeros((3, 8, 8), device=DEV)
    with pytest.raises(gl.GlassNetError) as ei:
        gl.glassnet_render_fp32_static(m.handle, lat.handle, _dev(f.gbuf), _dev(f.tbuf),
                                       _dev(f.counts), 1, 8, 8, out)
    assert ei.value.code == gl.GN_EINVAL
