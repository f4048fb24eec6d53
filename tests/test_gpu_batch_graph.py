"""Batched persistent launch and CUDA graphs of it, through the C ABI.

The batched workload: 16 frames, each a square resolution drawn from a size
set, K ~ U{2..8}, every slot valid, 4 scenes (frame i uses scene i mod 4).
Every frame of a batch must equal its own single-frame render bit for bit,
a graph replay must equal the direct batched launch bit for bit, and sampled
pixels must match the FP64 oracle within the BF16 tolerance.
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


class Batch:
    """Host frames, device buffers and latents of one batch spec list."""

    def __init__(self, model, specs, seed):
        self.specs = specs
        self.scenes = [synth.make_scene(100 + s) for s in range(4)]
        self.lats = [model.encode(sc) for sc in self.scenes]
        self.host = [synth.make_frame(sp.h, sp.w, sp.K, counts="all", seed=seed + i)
                     for i, sp in enumerate(specs)]
        self.frames = []
        for sp, f in zip(specs, self.host):
            self.frames.append(dict(latent=self.lats[sp.scene].handle, gbuf=_dev(f.gbuf),
                                    tbuf=_dev(f.tbuf), layer_count=_dev(f.counts), K=sp.K,
                                    h=sp.h, w=sp.w,
                                    out=torch.full((3, sp.h, sp.w), float("nan"), device=DEV)))

    def outputs(self):
        torch.cuda.synchronize()
        return [fr["out"].cpu().numpy().astype(np.float64) for fr in self.frames]

    def clear_outputs(self):
        for fr in self.frames:
            fr["out"].fill_(float("nan"))


@pytest.fixture(scope="module")
def net(cuda_lib):
    w = synth.make_weights(synth.DOUBLED_WIDTHS, seed=0)
    return w, gl.Model(w, gl.GN_BF16_FUSED)


def _oracle_samples(w, scene, f, n, seed):
    """FP64 oracle at n sampled pixels of frame f: (ys, xs, rgb [3][n])."""
    rng = np.random.default_rng(seed)
    idx = rng.choice(f.h * f.w, min(n, f.h * f.w), replace=False)
    ys, xs = idx // f.w, idx % f.w
    samp = synth.Frame(gbuf=f.gbuf[:, ys, xs][:, None, :].copy(),
                       tbuf=f.tbuf[:, :, ys, xs][:, :, None, :].copy(),
                       counts=f.counts[ys, xs][None, :].copy())
    return ys, xs, oracle.render_frame(w, scene, samp.gbuf, samp.tbuf, samp.counts)[:, 0, :]


SMALL_SIZES = (32, 64, 128, 256)


def test_batch_equals_single_renders_and_oracle(net):
    w, m = net
    b = Batch(m, synth.batch_specs(16, SMALL_SIZES, seed=1), seed=200)
    gl.glassnet_render_batch(m.handle, b.frames)
    m.check()
    got = b.outputs()
    for i, (sp, f) in enumerate(zip(b.specs, b.host)):
        single = torch.full((3, sp.h, sp.w), float("nan"), device=DEV)
        m.render(b.lats[sp.scene], _dev(f.gbuf), _dev(f.tbuf), _dev(f.counts), single)
        m.check()
        assert np.array_equal(got[i], single.cpu().numpy().astype(np.float64)), (i, sp)
        ys, xs, exp = _oracle_samples(w, b.scenes[sp.scene], f, 48, seed=i)
        err = np.abs(got[i][:, ys, xs] - exp)
        assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (i, sp, err.max(), err.mean())


def test_graph_replay_equals_batch_and_sees_new_contents(net):
    w, m = net
    specs = synth.batch_specs(16, SMALL_SIZES, seed=2)
    b = Batch(m, specs, seed=300)
    gl.glassnet_render_batch(m.handle, b.frames)
    m.check()
    direct = b.outputs()
    g = gl.glassnet_graph_create(m.handle, b.frames)
    try:
        b.clear_outputs()
        gl.glassnet_graph_launch(g)
        m.check()
        for i, out in enumerate(b.outputs()):
            assert np.array_equal(out, direct[i]), i
        # new inputs written into the captured buffers: the replay reads them
        fresh = [synth.make_frame(sp.h, sp.w, sp.K, counts="all", seed=900 + i)
                 for i, sp in enumerate(specs)]
        for fr, f in zip(b.frames, fresh):
            fr["gbuf"].copy_(_dev(f.gbuf))
            fr["tbuf"].copy_(_dev(f.tbuf))
        b.clear_outputs()
        gl.glassnet_graph_launch(g)
        m.check()
        replay = b.outputs()
        b.clear_outputs()
        gl.glassnet_render_batch(m.handle, b.frames)
        m.check()
        for i, out in enumerate(b.outputs()):
            assert np.array_equal(replay[i], out), i
            assert not np.array_equal(out, direct[i]), i
    finally:
        gl.glassnet_graph_free(g)


def test_graph_update_rebinds_and_rejects_other_shapes(net):
    w, m = net
    specs = synth.batch_specs(16, SMALL_SIZES, seed=3)
    b1 = Batch(m, specs, seed=400)
    b2 = Batch(m, specs, seed=500)
    g = gl.glassnet_graph_create(m.handle, b1.frames)
    try:
        gl.glassnet_graph_update(g, b2.frames)
        gl.glassnet_graph_launch(g)
        m.check()
        via_graph = b2.outputs()
        b2.clear_outputs()
        gl.glassnet_render_batch(m.handle, b2.frames)
        m.check()
        for i, out in enumerate(b2.outputs()):
            assert np.array_equal(via_graph[i], out), i
        other = [dict(fr) for fr in b2.frames]
        other[0]["K"] = other[0]["K"] - 1  # a different shape
        with pytest.raises(gl.GlassNetError) as ei:
            gl.glassnet_graph_update(g, other)
        assert ei.value.code == gl.GN_EINVAL
        with pytest.raises(gl.GlassNetError):
            gl.glassnet_graph_update(g, b2.frames[:15])
    finally:
        gl.glassnet_graph_free(g)


def test_batch_full_size_graph_sampled(net):
    """The full batched workload (sizes 128..1024, 6.46 Mpx for seed 0) as
    the bench runs it: a graph replay, checked against the direct batched
    launch bit for bit and against the oracle at 24 pixels per frame."""
    w, m = net
    specs = synth.batch_specs(16, synth.BATCH_SIZES_FULL, seed=0)
    b = Batch(m, specs, seed=0)
    g = gl.glassnet_graph_create(m.handle, b.frames)
    try:
        gl.glassnet_graph_launch(g)
        m.check()
        via_graph = b.outputs()
    finally:
        gl.glassnet_graph_free(g)
    b.clear_outputs()
    gl.glassnet_render_batch(m.handle, b.frames)
    m.check()
    for i, out in enumerate(b.outputs()):
        assert np.array_equal(via_graph[i], out), i
    for i, (sp, f) in enumerate(zip(specs, b.host)):
        ys, xs, exp = _oracle_samples(w, b.scenes[sp.scene], f, 24, seed=50 + i)
        err = np.abs(via_graph[i][:, ys, xs] - exp)
        assert err.max() <= BF16_MAX and err.mean() <= BF16_MEAN, (i, sp, err.max(), err.mean())
