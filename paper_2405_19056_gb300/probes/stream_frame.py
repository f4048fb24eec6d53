"""Streams the 512x512 K=8 Poisson(3) frame (seed 0, doubled widths) through
the pool API a few times: reset, the 8 layers (layer k covers the pixels
whose count exceeds k), resolve.  A driver for profiling the accumulate and
resolve launches:

    python paper_2405_19056_gb300/probes/stream_frame.py [frames]
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

import torch  # noqa: E402

from gen import synth  # noqa: E402
from paper_2405_19056_gb300 import glassnet as gl  # noqa: E402


def main():
    frames = int(sys.argv[1]) if len(sys.argv) > 1 else 3
    dev = torch.device("cuda")
    m = gl.Model(synth.make_weights(synth.DOUBLED_WIDTHS, seed=0), gl.GN_BF16_FUSED)
    lat = m.encode(synth.make_scene(0))
    f = synth.make_frame(512, 512, 8, counts="poisson3", seed=0)
    g, t, c = (torch.from_numpy(x).to(dev) for x in (f.gbuf, f.tbuf, f.counts))
    out = torch.empty((3, 512, 512), device=dev)
    covs = [(c > k).to(torch.uint8) for k in range(8)]
    pool = gl.glassnet_pool_create(m.handle, 512, 512)
    try:
        for _ in range(frames):
            gl.glassnet_pool_reset(pool)
            for k in range(8):
                gl.glassnet_accumulate_layer(m.handle, lat.handle, pool, t[k], covs[k])
            gl.glassnet_resolve(m.handle, lat.handle, pool, g, out)
        torch.cuda.synchronize()
        m.check()
    finally:
        gl.glassnet_pool_free(pool)
    print("streamed", frames, "frames")


if __name__ == "__main__":
    main()
