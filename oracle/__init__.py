"""Test infrastructure: the FP64 CPU oracle of the GlassNet per-pixel forward pass.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (its CPU
baseline and reference arm) may import this package.  The CUDA library never
does, and this package imports nothing from it.
"""
from .glassnet_oracle import (  # noqa: F401
    linear,
    relu,
    sigmoid,
    pe_freqs,
    positional_encoding,
    scene_encoder,
    per_layer_h,
    set_pool,
    set_sum,
    post_pool_rho,
    final_blend_B,
    render_R,
    render_R_frame,
    r_kernel,
    render_pixel,
    render_pixel_sum,
    render_frame,
    render_opaque_only,
    alpha_blend,
)
