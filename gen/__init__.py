"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This package draws random numbers and lays them out in the buffer formats of
the GlassNet forward pass; it holds none of the network's arithmetic.
"""
from .synth import (  # noqa: F401
    GBUF_CHANNELS,
    TBUF_CHANNELS,
    SCENE_DIM,
    OUT_CHANNELS,
    WEIGHT_ORDER,
    Widths,
    BASE_WIDTHS,
    DOUBLED_WIDTHS,
    weight_shapes,
    make_weights,
    make_scene,
    make_counts,
    make_frame,
    permute_layers,
    Frame,
)
