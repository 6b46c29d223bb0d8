"""Seeded synthetic inputs shaped like the thesis's sort-last workloads.

This module is the only code shared by the CUDA path's tests/benchmark and the
oracle's.  It draws random numbers and paints them into buffers; it holds none
of the compositing or codec arithmetic.  Every stream is seeded from
``numpy.random.SeedSequence([190208755, cfg, source, ...])`` (PCG64).

Depth sources stand in for the thesis's polygonal renderings (David statue,
RTNeuron circuits, thesis 5.2.1/5.3): axis-aligned boxes with one RGB colour
(alpha 255) and one depth each, painted in drawing order (later boxes cover
earlier ones) over a cleared background (RGBA 0, depth 1.0) until a target
fraction of the frame is covered.  Sort-last sources give compact regions
(thesis 5.3), so optionally all boxes of a source fall in a random
sub-rectangle about twice the covered area.  The ROI is the bounding box of the
covered pixels; a cropped source stores only a 4-pixel-aligned rectangle around
it.  Alpha layers stand in for volume-rendered slabs: i.i.d. per pixel,
alpha ~ U[0, amax], colour = alpha * U[0, 1) per channel (premultiplied).
"""
from .frames import (  # noqa: F401
    ROOT_SEED,
    DepthSource,
    Tile,
    alpha_layers,
    depth_source,
    depth_sources,
    grad_weights,
    rng,
    smooth_image,
    uneven_tiles,
)
