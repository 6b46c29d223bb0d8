"""GB300-native sort-last image compositing and run-length pixel coding.

After Eilemann, "Parallel Rendering and Large Data Visualization" (arXiv
1902.08755), chapter 5: depth-sorted and ordered (alpha) compositing of N
partial images restricted to their regions of interest, and the per-component,
bit-swizzled RLE codec that carries partial images between compositing stages.

The work runs in hand-written CUDA kernels for sm_103a behind the C ABI of
include/ec.h (libec.so, built in-tree by ``build.build()``); this package is
its Python binding.  There is no CPU fallback: without libec.so every entry
point raises.
"""
from ._abi import (  # noqa: F401
    EC_MAX_SOURCES,
    EC_OK,
    EC_RGBA8,
    EC_RGBA16F,
    EC_RGBA32F,
    EC_RLE_CHUNK,
    EcError,
    load,
)
from .api import (  # noqa: F401
    SCHEDULES,
    Batch,
    Schedule,
    Context,
    Job,
    Prepared,
    Image,
    assemble_pixels,
    assemble_tiles,
    average,
    composite_alpha,
    composite_alpha_backward,
    composite_alpha_fwd_bwd,
    composite_depth,
    composite_depth_backward,
    default_context,
    detect_roi,
    pixel_layout,
    prepare_rle_compress_batch,
    prepare_rle_decompress_batch,
    prepare_yuv_batch,
    rle_compress,
    rle_compress_batch,
    rle_decompress,
    rle_decompress_batch,
    rle_max_size,
    schedule_geometry,
    yuv_batch,
    yuv_decode,
    yuv_encode,
    yuv_packed_shape,
)
from .autograd import alpha_composite, alpha_composite_fwd_bwd, depth_composite  # noqa: F401,E402
