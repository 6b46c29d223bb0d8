"""ec_rle_compress_noalloc, the compressor variant for callers that cannot
allocate device memory (its scratch is a fixed array inside libec): called
through the C ABI twice in a row, it must write exactly the bytes and size that
ec_rle_compress writes for the same image, and refuse images beyond its fixed
scratch.  Collected last on purpose, so that a failure here stops a run only
after every other test has run; it also passes alone in a fresh process."""
import ctypes as C

import numpy as np
import pytest
import torch

import paper_1902_08755_gb300 as ec
import synthetic as S
from paper_1902_08755_gb300 import _abi as A

pytestmark = pytest.mark.gpu


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _noalloc(src: torch.Tensor, mode: int):
    lib = ec.load()
    h, w = src.shape
    cap = ec.rle_max_size(w, h)
    dst = torch.full((cap,), 0xAB, dtype=torch.uint8, device=src.device)
    size = torch.zeros(1, dtype=torch.uint64, device=src.device)
    status = torch.zeros(1, dtype=torch.int32, device=src.device)
    rc = lib.ec_rle_compress_noalloc(src.data_ptr(), w, h, src.stride(0), mode, dst.data_ptr(), cap,
                                     size.data_ptr(), status.data_ptr(), _stream())
    assert rc == A.EC_OK, A.STATUS_NAMES.get(rc, rc)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    n = int(size.item())
    return dst[:n].cpu().numpy().tobytes(), n


def _with_ctx(src: torch.Tensor, mode: int):
    buf, size = ec.rle_compress(src, mode)
    ec.default_context().check_status()
    n = int(size.item())
    return buf[:n].cpu().numpy().tobytes(), n


def test_noalloc_matches_context_compressor_twice():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    a = S.depth_source(1920, 1080, 0.3, 2, 0, clustered=True, cropped=True, device="cuda")
    b = S.depth_source(640, 480, 0.4, 1, 3, device="cuda")
    cases = [(a.color, 2), (b.depth.view(torch.uint32), 1)]   # two calls in a row, different sizes
    for src, mode in cases:
        got = _noalloc(src, mode)
        ref = _with_ctx(src, mode)
        assert got[1] == ref[1]
        assert got[0] == ref[0]


def test_noalloc_refuses_images_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    lib = ec.load()
    n = A.EC_RLE_NOALLOC_MAX_CHUNKS * A.EC_RLE_CHUNK + 1
    rc = lib.ec_rle_compress_noalloc(None, n, 1, n, 1, None, 0, None, None, _stream())
    assert rc == A.EC_ERR_UNSUPPORTED
