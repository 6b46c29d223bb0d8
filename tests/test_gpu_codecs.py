"""GPU parity of the other compressors of thesis 5.5 against the oracle:

* basic 64-bit RLE (mode 0): the CUDA compressor emits the oracle's bytes, the
  CUDA decompressor inverts its own and the oracle's streams, batches that mix
  modes 0, 1 and 2 code each job as the oracle does, and malformed mode-0
  streams are reported (EC_ERR_CORRUPT) without writing outside the image;
* the lossy YUV compressor: packed images and their decodes are bit-exact to
  the oracle's (the transform is integer arithmetic), and the YUV -> RLE ->
  decode -> inverse pipeline equals the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_08755_gb300 as ec
import synthetic as S
from ec_testutil import np_of, require_gpu
from test_oracle_rle0 import _images

pytestmark = pytest.mark.gpu


def _u32(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda().view(torch.uint32)


def _bytes(buf, size):
    return buf[:int(size.item())].cpu().numpy().tobytes()


def _stream(b: bytes) -> torch.Tensor:
    return torch.from_numpy(np.frombuffer(b, np.uint8).copy()).cuda()


@pytest.mark.parametrize("name", sorted(_images().keys()))
def test_mode0_matches_oracle(name):
    require_gpu()
    img = _images()[name]
    h, w = img.shape
    buf, size = ec.rle_compress(_u32(img), 0)
    ec.default_context().check_status()
    got = _bytes(buf, size)
    assert got == oracle.rle_compress(img, 0)
    out = ec.rle_decompress(buf, w, h, src_size=len(got))
    ec.default_context().check_status()
    assert np.array_equal(np_of(out), img)


@pytest.mark.parametrize("shape", [(0, 0), (1, 1), (1, 2), (1, 3), (1, 4095), (1, 4097), (65, 127),
                                   (3, 5001), (300, 301)])
def test_mode0_shapes_and_pitch(shape):
    require_gpu()
    h, w = shape
    r = np.random.default_rng(h * 13 + w)
    pitch = w + 7
    img = (r.integers(0, 3, size=(h, pitch)) * 0x01010101).astype(np.uint32)
    buf, size = ec.rle_compress(_u32(img), 0, w=w)
    ec.default_context().check_status()
    got = _bytes(buf, size)
    assert got == oracle.rle_compress(img, 0, w=w)
    dst = torch.full((h, pitch), 0x5A5A5A5A, dtype=torch.int32, device="cuda").view(torch.uint32)
    ec.rle_decompress(_stream(got), w, h, dst=dst)
    ec.default_context().check_status()
    d = np_of(dst)
    assert np.array_equal(d[:, :w], img[:, :w])
    assert (d[:, w:].view(np.int32) == 0x5A5A5A5A).all()     # pitch padding untouched


def test_mixed_mode_batch():
    require_gpu()
    srcs = S.depth_sources(2, 6, 640, 360, 0.3, clustered=True, cropped=True)
    jobs, refs = [], []
    for i, s in enumerate(srcs):
        c = s.color.view(torch.int32).numpy().view(np.uint32)
        d = s.depth.numpy().view(np.uint32)
        for arr, mode in ((c, i % 3), (d, (i + 1) % 3)):
            jobs.append((_u32(arr), mode, None, None, None))
            refs.append(oracle.rle_compress(np.ascontiguousarray(arr), mode))
    outs = ec.rle_compress_batch(jobs)
    ec.default_context().check_status()
    for (buf, size), ref in zip(outs, refs):
        assert _bytes(buf, size) == ref
    dec = ec.rle_decompress_batch([(buf, j[0].shape[1], j[0].shape[0], None, int(size.item()))
                                   for (buf, size), j in zip(outs, jobs)])
    ec.default_context().check_status()
    for d, j in zip(dec, jobs):
        assert torch.equal(d.view(torch.int32), j[0].view(torch.int32))


def test_mode0_full_size_source():
    """A 1920x1080 cropped source's colour and depth, as the cfg2 workload holds them."""
    require_gpu()
    s = S.depth_sources(2, 16, 1920, 1080, 0.3, clustered=True, cropped=True)[3]
    for arr in (s.color.view(torch.int32).numpy().view(np.uint32), s.depth.numpy().view(np.uint32)):
        buf, size = ec.rle_compress(_u32(arr), 0)
        ec.default_context().check_status()
        assert _bytes(buf, size) == oracle.rle_compress(np.ascontiguousarray(arr), 0)


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_sparse_chunks_that_overflow_the_pool(mode):
    """Every chunk is sparse (126 noisy elements, then one value) but codes to
    more bytes than the compressor's scratch pool holds per chunk on average
    (512), so part of them find the pool full and are coded again from the
    image when placed.  A fresh context sizes its scratch for exactly this
    job (2048 chunks), so the overflow is certain."""
    require_gpu()
    r = np.random.default_rng(90 + mode)
    img = np.repeat(r.integers(0, 2**32, size=(2048, 1), dtype=np.uint64).astype(np.uint32), 4096, axis=1)
    img[:, :126] = r.integers(0, 2**32, size=(2048, 126), dtype=np.uint64).astype(np.uint32)
    ctx = ec.Context()
    try:
        buf, size = ec.rle_compress(_u32(img), mode, ctx=ctx)
        ctx.check_status()
        assert _bytes(buf, size) == oracle.rle_compress(img, mode)
    finally:
        ctx.close()


def test_mode0_without_allocation():
    require_gpu()
    img = _images()["boxes"]
    h, w = img.shape
    src = _u32(img)
    dst = torch.empty(ec.rle_max_size(w, h), dtype=torch.uint8, device="cuda")
    size = torch.zeros(1, dtype=torch.uint64, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    from paper_1902_08755_gb300 import _abi as A
    A.check(A.load().ec_rle_compress_noalloc(src.data_ptr(), w, h, w, 0, dst.data_ptr(), dst.numel(),
                                             size.data_ptr(), st.data_ptr(),
                                             torch.cuda.current_stream().cuda_stream), "noalloc")
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert _bytes(dst, size) == oracle.rle_compress(img, 0)


def _corrupt_mode0():
    img = S.depth_source(100, 70, 0.4, 43, 0).color.numpy()
    buf = oracle.rle_compress(img, 0)
    HDR = 32
    out = []
    x = bytearray(buf); x[28] = 4; out.append(("n_planes", bytes(x), 100, 70))
    x = bytearray(buf); x[6] = 3; out.append(("mode", bytes(x), 100, 70))
    out.append(("truncated", buf[:-1], 100, 70))
    x = bytearray(buf); x[HDR:HDR + 4] = (0).to_bytes(4, "little"); out.append(("end0", bytes(x), 100, 70))
    two = oracle.rle_compress(np.full((1, 4), 7, np.uint32), 0)
    y = bytearray(two); y[HDR + 4] = 0x80; out.append(("short", bytes(y), 4, 1))
    three = oracle.rle_compress(np.array([[1, 2, 3]], np.uint32), 0)
    out.append(("no_tail", three[:-4], 3, 1))
    lits = bytes([0x00]) + (7).to_bytes(4, "little") * 2 + bytes([0x00]) + (7).to_bytes(4, "little") * 2
    out.append(("over_bound", bytes(two[:HDR]) + (len(lits)).to_bytes(4, "little") + lits, 4, 1))
    return out


@pytest.mark.parametrize("case", range(7))
def test_mode0_decoder_rejects_corrupt_streams(case):
    """EC_ERR_CORRUPT is recorded, and nothing outside the w x h image is written."""
    require_gpu()
    from paper_1902_08755_gb300 import _abi as A
    name, bad, w, h = _corrupt_mode0()[case]
    assert oracle.rle_decompress_status(bad, w, h) == oracle.ECORRUPT
    ctx = ec.default_context()
    ctx.status_sync()
    pad = 64
    full = torch.full((h + 2, w + 2 * pad), 0x33333333, dtype=torch.int32, device="cuda").view(torch.uint32)
    dst = full[1:h + 1, pad:pad + w]
    ec.rle_decompress(_stream(bad), w, h, dst=dst, src_size=len(bad))
    assert ctx.status_sync() == A.EC_ERR_CORRUPT, name
    f = np_of(full).view(np.int32)
    assert (f[0] == 0x33333333).all() and (f[-1] == 0x33333333).all(), name
    assert (f[:, :pad] == 0x33333333).all() and (f[:, pad + w:] == 0x33333333).all(), name


@pytest.mark.parametrize("h,w", [(1, 1), (2, 2), (3, 5), (7, 1), (64, 64), (97, 131), (1080, 1920)])
def test_yuv_matches_oracle(h, w):
    require_gpu()
    img = np.random.default_rng(h * 7 + w).integers(0, 2**32, size=(h, w + 3), dtype=np.uint64).astype(np.uint32)
    packed = ec.yuv_encode(_u32(img), w=w)
    ec.default_context().check_status()
    ref = oracle.yuv_encode(np.ascontiguousarray(img), w=w)
    assert np.array_equal(np_of(packed), ref)
    out = torch.full((h, w + 5), 0x11111111, dtype=torch.int32, device="cuda").view(torch.uint32)
    ec.yuv_decode(packed, w, h, out=out)
    ec.default_context().check_status()
    o = np_of(out)
    assert np.array_equal(o[:, :w], oracle.yuv_decode(ref, w, h))
    assert (o[:, w:].view(np.int32) == 0x11111111).all()


def test_yuv_rle_pipeline_matches_oracle():
    """Colour of a cropped 1080p source: YUV -> RLE (mode 1) -> decompress ->
    inverse, on the GPU and in the oracle; identical streams and frames."""
    require_gpu()
    s = S.depth_sources(2, 16, 1920, 1080, 0.3, clustered=True, cropped=True)[5]
    img = s.color.view(torch.int32).numpy().view(np.uint32)
    h, w = img.shape
    packed = ec.yuv_encode(_u32(img))
    buf, size = ec.rle_compress(packed, 1)
    ec.default_context().check_status()
    ref_p = oracle.yuv_encode(np.ascontiguousarray(img))
    ref_s = oracle.rle_compress(ref_p, 1)
    assert _bytes(buf, size) == ref_s
    dec = ec.rle_decompress(buf, packed.shape[1], packed.shape[0], src_size=int(size.item()))
    out = ec.yuv_decode(dec, w, h)
    ec.default_context().check_status()
    assert np.array_equal(np_of(out), oracle.yuv_decode(ref_p, w, h))


def test_yuv_batch_matches_single_calls():
    """One launch over images of different sizes and pitches gives what the
    oracle gives for each."""
    require_gpu()
    r = np.random.default_rng(9)
    shapes = [(1, 1), (5, 3), (64, 129), (333, 200), (2, 8)]
    imgs = [r.integers(0, 2**32, size=(h, w + 2), dtype=np.uint64).astype(np.uint32) for h, w in shapes]
    srcs = [_u32(i) for i in imgs]
    packed = [torch.zeros(ec.yuv_packed_shape(w, h), dtype=torch.int32, device="cuda").view(torch.uint32)
              for h, w in shapes]
    ec.yuv_batch([(s, p, w, h) for s, p, (h, w) in zip(srcs, packed, shapes)], True)
    outs = [torch.zeros((h, w), dtype=torch.int32, device="cuda").view(torch.uint32) for h, w in shapes]
    ec.yuv_batch([(p, o, w, h) for p, o, (h, w) in zip(packed, outs, shapes)], False)
    ec.default_context().check_status()
    for img, p, o, (h, w) in zip(imgs, packed, outs, shapes):
        ref = oracle.yuv_encode(np.ascontiguousarray(img), w=w)
        assert np.array_equal(np_of(p), ref)
        assert np.array_equal(np_of(o), oracle.yuv_decode(ref, w, h))


@pytest.mark.parametrize("h,w,pad,col,ppad", [
    (9, 13, 3, 0, 1),      # pitch 16: 16-byte quads, ragged last block pair, odd height
    (8, 12, 0, 0, 1),      # 16-byte quads, packed pitch 7 (no 8-byte word pairs)
    (5, 7, 1, 1, 0),       # view one column in: 4-byte aligned only, scalar path
    (6, 10, 2, 2, 2),      # view two columns in: 8-byte aligned, 8-byte pairs
    (7, 17, 3, 4, 1),      # view four columns in: 16-byte aligned again
    (1, 4, 0, 0, 0),       # one pixel row
    (33, 530, 2, 0, 3),    # several CTA tiles wide, ragged
])
def test_yuv_access_widths(h, w, pad, col, ppad):
    """The encoder and decoder take 16-byte, 8-byte or 4-byte accesses on the
    RGBA side and 8- or 4-byte ones on the packed side, by alignment; every
    combination gives the oracle's bits and writes nothing outside its image."""
    require_gpu()
    r = np.random.default_rng(h * 1000 + w * 10 + col)
    big = r.integers(0, 2**32, size=(h, col + w + pad), dtype=np.uint64).astype(np.uint32)
    src = _u32(big)[:, col:col + w]
    rows, words = ec.yuv_packed_shape(w, h)
    pbig = torch.full((rows, words + ppad), 0x22222222, dtype=torch.int32, device="cuda").view(torch.uint32)
    packed = pbig[:, :words]
    ec.yuv_encode(src, w=w, out=packed)
    ec.default_context().check_status()
    ref = oracle.yuv_encode(np.ascontiguousarray(big[:, col:col + w]))
    assert np.array_equal(np_of(packed), ref)
    assert (np_of(pbig)[:, words:].view(np.int32) == 0x22222222).all()
    obig = torch.full((h, col + w + pad), 0x11111111, dtype=torch.int32, device="cuda").view(torch.uint32)
    ec.yuv_decode(packed, w, h, out=obig[:, col:col + w])
    ec.default_context().check_status()
    o = np_of(obig)
    assert np.array_equal(o[:, col:col + w], oracle.yuv_decode(ref, w, h))
    assert (o[:, :col].view(np.int32) == 0x11111111).all() and (o[:, col + w:].view(np.int32) == 0x11111111).all()
