"""GPU parity of the run-length codec against the oracle (thesis 5.5.1): the CUDA
compressor must emit the oracle's bytes exactly, the CUDA decompressor must
invert both its own and the oracle's streams, malformed streams must be
reported (EC_ERR_CORRUPT) without faults, and capacity is checked up front."""
import numpy as np
import pytest
import torch

import oracle
import paper_1902_08755_gb300 as ec
import synthetic as S
from ec_testutil import np_of, require_gpu
from test_oracle_rle import _adversarial_images

pytestmark = pytest.mark.gpu


def _u32(a: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int32)).cuda().view(torch.uint32)


def _gpu_bytes(buf: torch.Tensor, size: torch.Tensor) -> bytes:
    n = int(size.item())
    return buf[:n].cpu().numpy().tobytes()


def _roundtrip_check(img: np.ndarray, mode: int, w=None):
    h, pitch = img.shape
    w = pitch if w is None else w
    buf, size = ec.rle_compress(_u32(img), mode, w=w)
    ec.default_context().check_status()
    got = _gpu_bytes(buf, size)
    ref = oracle.rle_compress(np.ascontiguousarray(img), mode, w=w)
    assert got == ref
    out = ec.rle_decompress(buf, w, h, src_size=len(got))
    ec.default_context().check_status()
    assert np.array_equal(np_of(out), img[:, :w])
    # the decoder also reads the oracle's stream
    ob = torch.from_numpy(np.frombuffer(ref, np.uint8).copy()).cuda()
    out2 = ec.rle_decompress(ob, w, h)
    ec.default_context().check_status()
    assert np.array_equal(np_of(out2), img[:, :w])


@pytest.mark.parametrize("name", sorted(_adversarial_images().keys()))
@pytest.mark.parametrize("mode", [1, 2])
def test_adversarial_patterns_bit_exact(name, mode):
    require_gpu()
    _roundtrip_check(_adversarial_images()[name], mode)


@pytest.mark.parametrize("shape", [(1, 1), (1, 4095), (1, 4096), (1, 4097), (2, 3), (65, 127),
                                   (3, 5000), (40, 4096), (1080, 1920),
                                   # contiguous rows that are not 16-byte groups, 4k elements in all
                                   (12, 999), (4, 4099), (1050, 498)])
@pytest.mark.parametrize("mode", [1, 2])
def test_shapes_and_pitches(shape, mode):
    require_gpu()
    h, w = shape
    r = np.random.default_rng(h * 31 + w)
    img = (r.integers(0, 3, size=(h, w + 5)) * np.uint32(0x01010101)).astype(np.uint32)
    img ^= (r.random((h, w + 5)) < 0.1).astype(np.uint32) * np.uint32(0x00FF0F00)
    _roundtrip_check(img, mode, w=w)         # pitch w+5: element path
    _roundtrip_check(np.ascontiguousarray(img[:, :w]), mode)


@pytest.mark.parametrize("mode", [1, 2])
def test_cfg1_and_cfg2_sources(mode):
    require_gpu()
    for s in S.depth_sources(1, 4, 640, 480, 0.4) + S.depth_sources(2, 16, 1920, 1080, 0.3,
                                                                      clustered=True, cropped=True)[:6]:
        _roundtrip_check(np_of(s.color), mode)
        _roundtrip_check(np_of(s.depth).view(np.uint32), 1)


def test_batch_equals_single_calls():
    require_gpu()
    imgs = [np.zeros((0, 0), np.uint32), S.depth_source(333, 77, 0.4, 80, 0).color.numpy(),
            _adversarial_images()["noise"], np.full((5, 4096), 3, np.uint32),
            S.smooth_image(640, 200)]
    jobs = [(_u32(im), 1 + i % 2, None, None, None) for i, im in enumerate(imgs)]
    outs = ec.rle_compress_batch(jobs)
    ec.default_context().check_status()
    for i, ((buf, size), im) in enumerate(zip(outs, imgs)):
        ref = oracle.rle_compress(np.ascontiguousarray(im), 1 + i % 2, w=im.shape[1] if im.size else 0)
        assert _gpu_bytes(buf, size) == ref
    dec = ec.rle_decompress_batch([(b, im.shape[1], im.shape[0], None, None)
                                   for (b, _), im in zip(outs, imgs)])
    ec.default_context().check_status()
    for d, im in zip(dec, imgs):
        assert np.array_equal(np_of(d), im)


def test_unaligned_source_pointer():
    require_gpu()
    img = S.depth_source(256, 64, 0.4, 81, 0).color.numpy()
    big = torch.zeros((64 * 256 + 1,), dtype=torch.int32, device="cuda")
    big[1:] = _u32(img).view(torch.int32).reshape(-1)
    src = big[1:].view(torch.uint32).reshape(64, 256)
    buf, size = ec.rle_compress(src, 2)
    ec.default_context().check_status()
    assert _gpu_bytes(buf, size) == oracle.rle_compress(img, 2)


def test_capacity_checked_up_front():
    require_gpu()
    img = _u32(np.zeros((10, 10), np.uint32))
    small = torch.empty(ec.rle_max_size(10, 10) - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(ec.EcError) as e:
        ec.rle_compress(img, 1, dst=small)
    assert e.value.code == 2


def _corruptions(buf: bytes):
    from test_oracle_rle import _corruptions as oc
    yield from oc(buf)


def test_corrupt_streams_reported_not_faulting():
    require_gpu()
    img = S.depth_source(100, 70, 0.4, 43, 0).color.numpy()
    good = oracle.rle_compress(img, 2)
    for name, bad in _corruptions(good):
        t = torch.from_numpy(np.frombuffer(bad, np.uint8).copy()).cuda()
        dst = torch.full((70, 100), 7, dtype=torch.int32, device="cuda").view(torch.uint32)
        ec.rle_decompress(t, 100, 70, dst=dst, src_size=len(bad))
        assert ec.default_context().status_sync() == 4, name
    # a stream whose tokens parse but leave a plane one byte short
    four = bytearray(oracle.rle_compress(np.full((1, 4), 0x01010101, np.uint32), 1))
    four[48] = 0x82
    t = torch.from_numpy(np.frombuffer(bytes(four), np.uint8).copy()).cuda()
    ec.rle_decompress(t, 4, 1)
    assert ec.default_context().status_sync() == 4
    # wrong destination size
    t = torch.from_numpy(np.frombuffer(good, np.uint8).copy()).cuda()
    ec.rle_decompress(t, 99, 70)
    assert ec.default_context().status_sync() == 4
    # the context is still usable afterwards
    _roundtrip_check(img, 2)


@pytest.mark.parametrize("seed", range(10))
def test_random_bit_flips_never_fault(seed):
    require_gpu()
    r = np.random.default_rng(seed)
    img = S.depth_source(64, 64, 0.4, 44, seed % 3).color.numpy()
    buf = bytearray(oracle.rle_compress(img, 1))
    for _ in range(8):
        i = int(r.integers(0, len(buf)))
        buf[i] ^= 1 << int(r.integers(0, 8))
    t = torch.from_numpy(np.frombuffer(bytes(buf), np.uint8).copy()).cuda()
    out = ec.rle_decompress(t, 64, 64)
    st = ec.default_context().status_sync()
    assert st in (0, 4)
    assert st == oracle.rle_decompress_status(bytes(buf), 64, 64)
    if st == 0:
        assert np.array_equal(np_of(out), oracle.rle_decompress(bytes(buf), 64, 64))


@pytest.mark.slow
def test_8k_frame_and_size_limit():
    require_gpu()
    s = S.depth_source(7680, 4320, 0.25, 5, 0, device="cuda")
    for t, mode in ((s.color, 2), (s.depth.view(torch.uint32), 1)):
        buf, size = ec.rle_compress(t, mode)
        ec.default_context().check_status()
        ref = oracle.rle_compress(np_of(t), mode)
        assert _gpu_bytes(buf, size) == ref
        out = ec.rle_decompress(buf, 7680, 4320, src_size=len(ref))
        ec.default_context().check_status()
        assert torch.equal(out.view(torch.int32), t.view(torch.int32))
    big = torch.zeros((1, ec.EC_RLE_CHUNK * (1 << 15) + 1), dtype=torch.int32, device="cuda").view(torch.uint32)
    with pytest.raises(ec.EcError) as e:
        ec.rle_compress(big, 1)
    assert e.value.code == 5


def test_bounded_wait_times_out_and_context_survives():
    """Failure detection without a fault: the compressor's bounded mbarrier wait
    runs on a barrier that nothing arrives on, gives up after its try limit and
    records EC_ERR_TIMEOUT; the kernel ends and the context keeps working."""
    import time
    from paper_1902_08755_gb300 import _abi as A
    require_gpu()
    ctx = ec.default_context()
    ctx.status_sync()
    t0 = time.perf_counter()
    A.check(A.load().ec_selftest_wait_timeout(ctx.h, torch.cuda.current_stream().cuda_stream), "selftest")
    assert ctx.status_sync() == A.EC_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    img = S.depth_source(200, 90, 0.4, 42, 0).color.numpy()
    _roundtrip_check(img, 2)                 # the context still codes correctly
    assert ctx.status_sync() == 0
