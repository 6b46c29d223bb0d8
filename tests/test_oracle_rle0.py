"""Pins for the oracle's basic 64-bit RLE (mode 0; thesis 5.5.1: tokens that
compare two RGBA8 pixels at once, the starting point the per-component RLE
improves on).

Independent of the encoder: hand-derived worked examples (tests/golden, the
mode-0 container lines), a token decoder and a size formula written here from
the rules (run decomposition of the 8-byte units with itertools.groupby), the
all-literal capacity met with equality by incompressible data, the quantity
the thesis reports (mode 0 compresses worse than per-component RLE on images
whose pixels rarely repeat in pairs), and rejection of corrupt streams.
"""
import itertools

import numpy as np
import pytest

import synthetic as S

HDR = 32


def _units(chunk):
    """8-byte units of a chunk of elements (element 2k in the low half) and its odd tail."""
    n = len(chunk) // 2
    return [(int(chunk[2 * k]), int(chunk[2 * k + 1])) for k in range(n)], (
        int(chunk[-1]) if len(chunk) % 2 else None)


def _expected_size(chunk):
    """A run of L >= 2 equal units costs 9 * ceil(L / 128); a maximal span of m
    single units costs 8m + ceil(m / 128); an odd tail 4 bytes."""
    units, tail = _units(chunk)
    size, span = 0, 0
    for _, grp in itertools.groupby(units):
        L = len(list(grp))
        if L >= 2:
            size += 8 * span + -(-span // 128)
            span = 0
            size += 9 * -(-L // 128)
        else:
            span += 1
    size += 8 * span + -(-span // 128)
    return size + (4 if tail is not None else 0)


def _decode(stream, n_elems):
    """Decoding rule: control c < 128 copies c+1 units, c >= 128 repeats the next
    unit c-127 times; an odd chunk ends with one raw element."""
    out, i = [], 0
    while len(out) < n_elems // 2 * 2:
        c = stream[i]
        if c < 128:
            for k in range(c + 1):
                b = stream[i + 1 + 8 * k:i + 9 + 8 * k]
                out += [int.from_bytes(b[:4], "little"), int.from_bytes(b[4:], "little")]
            i += 1 + 8 * (c + 1)
        else:
            b = stream[i + 1:i + 9]
            out += [int.from_bytes(b[:4], "little"), int.from_bytes(b[4:], "little")] * (c - 127)
            i += 9
    if n_elems % 2:
        out.append(int.from_bytes(stream[i:i + 4], "little"))
        i += 4
    assert i == len(stream)
    return out


def _streams(buf):
    nc = int.from_bytes(buf[24:28], "little")
    assert int.from_bytes(buf[28:32], "little") == 1          # one plane
    ends = np.frombuffer(buf[HDR:HDR + 4 * nc], dtype="<u4")
    pay = buf[HDR + 4 * nc:]
    begins = np.concatenate([[0], ends[:-1]]) if nc else []
    return [pay[b:e] for b, e in zip(begins, ends)]


def _images():
    r = np.random.default_rng(5)
    imgs = {
        "all_equal": np.full((9, 301), 0xDEADBEEF, np.uint32),
        "pairs_of_pixels": np.repeat(np.arange(700, dtype=np.uint32), 4).reshape(7, 400),
        "alternating": np.tile(np.array([1, 2], np.uint32), (5, 333)),
        "noise": r.integers(0, 2**32, size=(33, 257), dtype=np.uint64).astype(np.uint32),
        "straddle_odd": np.zeros((1, 4097), np.uint32),
        "boxes": S.depth_source(200, 90, 0.4, 42, 0).color.numpy(),
        "depth_bits": S.depth_source(200, 90, 0.4, 42, 0).depth.numpy().view(np.uint32),
    }
    runs = []
    for L in (1, 2, 3, 4, 5, 127, 128, 129, 256, 257, 258, 259, 4095, 4097):
        runs += [L | 0x77000000] * L
    imgs["unit_run_lengths"] = np.array(runs[:len(runs) // 3 * 3], np.uint32).reshape(3, -1)
    # runs of units that are shifted by one element (pairs never align)
    imgs["shifted_pairs"] = np.repeat(np.arange(902, dtype=np.uint32), 2)[1:1802].reshape(1, 1801)
    return imgs


@pytest.mark.parametrize("name", sorted(_images().keys()))
def test_streams_decode_and_have_canonical_size(orc, name):
    img = _images()[name]
    h, w = img.shape
    buf = orc.rle_compress(img, 0)
    assert len(buf) <= orc.rle_max_size(w, h)
    flat = img.reshape(-1)
    nc = -(-flat.size // 4096)
    streams = _streams(buf)
    assert len(streams) == nc
    for c, s in enumerate(streams):
        chunk = flat[4096 * c:4096 * (c + 1)]
        assert _decode(s, len(chunk)) == [int(v) for v in chunk]
        assert len(s) == _expected_size(chunk)
    assert np.array_equal(orc.rle_decompress(buf, w, h), img)


@pytest.mark.parametrize("shape", [(0, 0), (1, 1), (1, 2), (1, 3), (1, 4095), (1, 4097), (65, 127), (3, 5001)])
def test_round_trip_shapes_and_pitch(orc, shape):
    h, w = shape
    r = np.random.default_rng(h * 31 + w)
    pitch = w + 5
    img = r.integers(0, 2, size=(h, pitch)).astype(np.uint32)
    buf = orc.rle_compress(img, 0, w=w)
    out = orc.rle_decompress(buf, w, h, pitch=pitch)
    assert np.array_equal(out[:, :w], img[:, :w])


def test_incompressible_meets_its_bound(orc):
    """Units that never repeat code as full literal tokens: 8u + ceil(u/128) bytes
    per chunk of u units, plus 4 for an odd tail."""
    for w, h in ((4096, 1), (4097, 1), (301, 13)):
        img = np.arange(w * h, dtype=np.uint32).reshape(h, w)
        n, size = w * h, HDR + 4 * -(-(w * h) // 4096)
        for c in range(-(-n // 4096)):
            L = min(4096, n - 4096 * c)
            u = L // 2
            size += 8 * u + -(-u // 128) + 4 * (L % 2)
        assert len(orc.rle_compress(img, 0)) == size


def test_per_component_coding_beats_pixel_pairs(orc):
    """Thesis 5.5.1: comparing whole pixel pairs finds few runs, the
    per-component streams (with or without the swizzle) find many more."""
    for img in (S.smooth_image(256, 128), S.depth_source(400, 300, 0.4, 42, 0).color.numpy()):
        m0, m1, m2 = (len(orc.rle_compress(img, m)) for m in (0, 1, 2))
        assert max(m1, m2) < m0 < 4 * img.size


def test_decoder_rejects_corrupt_streams(orc):
    img = S.depth_source(100, 70, 0.4, 43, 0).color.numpy()
    buf = orc.rle_compress(img, 0)
    assert orc.rle_decompress_status(buf, 100, 70) == 0
    nc = int.from_bytes(buf[24:28], "little")
    b = bytearray(buf)
    x = bytearray(b); x[28] = 4; assert orc.rle_decompress_status(bytes(x), 100, 70) == orc.ECORRUPT
    x = bytearray(b); x[6] = 3; assert orc.rle_decompress_status(bytes(x), 100, 70) == orc.ECORRUPT
    assert orc.rle_decompress_status(bytes(b[:-1]), 100, 70) == orc.ECORRUPT
    x = bytearray(b); x[HDR:HDR + 4] = (0).to_bytes(4, "little")
    assert orc.rle_decompress_status(bytes(x), 100, 70) == orc.ECORRUPT
    # a chunk whose stream yields one unit too few, and one whose odd tail is missing
    two = orc.rle_compress(np.full((1, 4), 7, np.uint32), 0)      # "81 unit"
    y = bytearray(two); y[HDR + 4] = 0x80
    assert orc.rle_decompress_status(bytes(y), 4, 1) == orc.ECORRUPT
    three = orc.rle_compress(np.array([[1, 2, 3]], np.uint32), 0)  # "00 unit" + tail
    assert orc.rle_decompress_status(three[:-4], 3, 1) == orc.ECORRUPT
    # the all-literal bound: a stream longer than 8u + ceil(u/128) + tail is refused
    lits = bytes([0x00]) + (7).to_bytes(4, "little") * 2 + bytes([0x00]) + (7).to_bytes(4, "little") * 2
    hdr = bytes(two[:HDR])
    assert orc.rle_decompress_status(hdr + (len(lits)).to_bytes(4, "little") + lits, 4, 1) == orc.ECORRUPT
    assert nc >= 1
