"""Pins for the RLE oracle (thesis 5.5.1: per-component streams, the bit-swizzle
preconditioner, data decomposition into independently coded sub-images).

The container and token rules are this project's reading of 5.5.1 (the figures
that showed the thesis's layout are not in the text).  Pins that do not use the
encoder itself: hand-derived worked examples (tests/golden), an independent
token decoder, an independent size formula from the run decomposition
(itertools.groupby), the swizzle's bit-permutation structure, and the capacity
bound met with equality by incompressible data.
"""
import itertools
import os

import numpy as np
import pytest

import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "rle_worked_examples.txt")
HDR = 32


def _golden():
    cases = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            kind, lhs, rhs = [s.strip() for s in line.split("|")]
            cases.append((kind, lhs, rhs))
    return cases


def _parse_run_list(spec):
    """'5*4,1,2' -> [5,5,5,5,1,2]"""
    out = []
    if spec == "-":
        return out
    for tok in spec.split(","):
        if "*" in tok:
            v, k = tok.split("*")
            out += [int(v, 0)] * int(k)
        else:
            out.append(int(tok, 0))
    return out


def _streams(buf):
    nc = int.from_bytes(buf[24:28], "little")
    ends = np.frombuffer(buf[HDR:HDR + 16 * nc], dtype="<u4")
    pay = buf[HDR + 16 * nc:]
    begins = np.concatenate([[0], ends[:-1]]) if nc else []
    return [pay[b:e] for b, e in zip(begins, ends)]


def _decode_tokens(s):
    """Decoding rule: control c < 128 copies the next c+1 bytes, c >= 128 repeats
    the next byte c-127 times."""
    out, i = bytearray(), 0
    while i < len(s):
        c = s[i]
        if c < 128:
            out += s[i + 1:i + 2 + c]
            i += 2 + c
        else:
            out += bytes([s[i + 1]]) * (c - 127)
            i += 2
    return bytes(out)


def _expected_stream_size(b):
    """Size from the run decomposition: a run of L >= 3 costs 2*ceil(L/128); each
    maximal span of shorter runs, m bytes, costs m + ceil(m/128)."""
    size, span = 0, 0
    for _, grp in itertools.groupby(b):
        L = len(list(grp))
        if L >= 3:
            size += span + -(-span // 128)
            span = 0
            size += 2 * -(-L // 128)
        else:
            span += L
    return size + span + -(-span // 128)


def _planes(img, mode, orc):
    flat = img.reshape(-1)
    if mode == 2:
        flat = np.array([orc.swizzle(int(v)) for v in flat], dtype=np.uint32)
    return [((flat >> (8 * p)) & 0xFF).astype(np.uint8) for p in range(4)]


@pytest.mark.parametrize("case", range(len(_golden())))
def test_golden_worked_examples(orc, case):
    kind, lhs, rhs = _golden()[case]
    if kind == "stream":
        # a plane-0 byte stream: elements carry it in their low byte, other bytes 0
        vals = _parse_run_list(lhs)
        buf = orc.rle_compress(np.array([vals], dtype=np.uint32), 1)
        assert _streams(buf)[0].hex() == rhs.replace(" ", "")
    elif kind == "container":
        w, h, mode, vals = lhs.split(";")
        img = np.array(_parse_run_list(vals), dtype=np.uint32).reshape(int(h), int(w))
        assert orc.rle_compress(img, int(mode)).hex() == rhs.replace(" ", "")
    elif kind == "swizzle":
        assert orc.swizzle(int(lhs, 16)) == int(rhs, 16)
        assert orc.unswizzle(int(rhs, 16)) == int(lhs, 16)
    else:
        raise AssertionError(kind)


def test_swizzle_is_a_bit_permutation(orc):
    """Every single input bit lands on a distinct single output bit (so the map,
    built from shifts, masks and ORs, is a bijection of the 32-bit words), and
    the most significant pair of each component lands in byte 0."""
    imgs = [orc.swizzle(1 << b) for b in range(32)]
    assert all(bin(v).count("1") == 1 for v in imgs)
    assert len(set(imgs)) == 32
    for comp in range(4):
        assert orc.swizzle(0xC0 << (8 * comp)) == 3 << (6 - 2 * comp)
    r = np.random.default_rng(0)
    for v in r.integers(0, 2**32, size=2000, dtype=np.uint64):
        s = orc.swizzle(int(v))
        assert orc.unswizzle(s) == int(v)
        assert bin(s).count("1") == bin(int(v)).count("1")


def _adversarial_images():
    imgs = {}
    imgs["all_equal"] = np.full((17, 300), 0xDEADBEEF, np.uint32)
    imgs["alternating"] = np.tile(np.array([0x01020304, 0x05060708], np.uint32), (9, 250))
    imgs["pairs"] = np.repeat(np.arange(1500, dtype=np.uint32) * 0x01010101, 2).reshape(10, 300)
    runs = []
    for L in (1, 2, 3, 127, 128, 129, 130, 255, 256, 257, 4095, 4096, 4097):
        runs += [L & 0xFF | 0x5500] * L
    imgs["run_lengths"] = np.array(runs[:len(runs) // 7 * 7], np.uint32).reshape(7, -1)
    # a run straddling the 4096-element chunk boundary, and a tail chunk of 1
    x = np.zeros(4097, np.uint32)
    x[4000:4200 if 4200 <= 4097 else 4097] = 9
    imgs["straddle"] = x.reshape(1, -1)
    r = np.random.default_rng(1)
    imgs["noise"] = r.integers(0, 2**32, size=(33, 257), dtype=np.uint64).astype(np.uint32)
    imgs["lit_run_mix"] = np.array(
        sum(([int(v)] * int(k) for v, k in zip(r.integers(0, 4, 3000), r.integers(1, 6, 3000))), []),
        np.uint32)[:8192].reshape(64, 128)
    # runs of exactly 3 alternating values: ~1365 repeat runs per plane and chunk
    imgs["runs_of_3"] = np.repeat(np.arange(2800, dtype=np.uint32) % 2 * np.uint32(0x01010101) + 7,
                                  3).reshape(6, 1400)
    imgs["boxes"] = S.depth_source(200, 90, 0.4, 42, 0).color.numpy()
    imgs["depth_bits"] = S.depth_source(200, 90, 0.4, 42, 0).depth.numpy().view(np.uint32)
    imgs["smooth"] = S.smooth_image(160, 120)
    return imgs


@pytest.mark.parametrize("name", sorted(_adversarial_images().keys()))
@pytest.mark.parametrize("mode", [1, 2])
def test_streams_decode_and_have_canonical_size(orc, name, mode):
    img = _adversarial_images()[name]
    h, w = img.shape
    buf = orc.rle_compress(img, mode)
    assert len(buf) <= orc.rle_max_size(w, h)
    streams = _streams(buf)
    planes = _planes(img, mode, orc)
    n = w * h
    nc = -(-n // 4096)
    assert len(streams) == 4 * nc
    for c in range(nc):
        for p in range(4):
            ref = planes[p][4096 * c:4096 * (c + 1)].tobytes()
            s = streams[4 * c + p]
            assert _decode_tokens(s) == ref
            assert len(s) == _expected_stream_size(ref)
    assert np.array_equal(orc.rle_decompress(buf, w, h), img)


@pytest.mark.parametrize("shape", [(0, 0), (0, 5), (3, 0), (1, 1), (1, 4095), (1, 4096),
                                   (1, 4097), (64, 64), (65, 127), (3, 5000)])
def test_round_trip_shapes_and_pitch(orc, shape):
    h, w = shape
    r = np.random.default_rng(h * 7919 + w)
    pitch = w + 3
    img = (r.integers(0, 3, size=(h, pitch)) * 0x01010101).astype(np.uint32)
    for mode in (1, 2):
        buf = orc.rle_compress(img, mode, w=w)
        if w * h == 0:
            assert len(buf) == HDR
        out = orc.rle_decompress(buf, w, h, pitch=pitch)
        assert np.array_equal(out[:, :w], img[:, :w])


def test_incompressible_meets_capacity_bound(orc):
    """Alternating bytes never form runs: every stream is all literals and the
    size equals the capacity formula exactly."""
    for w, h in ((4096, 1), (100, 50), (4097, 3)):
        img = np.tile(np.array([0x00000000, 0x01010101], np.uint32), (h, (w + 1) // 2))[:, :w].copy()
        assert len(orc.rle_compress(img, 1)) == orc.rle_max_size(w, h)


@pytest.mark.parametrize("seed", range(40))
def test_random_streams_bound_and_round_trip(orc, seed):
    r = np.random.default_rng(500 + seed)
    w, h = int(r.integers(1, 300)), int(r.integers(1, 40))
    vals = r.integers(0, 1 + seed % 4, size=(h, w)).astype(np.uint32) * np.uint32(0x01010101)
    vals ^= (r.random((h, w)) < 0.05).astype(np.uint32) * np.uint32(r.integers(0, 2**32))
    for mode in (1, 2):
        buf = orc.rle_compress(np.ascontiguousarray(vals), mode)
        assert len(buf) <= orc.rle_max_size(w, h)
        assert np.array_equal(orc.rle_decompress(buf, w, h), vals)


def test_brute_force_4x4_all_modes(orc):
    """4x4 images over a 2-value alphabet per byte, 300 random draws."""
    r = np.random.default_rng(9)
    for _ in range(300):
        img = (r.integers(0, 2, size=(4, 4, 4)) * r.integers(1, 255)).astype(np.uint32)
        v = (img[..., 0] | img[..., 1] << 8 | img[..., 2] << 16 | img[..., 3] << 24).astype(np.uint32)
        for mode in (1, 2):
            buf = orc.rle_compress(v, mode)
            assert np.array_equal(orc.rle_decompress(buf, 4, 4), v)


def test_swizzle_helps_smooth_colour(orc):
    """Thesis 5.5.1: per-component RLE beats raw pixels on smooth colour, and
    swizzling improves it further (10% -> 25% -> 40% in the thesis's scenario)."""
    img = S.smooth_image(512, 384)
    raw = img.nbytes
    m1 = len(orc.rle_compress(img, 1))
    m2 = len(orc.rle_compress(img, 2))
    assert m2 < m1 < raw


def _corruptions(buf):
    b = bytearray(buf)
    yield "truncated_header", bytes(b[:20])
    yield "truncated_payload", bytes(b[:-1])
    x = bytearray(b); x[0] ^= 1; yield "magic", bytes(x)
    x = bytearray(b); x[4] = 2; yield "version", bytes(x)
    x = bytearray(b); x[6] = 7; yield "mode", bytes(x)
    x = bytearray(b); x[16] = 8; yield "elem_bytes", bytes(x)
    x = bytearray(b); x[20] ^= 1; yield "chunk_px", bytes(x)
    x = bytearray(b); x[24] ^= 1; yield "n_chunks", bytes(x)
    x = bytearray(b); x[HDR:HDR + 4] = (0xFFFFFF).to_bytes(4, "little"); yield "end_past", bytes(x)
    x = bytearray(b); x[HDR + 4:HDR + 8] = (0).to_bytes(4, "little"); yield "end_nonmonotone", bytes(x)


def test_decoder_rejects_corrupt_streams(orc):
    img = S.depth_source(100, 70, 0.4, 43, 0).color.numpy()
    buf = orc.rle_compress(img, 2)
    assert orc.rle_decompress_status(buf, 100, 70) == 0
    for name, bad in _corruptions(buf):
        assert orc.rle_decompress_status(bad, 100, 70) == orc.ECORRUPT, name
    assert orc.rle_decompress_status(buf, 99, 70) == orc.ECORRUPT
    # every token parses but stream 0 yields 3 of its 4 bytes ("83 01" -> "82 01")
    four = orc.rle_compress(np.full((1, 4), 0x01010101, np.uint32), 1)
    assert four[HDR + 16:HDR + 18] == bytes([0x83, 0x01])
    short = bytearray(four)
    short[HDR + 16] = 0x82
    assert orc.rle_decompress_status(bytes(short), 4, 1) == orc.ECORRUPT
    # ... and a stream that runs one byte long ("83 01" -> "84 01")
    short[HDR + 16] = 0x84
    assert orc.rle_decompress_status(bytes(short), 4, 1) == orc.ECORRUPT
    # a non-canonical but parseable stream is accepted within the length bound
    # (4 one-byte literals "00 01" x4 = 8 bytes > 4 + 1), and rejected above it
    lits = bytes([0x00, 0x01] * 4)
    streams = [lits, bytes([0x83, 0x01]), bytes([0x83, 0x01]), bytes([0x83, 0x01])]
    ends, off = [], 0
    for st in streams:
        off += len(st)
        ends.append(off)
    hdr = bytes(four[:HDR])
    table = b"".join(e.to_bytes(4, "little") for e in ends)
    assert orc.rle_decompress_status(hdr + table + b"".join(streams), 4, 1) == orc.ECORRUPT
    streams[0] = bytes([0x00, 0x01, 0x82, 0x01])       # 4 bytes <= bound: accepted
    ends, off = [], 0
    for st in streams:
        off += len(st)
        ends.append(off)
    table = b"".join(e.to_bytes(4, "little") for e in ends)
    assert orc.rle_decompress_status(hdr + table + b"".join(streams), 4, 1) == 0


@pytest.mark.parametrize("seed", range(20))
def test_decoder_never_accepts_a_wrong_image(orc, seed):
    """Random byte flips in the payload either fail validation or decode to some
    image of the right size -- never crash; a flipped control byte that still
    parses must change the decoded plane lengths consistently."""
    r = np.random.default_rng(seed)
    img = S.depth_source(64, 64, 0.4, 44, seed % 3).color.numpy()
    buf = bytearray(orc.rle_compress(img, 1))
    nc = int.from_bytes(buf[24:28], "little")
    lo = HDR + 16 * nc
    for _ in range(5):
        i = int(r.integers(lo, len(buf)))
        buf[i] ^= 1 << int(r.integers(0, 8))
    rc = orc.rle_decompress_status(bytes(buf), 64, 64)
    assert rc in (0, orc.ECORRUPT)
