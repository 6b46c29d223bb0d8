"""CPU check of the library's schedule planner (thesis 5.2.2, 5.2.3) against
the oracle's, on geometry alone: for random frames, resource counts and ROIs
(empty, partly outside the frame, covering it), ec_schedule_geometry yields
the same stages, the same transfers (sender, receiver, level and rectangle)
and the same final regions as the oracle's planner.  No device work."""
import numpy as np
import pytest

import paper_1902_08755_gb300 as ec
from paper_1902_08755_gb300 import _abi as A
from oracle import schedules as OS

ALGOS = {OS.CHAIN: "stream", OS.DIRECT_SEND: "direct_send", OS.BINARY_SWAP: "binary_swap",
         OS.TWO_THREE_SWAP: "two_three_swap"}


def _rois(r, n, frame):
    fx, fy, fw, fh = frame
    out = []
    for i in range(n):
        k = r.integers(0, 6)
        if k == 0:
            out.append((0, 0, 0, 0))
        elif k == 1:
            out.append(frame)
        elif k == 2:        # reaching outside the frame
            out.append((fx - int(r.integers(0, 40)), fy - int(r.integers(0, 40)),
                        fw + int(r.integers(0, 80)), fh + int(r.integers(0, 80))))
        else:
            x0, x1 = sorted(r.integers(fx, fx + max(fw, 1) + 1, size=2))
            y0, y1 = sorted(r.integers(fy, fy + max(fh, 1) + 1, size=2))
            out.append((int(x0), int(y0), int(x1 - x0), int(y1 - y0)))
    return out


def _cases():
    r = np.random.default_rng(20190208)
    cases = []
    for algo in ALGOS:
        for t in range(60):
            n = int(r.choice([1, 2, 4, 8, 16, 32])) if algo == OS.BINARY_SWAP else int(r.integers(1, 34))
            frame = (int(r.integers(-50, 50)), int(r.integers(-50, 50)),
                     int(r.choice([1, 2, 3, 7, 64, 333, 1920])), int(r.choice([1, 2, 5, 31, 100, 1080])))
            cases.append((algo, n, frame, _rois(r, n, frame)))
    return cases


def _oracle(algo, rois, frame):
    pl = OS.plan(algo, frame, rois)
    msgs = [(li, m.sender, m.receiver, m.piece) for li, lv in enumerate(pl.levels) for m in lv.messages]
    return msgs, len(pl.levels), [tuple(R) if not OS.is_empty(R) else None for R in pl.region]


def _norm(regions):
    return [tuple(R) if R[2] > 0 and R[3] > 0 else None for R in regions]


def test_planner_matches_oracle_on_random_geometry():
    for algo, n, frame, rois in _cases():
        msgs, nl, regions = ec.schedule_geometry(ALGOS[algo], rois, frame)
        omsgs, onl, oregions = _oracle(algo, rois, frame)
        ctx = (ALGOS[algo], n, frame, rois)
        assert nl == onl, ctx
        assert sorted(msgs) == sorted(omsgs), ctx
        assert _norm(regions) == oregions, ctx
        # within a stage the transfers come in compositing order
        for li in range(nl):
            for recv in range(n):
                got = [m[1:] for m in msgs if m[0] == li and m[2] == recv]
                want = [m[1:] for m in omsgs if m[0] == li and m[2] == recv]
                assert got == want, ctx


@pytest.mark.parametrize("n", [3, 5, 6, 12])
def test_binary_swap_refuses_non_power_of_two(n):
    with pytest.raises(ValueError):
        OS.plan(OS.BINARY_SWAP, (0, 0, 64, 64), [(0, 0, 64, 64)] * n)
    with pytest.raises(A.EcError):
        ec.schedule_geometry("binary_swap", [(0, 0, 64, 64)] * n, (0, 0, 64, 64))


def test_capacity_is_reported():
    lib = A.load()
    rois = (A.ec_rect * 4)(*[A.ec_rect(0, 0, 64, 64)] * 4)
    nm, nl = A.C.c_int32(), A.C.c_int32()
    msgs = (A.ec_sched_message * 2)()
    code = lib.ec_schedule_geometry(A.EC_SCHED_DIRECT_SEND, rois, 4, A.ec_rect(0, 0, 64, 64), msgs, 2,
                                    A.C.byref(nm), A.C.byref(nl), None)
    assert code == A.EC_ERR_CAPACITY and nm.value == 12 and nl.value == 1
    code = lib.ec_schedule_geometry(A.EC_SCHED_DIRECT_SEND, rois, 0, A.ec_rect(0, 0, 64, 64), msgs, 2,
                                    A.C.byref(nm), A.C.byref(nl), None)
    assert code == A.EC_ERR_INVALID_ARG


def test_argument_errors():
    lib = A.load()
    nm, nl = A.C.c_int32(), A.C.c_int32()
    frame = A.ec_rect(0, 0, 8, 8)
    four = (A.ec_rect * 4)(*[A.ec_rect(0, 0, 8, 8)] * 4)
    call = lambda alg, arr, n: lib.ec_schedule_geometry(alg, arr, n, frame, None, 0, A.C.byref(nm),
                                                        A.C.byref(nl), None)
    assert call(7, four, 4) == A.EC_ERR_INVALID_ARG                  # unknown algorithm
    assert call(A.EC_SCHED_BINARY_SWAP, four, 3) == A.EC_ERR_INVALID_ARG
    neg = (A.ec_rect * 1)(A.ec_rect(0, 0, -1, 8))
    assert call(A.EC_SCHED_DIRECT_SEND, neg, 1) == A.EC_ERR_INVALID_ARG
    many = (A.ec_rect * 600)(*[A.ec_rect(0, 0, 8, 8)] * 600)
    assert call(A.EC_SCHED_DIRECT_SEND, many, 600) == 5                 # EC_ERR_UNSUPPORTED
    assert call(A.EC_SCHED_STREAM, four, 4) == A.EC_ERR_CAPACITY and nm.value == 3 and nl.value == 3
