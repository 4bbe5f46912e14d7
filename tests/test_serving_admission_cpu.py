"""The serving runtime's admission policy, run on the CPU through the library's test hook (the
same decision function the worker thread uses). A flight visits the queued requests in arrival
order and takes the next chunk of each (a large request is cut into chunks) while its device
footprint fits the budget next to what is already running and the flight's work stays under its
cap; a chunk that does not fit stops the flight (no overtaking), one that could never fit fails
with OOM, FP64 and kNN-output requests run alone, a flight holds at most max_items chunks and
always takes its first chunk whatever its work."""
import numpy as np
import pytest

from paper_1511_02186_gb300 import aidw, build

TAKE, SOLO, OOM, WAIT = 0, 1, 2, 3


@pytest.fixture(scope="module")
def lib():
    build.build()
    return aidw.load()


def admit(lib, footprints, budget, in_flight=0, max_items=256, solo=(), pairs=None,
          max_pairs=0.0):
    n = len(footprints)
    s = np.zeros(n, dtype=np.int32)
    for i in solo:
        s[i] = 1
    f = np.asarray(footprints, dtype=np.uint64)
    pr = None if pairs is None else np.asarray(pairs, dtype=np.float64)
    out = np.full(n, -1, dtype=np.int32)
    rc = lib.aidw_debug_admission(n, s.ctypes.data, f.ctypes.data, budget, in_flight, max_items,
                                  None if pr is None else pr.ctypes.data, float(max_pairs),
                                  out.ctypes.data)
    assert rc == aidw.OK
    return out.tolist()


def test_requests_join_while_they_fit(lib):
    assert admit(lib, [1, 2, 3], 10) == [TAKE, TAKE, TAKE]
    assert admit(lib, [4, 4, 4], 10) == [TAKE, TAKE, WAIT]
    assert admit(lib, [4, 6, 1], 10) == [TAKE, TAKE, WAIT]  # exactly full, then the next waits
    assert admit(lib, [4, 4], 10, in_flight=5) == [TAKE, WAIT]


def test_arrival_order_is_kept(lib):
    # A request that does not fit holds back the smaller ones behind it.
    assert admit(lib, [8, 1, 1], 10, in_flight=5) == [WAIT, WAIT, WAIT]
    assert admit(lib, [3, 8, 1], 10) == [TAKE, WAIT, WAIT]


def test_oversized_requests_fail_and_the_queue_moves_on(lib):
    assert admit(lib, [20, 1], 10) == [OOM, TAKE]
    assert admit(lib, [1, 11, 2], 10, in_flight=9) == [TAKE, OOM, WAIT]


def test_solo_requests_run_alone(lib):
    assert admit(lib, [5, 1, 2], 10, solo=[0]) == [SOLO, TAKE, TAKE]
    assert admit(lib, [1, 5, 2], 10, solo=[1]) == [TAKE, WAIT, WAIT]
    assert admit(lib, [5, 5, 1], 10, solo=[0, 1]) == [SOLO, SOLO, TAKE]


def test_flight_size_limit(lib):
    assert admit(lib, [1] * 5, 100, max_items=3) == [TAKE, TAKE, TAKE, WAIT, WAIT]


def test_flight_work_cap(lib):
    # Chunks join while the flight's pair-evaluations stay within the cap ...
    assert admit(lib, [1, 1, 1, 1], 100, pairs=[4, 3, 3, 1], max_pairs=10) == [TAKE] * 3 + [WAIT]
    # ... a flight always takes its first chunk, however large ...
    assert admit(lib, [1, 1], 100, pairs=[50, 1], max_pairs=10) == [TAKE, WAIT]
    # ... no cap without one, and the cap does not let a later chunk overtake.
    assert admit(lib, [1, 1, 1], 100, pairs=[9, 9, 9]) == [TAKE, TAKE, TAKE]
    assert admit(lib, [1, 1, 1], 100, pairs=[5, 6, 1], max_pairs=10) == [TAKE, WAIT, WAIT]


def test_bad_arguments(lib):
    assert lib.aidw_debug_admission(-1, None, None, 1, 0, 4, None, 0.0,
                                    None) == aidw.ERR_INVALID_ARG
    assert lib.aidw_debug_admission(2, None, None, 1, 0, 4, None, 0.0,
                                    None) == aidw.ERR_INVALID_ARG
    z = np.zeros(1, dtype=np.int32)
    f = np.zeros(1, dtype=np.uint64)
    assert lib.aidw_debug_admission(1, z.ctypes.data, f.ctypes.data, 1, 0, 0, None, 0.0,
                                    z.ctypes.data) == aidw.ERR_INVALID_ARG
    assert lib.aidw_debug_admission(0, None, None, 1, 0, 4, None, 0.0, None) == aidw.OK
