"""Host logic of the request loop: FIFO admission by device-memory budget (no GPU)."""
import numpy as np
import pytest

from paper_2205_11226_gb300.serving import Admission, Request


def req(i, kb):
    f = np.zeros((16, kb * 32), np.uint8)  # 2 * 512*kb bytes + mask
    return Request(i, float(i), f, np.zeros((1, 2 * kb), np.uint8))


def test_fifo_admission_within_budget():
    a = Admission(budget_bytes=3 * 1024 + 100)
    for i in range(5):
        a.arrive(req(i, 1))
    first = a.admit()
    assert [r.rid for r in first] == [0, 1, 2]
    assert a.admit() == []                      # budget full
    a.release(first[:1])
    assert [r.rid for r in a.admit()] == [3]    # oldest waiting first
    a.release(first[1:])
    assert [r.rid for r in a.admit(limit=1)] == [4]
    assert a.in_flight > 0 and not a.waiting


def test_oversized_request_rejected():
    a = Admission(budget_bytes=100)
    a.arrive(req(0, 1))
    with pytest.raises(ValueError):
        a.admit()


def test_resident_concurrency_of_launch_intervals():
    from paper_2205_11226_gb300.serving import resident_concurrency
    # [0, 10] and [5, 15]: busy 15, two resident for 5 -> mean (5 + 2*5 + 5) / 15
    r = resident_concurrency([(0, 10), (5, 15)])
    assert r["max_resident_launches"] == 2
    assert abs(r["mean_resident_launches"] - 20 / 15) < 1e-12
    # disjoint intervals never overlap; the gap is not busy time
    r = resident_concurrency([(0, 10), (20, 30)])
    assert r["max_resident_launches"] == 1 and r["mean_resident_launches"] == 1.0
    assert abs(r["device_busy_s"] - 20e-9) < 1e-18
