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
