"""Host logic of the serving loop's admission (no GPU): streams are admitted in arrival
order while a slot is free and their HBM need fits the budget left by active streams; a
departing stream frees its bytes and slot for the streams waiting behind it."""
import numpy as np
import pytest

from paper_1605_02406_b300.serve import Admission


def test_admission_waits_in_order_and_refills_on_departure():
    a = Admission(10.0, 3)
    for k, need in enumerate([4.0, 4.0, 4.0, 1.0]):
        a.request(k, need)
    assert a.admit() == [0, 1]          # stream 2 does not fit; stream 3 may not overtake it
    assert a.admit() == []
    a.release(0)
    assert a.admit() == [2, 3]          # 4 + 4 + 1 = 9 of 10, three slots
    a.request(4, 1.0)
    assert a.admit() == []              # slots full although the bytes would fit
    a.release(3)
    assert a.admit() == [4]
    assert a.used == pytest.approx(9.0)


def test_admission_rejects_a_stream_larger_than_the_budget():
    a = Admission(10.0, 4)
    with pytest.raises(ValueError):
        a.request(0, 10.5)


def test_admission_random_sequence_keeps_budget_slots_and_order():
    rng = np.random.default_rng(5)
    budget, slots = 100.0, 6
    a = Admission(budget, slots)
    order, nxt = [], 0
    for step in range(2000):
        if rng.random() < 0.5:
            a.request(nxt, float(rng.uniform(1, 60)))
            nxt += 1
        elif a.active:
            a.release(int(rng.choice(list(a.active))))
        order += a.admit()
        assert a.used <= budget + 1e-9 and len(a.active) <= slots
        assert a.used == pytest.approx(sum(a.active.values()))
    assert order == sorted(order) and order == list(range(len(order)))
