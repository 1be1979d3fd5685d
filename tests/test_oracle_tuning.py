"""Pins of the paper's tuning-model oracle (Sec. 4.1), hand-worked values."""
from oracle import tuning
from tests.conftest import read_golden


def test_hand_worked_model():
    for head, expect, _why in read_golden("tuning_model.txt"):
        arch, r = head.split()
        ssrs, srs = (int(v) for v in expect.split())
        assert tuning.model_sizes(float(r), arch) == (ssrs, srs), head


def test_search_grid():
    assert tuning.search_grid() == [4, 6, 8, 12, 16, 24, 32, 48]


def test_cases():
    assert [tuning.case_of(r) for r in (1, 8, 8.01, 16, 16.5, 32, 33)] == [1, 1, 2, 2, 3, 3, 4]
