"""Pins of the super-row pointer oracle (Sec. 2.2, Fig. 1)."""
import numpy as np

from oracle import csrk
from tests.conftest import read_golden


def _ints(s):
    return [int(v) for v in s.split(",")]


def test_hand_worked_pointers():
    for head, srp, ssrp in read_golden("csrk_pointers.txt"):
        if head.startswith("fig1"):
            n = int(head.split()[1])
            assert csrk.validate_pointers(n, _ints(srp), _ints(ssrp)) == []
            continue
        n, sr, ssr = (int(v) for v in head.split())
        a, b = csrk.fixed_pointers(n, sr, ssr)
        assert a.tolist() == _ints(srp), head
        assert b.tolist() == _ints(ssrp), head
        assert csrk.validate_pointers(n, a, b) == []


def test_validator_rejects():
    assert csrk.validate_pointers(9, [0, 2, 5, 7, 8], [0, 2, 4]) != []     # misses row 8
    assert csrk.validate_pointers(9, [0, 2, 5, 7, 9], [0, 2, 3]) != []     # misses SR 3
    assert csrk.validate_pointers(9, [0, 5, 2, 7, 9], [0, 2, 4]) != []     # decreasing


def test_group_sizes():
    for n in (1, 31, 32, 33, 1000):
        for sr in (1, 7, 32):
            for ssr in (1, 3, 8):
                a, b = csrk.fixed_pointers(n, sr, ssr)
                d = np.diff(a)
                assert np.all(d[:-1] == sr) and 1 <= d[-1] <= sr
                e = np.diff(b)
                assert np.all(e[:-1] == ssr) and 1 <= e[-1] <= ssr
