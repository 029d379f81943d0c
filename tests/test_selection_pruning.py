"""The pruning rule behind the k x k selection networks, checked on the CPU.

After sorting every column of a k x k block and then every rank-row across
the columns, entry (i, j) has at least (i+1)(j+1) entries at or below it and
(k-i)(k-j) at or above it.  With M = (k^2+1)/2 the median is then the
(M - #{(k-i)(k-j) > M})-th smallest of the entries with (i+1)(j+1) <= M and
(k-i)(k-j) <= M.  This restates the rule in numpy and compares it with a
plain sort, including blocks full of ties."""
import numpy as np
import pytest


def pruned_median(block: np.ndarray) -> int:
    k = block.shape[0]
    m = (k * k + 1) // 2
    s = np.sort(block, axis=0)          # columns
    s = np.sort(s, axis=1)              # rank-rows across the columns
    cand, below = [], 0
    for i in range(k):
        for j in range(k):
            if (k - i) * (k - j) > m:
                below += 1
            elif (i + 1) * (j + 1) <= m:
                cand.append(s[i, j])
    cand.sort()
    return cand[m - below - 1]


@pytest.mark.parametrize("k,ncand", [(3, 3), (5, 13), (7, 29), (9, 47), (11, 73), (13, 105)])
def test_pruned_selection_equals_sorted_median(k, ncand):
    rng = np.random.default_rng(k)
    m = (k * k + 1) // 2
    c = sum(1 for i in range(k) for j in range(k) if (i + 1) * (j + 1) <= m and (k - i) * (k - j) <= m)
    assert c == ncand
    for trial in range(300):
        hi = [2, 5, 256, 65536][trial % 4]   # heavy ties through full range
        block = rng.integers(0, hi, size=(k, k))
        assert pruned_median(block) == np.sort(block, axis=None)[m - 1]


def test_sorted_rows_keep_sorted_columns():
    """Sorting rank-rows of a column-sorted block keeps the columns sorted,
    the property the (i+1)(j+1) bound rests on."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        b = np.sort(rng.integers(0, 50, size=(7, 7)), axis=0)
        s = np.sort(b, axis=1)
        assert np.all(np.diff(s, axis=0) >= 0)
