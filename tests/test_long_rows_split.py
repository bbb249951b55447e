"""Index logic of the dense-coupling-row split, restated on the host: block b
of nb takes entries [L b / nb, L (b + 1) / nb) of the concatenated long rows
and writes one partial per long row its range meets; the combining block
sums, per row, the partials of the blocks whose range overlaps the row.  For
any lengths and grid sizes every entry must be counted exactly once and the
combining block must read exactly the partials that were written."""
import numpy as np
import pytest


def cut(L, b, nb):
    return L * b // nb


def written(ptr, nb):
    """(row, block) pairs a row pass writes, following the partial loop."""
    L, nlr, out = ptr[-1], len(ptr) - 1, set()
    for b in range(nb):
        e0, e1 = cut(L, b, nb), cut(L, b + 1, nb)
        if e0 >= e1:
            continue
        s = 0
        while s + 1 < nlr and ptr[s + 1] <= e0:
            s += 1
        while s < nlr and ptr[s] < e1:
            out.add((s, b))
            s += 1
    return out


def read(ptr, nb):
    """(row, block) pairs the combining block sums, following its overlap test."""
    L, out = ptr[-1], set()
    for s in range(len(ptr) - 1):
        p0, p1 = ptr[s], ptr[s + 1]
        for b in range(nb):
            e0, e1 = cut(L, b, nb), cut(L, b + 1, nb)
            if e0 < e1 and e0 < p1 and e1 > p0:
                out.add((s, b))
    return out


@pytest.mark.parametrize("seed", range(40))
def test_split_covers_each_entry_once(seed):
    rng = np.random.default_rng(seed)
    nlr = int(rng.integers(1, 65))
    lens = rng.integers(1025, 5000, size=nlr) if seed % 3 else rng.integers(1025, 1100, size=nlr)
    ptr = np.concatenate([[0], np.cumsum(lens)]).tolist()
    nb = int(rng.choice([1, 2, 7, 152, 456, 1216, ptr[-1] + 5]))
    w, r = written(ptr, nb), read(ptr, nb)
    assert w == r
    # Entry coverage: the block ranges tile [0, L) and each (row, block) pair
    # sums exactly the intersection of the two ranges.
    L = ptr[-1]
    count = np.zeros(L, dtype=np.int64)
    for s, b in w:
        lo = max(cut(L, b, nb), ptr[s])
        hi = min(cut(L, b + 1, nb), ptr[s + 1])
        assert lo < hi
        count[lo:hi] += 1
    assert np.all(count == 1)
