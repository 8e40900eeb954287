"""The rule that forms packed query sets (host logic, CPU only).

A plan packs queries of fewer than 32 lanes 32 / lanes to a warp.  Among the
queries of one lane count, sorted by words per lane, it takes runs of
consecutive queries as sets; a set is padded to its largest word count H and
costs (32 / lanes) x H warp-words per row, a query left alone 5/4 of its own
words.  ``mpf_plan_pack_sets`` reports the runs the library picks; these
tests check them against brute force over every partition of small lists
(the least total cost, and a valid partition), and on the documented cases.
"""
import ctypes
import itertools

import numpy as np
import pytest

from paper_1707_09683_gb300 import build, mpf

GB300_SMEM = 232448   # shared memory per block on the GPU (227 KB)


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return mpf.load()


def _packable(h):
    # Built packed kernels: even word counts 8..48; at 227 KB every such
    # set's tables fit (the largest, 1 lane x 48 words x 32 queries, 209 KB).
    return h % 2 == 0 and 8 <= h <= 48


def _cost(words, runs, qp):
    c = 0
    for a, b in runs:
        c += 4 * qp * words[b - 1] if b - a >= 2 else 5 * words[a]
    return c


def _runs_of(set_start):
    runs, i = [], 0
    n = len(set_start)
    while i < n:
        if set_start[i] < 0:
            runs.append((i, i + 1))
            i += 1
        else:
            assert set_start[i] == i
            j = i
            while j < n and set_start[j] == i:
                j += 1
            runs.append((i, j))
            i = j
    return runs


def _best(words, qp):
    """Least cost over every partition into consecutive runs (brute force)."""
    n = len(words)
    best = None
    for cuts in itertools.product((0, 1), repeat=max(n - 1, 0)):
        bounds = [0] + [i + 1 for i, c in enumerate(cuts) if c] + [n]
        runs = list(zip(bounds[:-1], bounds[1:]))
        if any(b - a > qp or (b - a >= 2 and not _packable(words[b - 1])) for a, b in runs):
            continue
        c = _cost(words, runs, qp)
        best = c if best is None else min(best, c)
    return best


@pytest.mark.parametrize("lanes", [1, 2, 4, 8, 16])
def test_sets_have_the_least_cost(lanes):
    qp = 32 // lanes
    rng = np.random.default_rng(lanes)
    for _ in range(150):
        n = int(rng.integers(1, 10))
        choices = [6, 7, 8, 10, 12, 14, 18, 22, 26, 30, 38, 48] if rng.integers(3) else [20, 22, 24, 26]
        words = sorted(int(x) for x in rng.choice(choices, size=n))
        got = mpf.pack_sets(lanes, words, GB300_SMEM)
        runs = _runs_of(got)
        assert [a for r in runs for a in range(*r)] == list(range(n))
        for a, b in runs:
            assert b - a <= qp
            if b - a >= 2:
                assert _packable(words[b - 1]), (words, got)
        assert _cost(words, runs, qp) == _best(words, qp), (lanes, words, got)


def test_documented_cases():
    # Four 8-lane queries of 22 words: one set (16 x 22 < 5/4 x 88).
    assert list(mpf.pack_sets(8, [22] * 4)) == [0] * 4
    # Three of them: a set of 4 slots with one empty costs more than alone.
    assert list(mpf.pack_sets(8, [22] * 3)) == [-1] * 3
    # Seven 4-lane queries of 26 words fill 7 of 8 slots: a set.
    assert list(mpf.pack_sets(4, [26] * 7)) == [0] * 7
    # 27 one-lane queries of 14 words: a set of 32 slots; 17 do not pay.
    assert list(mpf.pack_sets(1, [14] * 27)) == [0] * 27
    assert list(mpf.pack_sets(1, [14] * 17)) == [-1] * 17
    # Sorted lists are cut where the padding would cost too much.
    assert list(mpf.pack_sets(16, [18, 18, 30, 30, 46])) == [0, 0, 2, 2, -1]
    assert list(mpf.pack_sets(8, [12] * 4 + [22] * 4 + [38])) == [0] * 4 + [4] * 4 + [-1]


def test_unbuilt_word_counts_and_small_shared_memory_never_pack():
    assert list(mpf.pack_sets(8, [6] * 4)) == [-1] * 4      # below 8 words: no packed kernel
    assert list(mpf.pack_sets(8, [21] * 4)) == [-1] * 4     # odd: no kernel of that word count
    assert list(mpf.pack_sets(8, [22] * 4, 0)) == [-1] * 4  # tables cannot fit
    # The largest 16-lane set (2 x 101.5 KB) fits 227 KB but not 150 KB.
    assert list(mpf.pack_sets(16, [48, 48], GB300_SMEM)) == [0, 0]
    assert list(mpf.pack_sets(16, [48, 48], 150 * 1024)) == [-1, -1]
    assert list(mpf.pack_sets(2, [])) == []


def test_invalid_arguments(lib):
    w = (ctypes.c_int * 3)(8, 10, 12)
    out = (ctypes.c_int * 3)()
    for lanes in (0, 3, 32, 64):
        assert lib.mpf_plan_pack_sets(lanes, w, 3, GB300_SMEM, out) == mpf.MPF_EINVAL
    desc = (ctypes.c_int * 3)(12, 10, 8)
    assert lib.mpf_plan_pack_sets(8, desc, 3, GB300_SMEM, out) == mpf.MPF_EINVAL
    assert lib.mpf_plan_pack_sets(8, None, 3, GB300_SMEM, out) == mpf.MPF_EINVAL
    assert lib.mpf_plan_pack_sets(8, w, 3, GB300_SMEM, None) == mpf.MPF_EINVAL
    assert lib.mpf_plan_pack_sets(8, w, -1, GB300_SMEM, out) == mpf.MPF_EINVAL
