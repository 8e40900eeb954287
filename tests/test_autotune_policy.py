"""The paper's kernel-selection rule (Eq. 2-5) against the kernel types and
H values printed in Tables 3 and 4, and the candidate set of the autotuner."""
import json
import os

import pytest

from paper_1707_09683_gb300 import autotune

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables_3_4_kernel_selection.json")


@pytest.mark.parametrize("filt,key", [("msv", "msv_table_3"), ("ssv", "ssv_table_4")])
def test_eq4_eq5_reproduce_tables_3_and_4(filt, key):
    rows = json.load(open(GOLDEN))[key]
    assert len(rows) == 14
    for S, m, H, H1 in rows:
        ch = autotune.paper_policy(m, filt, switch=False)
        assert (ch.S, ch.H) == (S, H), (filt, m)
        assert ch.W == 128 // S and ch.L == -(-32 // S)        # L = ceil(s / S), Eq. 3
        single = autotune.PaperChoice(S=1, W=128, L=32, H=max(2, -(-m // 128)))
        assert single.H == H1, (filt, m)


def test_eq3_closed_forms():
    # W = s w_r / (w_v S) = 128 / S; the 2-lane kernel covers 64 * H_max.
    for i in range(1, 8):
        assert autotune._w(2 ** i) == 128 // 2 ** i
    assert autotune.paper_policy(64 * 45, "msv", switch=False).S == 2
    assert autotune.paper_policy(64 * 45 + 1, "msv", switch=False).S == 1
    assert autotune.paper_policy(64 * 50 + 1, "ssv", switch=False).S == 1
    assert autotune.paper_policy(1, "msv", switch=False).H == 2


def test_performance_switch():
    assert autotune.paper_policy(15, "msv").S == 32          # m <= m_min
    assert autotune.paper_policy(21, "msv").S == 128
    assert autotune.paper_policy(2450, "msv").S == 2
    assert autotune.paper_policy(2451, "msv").S == 1          # m > m_max (MSV)
    assert autotune.paper_policy(1000, "ssv").S == 4
    assert autotune.paper_policy(1001, "ssv").S == 1          # m > m_max (SSV)


def test_candidates_cover_and_include_paper_point():
    for m in (1, 24, 48, 100, 400, 1111, 2405, 3072):
        c = autotune.candidates(m)
        assert c, m
        for lanes, words in c:
            assert 2 * lanes * words >= m
            assert lanes in autotune.LANES and words in autotune.WORDS
        pp = autotune.paper_point(m, "msv")
        assert pp in c
