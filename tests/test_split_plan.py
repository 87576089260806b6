"""The split-K plan of grouped Grams (plv_gram_split_plan, host only): which
tiles run as several parts, and how many, for the tuner's factors.  No GPU:
the plan is host arithmetic in the library."""
import math

import pytest

from paper_1710_08037_gb300 import _lib


def plan(nkb, chunk=16, grid=152, split=1):
    import paper_1710_08037_gb300 as plv
    return plv.gram_split_plan(nkb, chunk, grid, split)


def test_no_split_factor_keeps_every_tile_whole():
    assert plan([313, 250, 32, 1], split=0) == [1, 1, 1, 1]
    assert plan([], split=4) == []


def test_few_long_tiles_split_into_parts_of_at_least_2048_samples():
    # 8 tiles of 313 K blocks: W = 2504, the fair share ceil(2504 / 152) = 17
    # is below the 64-block minimum part, so L = 64 and S = ceil(313 / 64) = 5
    assert plan([313] * 8) == [5] * 8
    assert plan([313] * 8, chunk=4) == [5] * 8
    assert plan([313] * 8, split=4) == [5] * 8


def test_parts_are_whole_chunks_of_at_least_64_blocks():
    for chunk in (4, 16):
        for n in (1, 3, 16, 17, 64, 65, 100, 313, 384):
            (S,) = plan([n], chunk=chunk, grid=152, split=64)
            nch = math.ceil(n / chunk)
            want = 1 if n <= 64 else min(math.ceil(n / 64), nch)
            assert S == want, (chunk, n, S)
            assert 1 <= S <= nch


def test_only_tiles_longer_than_the_fair_share_split():
    # 1000 tiles of 32 K blocks and one of 384: W = 32384, fair share per CTA
    # at f = 1 is ceil(32384 / 152) = 214 K blocks: only the long tile splits
    nkb = [384] + [32] * 1000
    S = plan(nkb)
    assert S[0] == 2 and set(S[1:]) == {1}
    # f = 4: the share is 54, below the 64-block minimum: 6 parts
    S = plan(nkb, split=4)
    assert S[0] == 6 and set(S[1:]) == {1}
    # longer tiles never get fewer parts than shorter ones
    nkb = [10, 50, 100, 200, 300, 384, 20, 250]
    for f in (1, 2, 4):
        S = plan(nkb, split=f, grid=8)
        for a in range(len(nkb)):
            for b in range(len(nkb)):
                if nkb[a] >= nkb[b]:
                    assert S[a] >= S[b]


def test_partial_slots_are_bounded():
    # 2000 tiles of 384 K blocks take 6 slots (one per part) each when split:
    # at most 8192 slots (1 GiB) are handed out, longest tiles first
    nkb = [384] * 2000
    S = plan(nkb, chunk=4, grid=4000, split=64)
    split = [s for s in S if s > 1]
    assert set(split) == {6}
    assert 0 < len(split) < len(nkb)
    assert sum(split) <= 8192 < sum(split) + 6


def test_bad_arguments_are_rejected():
    import paper_1710_08037_gb300 as plv
    for args in (([5], 0, 152, 1), ([5], 16, 0, 1), ([5], 16, 152, -1), ([5], 16, 152, 65),
                 ([0], 16, 152, 1)):
        with pytest.raises(_lib.PlvError) as ei:
            plv.gram_split_plan(*args)
        assert ei.value.status == _lib.PLV_ERR_INVALID
