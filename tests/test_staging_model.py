"""Host model of a merge CTA's staging plan (merge_tile.cuh: merge_plan_warp
and MergeGeom), checked for the rules a TMA bulk copy must follow.

For one output tile the plan stages K segments (segment r = items
[gsrc_r, gsrc_r + len_r) of the round's input `in`, n items long, which may
itself start off the 16-byte grid inside a larger buffer) into consecutive
spans of the shared buffer: span r starts at R_r, holds `head_r` items of
alignment slack, the segment, rounding up to 16 bytes, and 32 items of
transpose slack.  One bulk copy per segment runs from the 16-byte boundary at
or before the segment's start to the boundary at or after its end, or, where
that would pass the end of `in`, to the last boundary inside the segment, with
plain loads for the rest.  The model replays that arithmetic and checks, for
random tiles, key widths, fanouts, array ends and misaligned array bases:
  * source and destination of every copy are 16-byte aligned and its size is
    a multiple of 16 bytes (what cp.async.bulk requires);
  * no copy reads past the end of `in` or before the start of the buffer
    holding it;
  * each copy stays in its own span, spans do not overlap, and all fit the
    capacity MergeGeom reserves (S + K * (2E + 32) + E items);
  * the copies and the plain loads together deliver each segment exactly.
"""
import numpy as np
import pytest

SLACK = 32


def cap(S, K, E):
    return S + K * (2 * E + SLACK) + E


def plan(base_items, n, segs, size, S):
    """Replays the staging arithmetic.  base_items: offset of `in` (in items)
    from a 16-byte-aligned buffer start; segs: list of (gsrc, len)."""
    E = 16 // size
    in_mis = base_items % E
    spans, copies, plains = [], [], []
    R = 0
    for gsrc, ln in segs:
        head = (in_mis + gsrc) % E
        span = (head + ln + E - 1) // E * E + SLACK
        bulk_lo = gsrc - head
        bulk_up = (in_mis + gsrc + ln + E - 1) // E * E - in_mis
        bulk_hi = bulk_up if bulk_up <= n else (in_mis + gsrc + ln) // E * E - in_mis
        nbytes = (bulk_hi - bulk_lo) * size if (ln > 0 and bulk_hi > bulk_lo) else 0
        if nbytes:
            copies.append((R, bulk_lo, nbytes))                  # dst item offset, src item index, bytes
        first_plain = bulk_hi if nbytes else gsrc
        for e in range(max(first_plain, gsrc), gsrc + ln):
            plains.append((R + head + (e - gsrc), e))
        spans.append((R, span, head, gsrc, ln))
        R += span
    return in_mis, spans, copies, plains, R


@pytest.mark.parametrize("size", [4, 8])
@pytest.mark.parametrize("K", [2, 3, 4, 8, 16, 32])
def test_staging_obeys_bulk_copy_rules(size, K):
    rng = np.random.default_rng(size * 100 + K)
    E = 16 // size
    S = 8192 if size == 4 else 4096
    for trial in range(200):
        base_items = int(rng.integers(0, 4 * E))               # `in` may start off the 16-byte grid
        want = int(rng.integers(1, S + 1))                     # tile size (short at an array end)
        cuts = np.sort(rng.integers(0, want + 1, K - 1))
        lens = np.diff(np.concatenate([[0], cuts, [want]])).astype(int)
        starts = []
        pos = int(rng.integers(0, 1000))
        for ln in lens:                                        # runs one after another, gaps between
            starts.append(pos)
            pos += int(ln) + int(rng.integers(0, 50))
        n = pos - int(rng.integers(0, 50)) if rng.random() < 0.5 else pos   # sometimes end right at a segment
        n = max(n, max(s + int(l) for s, l in zip(starts, lens)))
        segs = list(zip(starts, (int(l) for l in lens)))
        in_mis, spans, copies, plains, total = plan(base_items, n, segs, size, S)
        assert total <= cap(S, K, E)
        stage = np.full(total, -1, dtype=np.int64)
        for dst, src, nbytes in copies:
            assert (dst * size) % 16 == 0                        # stage is 16-byte aligned
            assert ((base_items + src) * size) % 16 == 0         # absolute source address
            assert nbytes % 16 == 0 and nbytes > 0
            cnt = nbytes // size
            assert src + cnt <= n                                # never past the end of `in`
            assert base_items + src >= 0                         # never before the buffer start
            span = next(sp for sp in spans if sp[0] == dst)
            assert dst + cnt <= span[0] + span[1] - SLACK        # inside its own span, before the slack
            stage[dst: dst + cnt] = np.arange(src, src + cnt)
        for dst, src in plains:
            stage[dst] = src
        for (R, span, head, gsrc, ln), nxt in zip(spans, spans[1:] + [None]):
            assert head + ln <= span - SLACK
            if nxt is not None:
                assert R + span == nxt[0]                        # consecutive, no overlap
            assert np.array_equal(stage[R + head: R + head + ln], np.arange(gsrc, gsrc + ln))


def test_segment_ending_at_the_array_end_uses_plain_loads():
    """A segment whose last 16-byte chunk would pass the end of `in` is copied
    to the last boundary inside it and finished with plain loads."""
    in_mis, spans, copies, plains, _ = plan(0, 1003, [(900, 103)], 4, 8192)
    assert copies == [(0, 900, (1000 - 900) * 4)]
    assert [src for _, src in plains] == [1000, 1001, 1002]
