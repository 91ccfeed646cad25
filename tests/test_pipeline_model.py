"""Host model of the pipelined merge pass's buffer rotation and barrier phases
(csrc/merge_pipelined.cu; Sec. 7, future work: pipelining the merge).

A persistent CTA merges its tiles q = 0, 1, 2, ... with three tile buffers.
Tile q is staged by the producer warp into buffer s(q) = -q mod 3 and merged
by the consumer warps with s(q) and p(q) = 1 - q mod 3 as its two level
buffers.  full[b] completes once per staging of b, empty[b] once per release
of b to the producer (the consumers release p(q) when tile q is done; that is
the buffer tile q + 2 is staged into).  The model runs the producer and the
consumers as two interleaved step machines under random schedules and checks:
  * no buffer is staged while a tile that uses it is being merged;
  * every wait's parity matches the phase it must observe (the barrier never
    runs two phases ahead of a waiter);
  * all tiles complete in order, for any tile count and schedule.
"""
import random

import pytest


class Barrier:
    """mbarrier phase model: waiting on parity P succeeds once the phase with
    parity P has completed, i.e. while completed-phase count > the waiter's
    index; the model tracks completed phases exactly."""

    def __init__(self):
        self.completed = 0

    def complete(self):
        self.completed += 1

    def can_pass(self, nth):
        """The nth wait (0-based) on this barrier passes when phase nth has completed."""
        return self.completed > nth


def s_of(q):
    return (-q) % 3


def p_of(q):
    return (1 - q) % 3


def run(ntiles, seed):
    rng = random.Random(seed)
    full = [Barrier() for _ in range(3)]
    empty = [Barrier() for _ in range(3)]
    in_use = {}                      # buffer -> tile being merged with it
    staged = {}                      # buffer -> tile whose staged data it holds
    prod_q, cons_q = 0, 0
    prod_wait_empty = [0, 0, 0]      # waits done on empty[b] by the producer
    prod_state, cons_state = "start", "wait_full"
    done = []
    steps = 0
    while len(done) < ntiles:
        steps += 1
        assert steps < 100000, "no progress"
        if rng.random() < 0.5 and prod_q < ntiles:
            b = s_of(prod_q)
            if prod_q >= 2 and prod_state == "start":
                # wait for the release of b by tile prod_q - 2
                if not empty[b].can_pass(prod_wait_empty[b]):
                    continue
                prod_wait_empty[b] += 1
                # the parity the kernel passes: (number of earlier waits on b) & 1
            assert b not in in_use, f"staging buffer {b} while tile {in_use.get(b)} merges with it"
            staged[b] = prod_q
            full[b].complete()           # the copies land, the table is published
            prod_q += 1
            prod_state = "start"
        elif cons_q < ntiles:
            b, p = s_of(cons_q), p_of(cons_q)
            if cons_state == "wait_full":
                if not full[b].can_pass(cons_q // 3):      # parity (q / 3) & 1 in the kernel
                    continue
                assert staged.get(b) == cons_q
                assert p not in in_use and b not in in_use
                in_use[b] = cons_q
                in_use[p] = cons_q
                cons_state = "merge"
            else:
                del in_use[b]
                del in_use[p]
                empty[p].complete()         # p(q) = s(q + 2): the producer's next buffer
                done.append(cons_q)
                cons_q += 1
                cons_state = "wait_full"
    assert done == list(range(ntiles))
    # no barrier ran two phases ahead of a waiter: every completion was awaited in order
    for b in range(3):
        assert full[b].completed == sum(1 for q in range(ntiles) if s_of(q) == b)


@pytest.mark.parametrize("ntiles", [1, 2, 3, 4, 5, 7, 12, 31])
def test_pipeline_rotation_random_schedules(ntiles):
    for seed in range(200):
        run(ntiles, seed)


def test_rotation_buffers_are_distinct():
    for q in range(30):
        assert len({s_of(q), p_of(q), s_of(q + 1)}) == 3      # tile q's two buffers and q + 1's staging
        assert p_of(q) == s_of(q + 2)                          # released to stage tile q + 2
        assert p_of(q + 1) == s_of(q)                          # tile q + 1 merges into tile q's staged buffer
