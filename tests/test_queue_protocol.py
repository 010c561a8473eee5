"""The flag-queue protocol of the persistent form (csrc/k_persist.cu at depth 1,
csrc/k_queue.cu at depth T), checked as a model on the host: two slots per
directed edge suffice.

Every segment i runs blocks b = 0, 1, ...; its block b needs message b from
both neighbours (their edge values at time bT) and, once done, sends message
b + 1 to both.  Message m goes into slot m % 2 of the edge's queue and is
published by raising the edge's sequence word to m + 1; a consumer reads
message m once the word is at least m + 1.  The model runs every interleaving
a random scheduler produces (a CTA's edge tiles are independent actors, as in
k_queue.cu, where the left and right edge tiles are different warps) and
checks that no message is overwritten before its consumer read it, that every
message read is the one expected, and that the run always finishes (no
deadlock).
"""
import random

import pytest


def run_model(S: int, blocks: int, seed: int, edge_tiles_split: bool) -> None:
    rng = random.Random(seed)
    # one queue per mailbox, as in the kernels: (i, "inL") carries the left
    # neighbour's right-edge values to segment i's left edge, (i, "inR") the
    # right neighbour's left-edge values to its right edge (with one or two
    # segments these are still distinct queues)
    slots, seq, read = {}, {}, {}
    for i in range(S):
        for q in ("inL", "inR"):
            slots[(i, q)] = [None, None]
            seq[(i, q)] = 0
            read[(i, q)] = set()

    def send(mb, m):
        old = slots[mb][m % 2]
        # the slot's previous message (m - 2) must have been read already
        assert old is None or old in read[mb], (mb, m, old)
        slots[mb][m % 2] = m
        seq[mb] = max(seq[mb], m + 1)

    def inbox(i, side):
        return (i, "inL") if side == "L" else (i, "inR")

    def outbox(i, side):     # where this side's edge values go
        return ((i - 1) % S, "inR") if side == "L" else ((i + 1) % S, "inL")

    # message 0 of every queue: the initial state
    for i in range(S):
        for side in ("L", "R"):
            send(outbox(i, side), 0)

    # actors: each segment's left-edge and right-edge work (one actor when the
    # segment is a single tile), each with its own block counter; a segment's
    # interior needs no queue.  Both edges of a block must finish before the
    # segment's next block starts (the CTA barrier).
    sides = [("L", "R")] if not edge_tiles_split else [("L",), ("R",)]
    actors = [(i, sd) for i in range(S) for sd in sides]
    block = {a: 0 for a in actors}
    seg_block = [0] * S
    done_sides = [set() for _ in range(S)]
    steps = 0
    while min(seg_block) < blocks:
        ready = [a for a in actors
                 if block[a] < blocks and block[a] <= seg_block[a[0]]
                 and all(seq[inbox(a[0], side)] >= block[a] + 1 for side in a[1])]
        assert ready, "deadlock"
        a = rng.choice(ready)
        i, sd = a
        b = block[a]
        for side in sd:
            mb = inbox(i, side)
            assert slots[mb][b % 2] == b, (mb, b, slots[mb])
            read[mb].add(b)
        for side in sd:
            send(outbox(i, side), b + 1)   # this side's edge values after block b
            done_sides[i].add(side)
        block[a] = b + 1
        if done_sides[i] == {"L", "R"}:
            done_sides[i] = set()
            seg_block[i] += 1
        steps += 1
        assert steps < 100 * S * blocks


@pytest.mark.parametrize("S", [1, 2, 3, 7])
@pytest.mark.parametrize("split", [False, True])
def test_two_slots_suffice_under_random_interleavings(S, split):
    for seed in range(40):
        run_model(S, blocks=12, seed=seed, edge_tiles_split=split)


def test_the_model_catches_a_single_slot_queue():
    """With one slot per edge the same scheduler finds an overwrite of an
    unread message (the check is not vacuous)."""
    def run_one_slot(seed):
        rng = random.Random(seed)
        S, blocks = 3, 8
        slot, seq, read = {}, {}, {}
        for i in range(S):
            for d in (-1, 1):
                e = (i, (i + d) % S)
                slot[e], seq[e], read[e] = 0, 1, set()
        block = [0] * S
        while min(block) < blocks:
            ready = [i for i in range(S) if block[i] < blocks and
                     seq[((i - 1) % S, i)] >= block[i] + 1 and seq[((i + 1) % S, i)] >= block[i] + 1]
            i = rng.choice(ready)
            b = block[i]
            for nb in ((i - 1) % S, (i + 1) % S):
                if slot[(nb, i)] != b:
                    return True          # read a message other than b: overwritten
                read[(nb, i)].add(b)
            for nb in ((i - 1) % S, (i + 1) % S):
                slot[(i, nb)] = b + 1
                seq[(i, nb)] = b + 2
            block[i] = b + 1
        return False
    assert any(run_one_slot(seed) for seed in range(200))
