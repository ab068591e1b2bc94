"""Model check, on the CPU, of the tile hand-over of the fused pack + filter
kernel (csrc/shouji_pack_filter.cu).

Actors: 2 producer groups and 8 filter warps of one CTA, over its range of
tiles, and a queue of S slots (S is read from the kernel source).  Group g
packs blocks i = g, g + 2, ... (8 blocks per tile) and, after its last block
of tile t, waits for `freed[s]` phase k - 1 (k > 0) and then arrives on
`ready[s]`, where s = t % S and k = t // S.  A filter warp that is free takes
the next tile r from a shared counter, waits for `ready[r % S]` phase r // S,
filters the tile and arrives on `freed[r % S]`.  A barrier only knows its
current phase; a wait on parity P returns as soon as the current phase's
parity differs from P, which is what the hardware's parity wait does.

Random interleavings check that every tile a filter warp accepts is the one
it took, with all its producer arrivals and no arrival of another tile in the
same phase, and that the actors never deadlock.  Two planted mistakes must
fail the check: producers that skip the `freed` wait, and a queue with fewer
slots than filter warps.

Ring mode (shouji_pack_filter_results): tile t is packed into the ring entry
of slot s, over tile t - S, so each group waits for `freed[s]` phase k - 1
before its first block of t (not before its last), and no block of t may be
written while a filter warp still reads the entry.  With the wait before the
last block instead (a planted mistake) that check fails.
"""
import os
import random
import re

import pytest

GROUPS, CONSUMERS, BLOCKS = 2, 8, 8
_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1809_07858_gb300", "csrc", "shouji_pack_filter.cu")
SLOTS = int(re.search(r"#define SHOUJI_FUSED_SLOTS (\d+)", open(_SRC).read()).group(1))


class Barrier:
    def __init__(self, count):
        self.count = count
        self.pending = 0
        self.phase = 0          # completed phases
        self.tags = set()       # tiles whose arrivals went into the current phase
        self.history = []       # tiles of each completed phase

    def arrive(self, tag):
        self.pending += 1
        self.tags.add(tag)
        if self.pending == self.count:
            self.history.append(self.tags)
            self.pending, self.tags = 0, set()
            self.phase += 1

    def try_wait(self, parity):
        return (self.phase & 1) != parity


class Producer:
    def __init__(self, g, n_tiles, ready, freed, slots, wait_freed=True, ring=None,
                 wait_at_first=False):
        self.g, self.ready, self.freed, self.wait_freed = g, ready, freed, wait_freed
        self.slots = slots
        self.ring = ring                  # ring mode: slot -> tile being read, or None
        self.wait_at_first = wait_at_first
        self.blocks = list(range(g, n_tiles * BLOCKS, GROUPS))
        self.pos = 0

    def done(self):
        return self.pos == len(self.blocks)

    def step(self):
        """Packs one block; at the group's last block of a tile, hands the tile
        over.  False when blocked on `freed`."""
        i = self.blocks[self.pos]
        t = i // BLOCKS
        s, k = t % self.slots, t // self.slots
        first, last = i % BLOCKS < GROUPS, i % BLOCKS >= BLOCKS - GROUPS
        if self.wait_freed and k > 0 and (first if self.wait_at_first else last):
            if not self.freed[s].try_wait((k - 1) & 1):
                return False
        if self.ring is not None:
            # the block's words go to the ring entry of slot s
            assert self.ring[s] is None, "tile %d written over tile %d, still being read" % (
                t, self.ring[s])
        if last:
            self.ready[s].arrive(t)
        self.pos += 1
        return True


class Queue:
    def __init__(self, n_tiles):
        self.next, self.n_tiles = 0, n_tiles


class Consumer:
    def __init__(self, w, queue, ready, freed, slots, rng, ring=None):
        self.w, self.q, self.ready, self.freed, self.rng = w, queue, ready, freed, rng
        self.slots = slots
        self.ring = ring
        self.tile = None   # the tile taken, not yet accepted
        self.work = 0      # filter steps left on the accepted tile
        self.finished = False
        self.taken = []

    def done(self):
        return self.finished

    def step(self):
        if self.tile is None and self.work == 0:
            r = self.q.next
            self.q.next += 1
            if r >= self.q.n_tiles:
                self.finished = True
                return True
            self.tile = r
            self.taken.append(r)
            return True
        if self.tile is not None:
            r = self.tile
            s, k = r % self.slots, r // self.slots
            if not self.ready[s].try_wait(k & 1):
                return False
            b = self.ready[s]
            assert b.phase == k + 1, "warp %d saw phase %d of slot %d for tile %d" % (
                self.w, b.phase, s, r)
            assert b.history[k] == {r}, "phase %d of ready[%d] held tiles %s, not %d" % (
                k, s, sorted(b.history[k]), r)
            self.work = 1 + self.rng.randrange(12)
            self.tile = None
            self.accepted = r
            if self.ring is not None:
                self.ring[s] = r          # reads the entry until it frees the slot
            return True
        self.work -= 1
        if self.work == 0:
            if self.ring is not None:
                self.ring[self.accepted % self.slots] = None
            self.freed[self.accepted % self.slots].arrive(self.accepted)
        return True


def run(n_tiles, seed, wait_freed=True, slots=SLOTS, producer_turns=6, ring_mode=False,
        wait_at_first=None):
    rng = random.Random(seed)
    ready = [Barrier(GROUPS) for _ in range(slots)]
    freed = [Barrier(1) for _ in range(slots)]
    queue = Queue(n_tiles)
    ring = [None] * slots if ring_mode else None
    if wait_at_first is None:
        wait_at_first = ring_mode
    actors = [Producer(g, n_tiles, ready, freed, slots, wait_freed, ring, wait_at_first)
              for g in range(GROUPS)]
    consumers = [Consumer(w, queue, ready, freed, slots, rng, ring) for w in range(CONSUMERS)]
    actors += consumers
    while True:
        live = [a for a in actors if not a.done()]
        if not live:
            break
        rng.shuffle(live)
        # producers often run ahead, filter warps run at uneven speeds: give
        # actors extra turns at random
        moved = False
        for a in live:
            turns = producer_turns if isinstance(a, Producer) else 6
            for _ in range(1 + rng.randrange(turns)):
                if a.done() or not a.step():
                    break
                moved = True
        assert moved, "deadlock with %d tiles" % n_tiles
    assert sorted(t for c in consumers for t in c.taken) == list(range(n_tiles))
    for s in range(slots):
        assert ready[s].phase == len(range(s, n_tiles, slots))
        assert ready[s].pending == 0 and freed[s].pending == 0


def test_queue_holds_at_least_one_slot_per_filter_warp():
    assert SLOTS >= CONSUMERS


@pytest.mark.parametrize("n_tiles", [1, 2, 7, 8, 9, 10, 11, 16, 17, 33, 64, 193])
def test_handover_delivers_each_tile_once(n_tiles):
    for seed in range(40):
        run(n_tiles, seed)


def test_handover_without_the_freed_wait_fails():
    """Planted mistake: producers that do not wait for `freed` lap a filter
    warp, and a parity wait then misses or misreads a phase."""
    failures = 0
    for seed in range(40):
        try:
            # producers far faster than the filter warps, so that they lap them
            run(64, seed, wait_freed=False, producer_turns=200)
        except AssertionError:
            failures += 1
    assert failures > 0


def test_handover_with_fewer_slots_than_filter_warps_fails():
    """Planted mistake: with 4 slots a filter warp can take tile r before
    tile r - 4 is packed, and its parity wait then reads the older phase."""
    failures = 0
    for seed in range(40):
        try:
            run(64, seed, slots=4)
        except AssertionError:
            failures += 1
    assert failures > 0


@pytest.mark.parametrize("n_tiles", [1, 2, 7, 11, 12, 13, 24, 25, 64, 193])
def test_ring_mode_never_overwrites_a_tile_being_read(n_tiles):
    for seed in range(40):
        run(n_tiles, seed, ring_mode=True, producer_turns=50)


def test_ring_mode_with_the_wait_before_the_last_block_fails():
    """Planted mistake: in ring mode, waiting for `freed` only before the
    last block of a tile lets the first blocks overwrite a tile still being
    filtered."""
    failures = 0
    for seed in range(40):
        try:
            run(64, seed, ring_mode=True, wait_at_first=False, producer_turns=200)
        except AssertionError:
            failures += 1
    assert failures > 0
