"""Model check, on the CPU, of the tile hand-over of the fused pack + filter
kernel (csrc/shouji_pack_filter.cu).

Actors: 2 producer groups and 8 filter warps of one CTA, over its range of
tiles.  Group g packs blocks i = g, g + 2, ... (8 blocks per tile) and, after
its last block of tile t, waits for `freed[w]` phase k - 1 (k > 0) and then
arrives on `ready[w]`, where w = t % 8 and k = t // 8.  Filter warp w takes
tiles w, w + 8, ...: it waits for `ready[w]` phase k, filters the tile and
arrives on `freed[w]`.  A barrier only knows its current phase; a wait on
parity P returns as soon as the current phase's parity differs from P, which
is what the hardware's parity wait does.

Random interleavings check that every tile a filter warp accepts is the one
it expects, with all its producer arrivals and no arrival of another tile in
the same phase, and that the actors never deadlock.  The same model without
the producers' `freed` wait (the planted mistake) must fail the check.
"""
import random

import pytest

GROUPS, CONSUMERS, BLOCKS = 2, 8, 8


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
    def __init__(self, g, n_tiles, ready, freed, wait_freed=True):
        self.g, self.ready, self.freed, self.wait_freed = g, ready, freed, wait_freed
        self.blocks = list(range(g, n_tiles * BLOCKS, GROUPS))
        self.pos = 0

    def done(self):
        return self.pos == len(self.blocks)

    def step(self):
        """Packs one block; at the group's last block of a tile, hands the tile
        over.  False when blocked on `freed`."""
        i = self.blocks[self.pos]
        if i % BLOCKS >= BLOCKS - GROUPS:
            t = i // BLOCKS
            w, k = t % CONSUMERS, t // CONSUMERS
            if self.wait_freed and k > 0 and not self.freed[w].try_wait((k - 1) & 1):
                return False
            self.ready[w].arrive(t)
        self.pos += 1
        return True


class Consumer:
    def __init__(self, w, n_tiles, ready, freed, rng):
        self.w, self.ready, self.freed, self.rng = w, ready, freed, rng
        self.tiles = list(range(w, n_tiles, CONSUMERS))
        self.pos = 0
        self.work = 0  # filter steps left on the current tile

    def done(self):
        return self.pos == len(self.tiles)

    def step(self):
        k, t = self.pos, self.tiles[self.pos]
        if self.work == 0:
            if not self.ready[self.w].try_wait(k & 1):
                return False
            r = self.ready[self.w]
            assert r.phase == k + 1, "warp %d saw phase %d for its tile %d" % (self.w, r.phase, k)
            assert r.history[k] == {t}, "phase %d of ready[%d] held tiles %s, not %d" % (
                k, self.w, sorted(r.history[k]), t)
            self.work = 1 + self.rng.randrange(12)
            return True
        self.work -= 1
        if self.work == 0:
            self.freed[self.w].arrive(t)
            self.pos += 1
        return True


def run(n_tiles, seed, wait_freed=True):
    rng = random.Random(seed)
    ready = [Barrier(GROUPS) for _ in range(CONSUMERS)]
    freed = [Barrier(1) for _ in range(CONSUMERS)]
    actors = [Producer(g, n_tiles, ready, freed, wait_freed) for g in range(GROUPS)]
    actors += [Consumer(w, n_tiles, ready, freed, rng) for w in range(CONSUMERS)]
    while True:
        live = [a for a in actors if not a.done()]
        if not live:
            break
        rng.shuffle(live)
        # producers often run ahead: give them extra turns at random
        moved = False
        for a in live:
            for _ in range(1 + (rng.randrange(6) if isinstance(a, Producer) else 0)):
                if a.done() or not a.step():
                    break
                moved = True
        assert moved, "deadlock with %d tiles" % n_tiles
    for w in range(CONSUMERS):
        assert ready[w].phase == len(range(w, n_tiles, CONSUMERS))
        assert ready[w].pending == 0 and freed[w].pending == 0


@pytest.mark.parametrize("n_tiles", [1, 2, 7, 8, 9, 16, 17, 33, 64, 193])
def test_handover_delivers_each_tile_once_in_order(n_tiles):
    for seed in range(40):
        run(n_tiles, seed)


def test_handover_without_the_freed_wait_fails():
    """The planted mistake: producers that do not wait for `freed` lap a
    filter warp, and a parity wait then misses or misreads a phase."""
    failures = 0
    for seed in range(40):
        try:
            run(64, seed, wait_freed=False)
        except AssertionError:
            failures += 1
    assert failures > 0
