"""The mbarrier protocol of the persistent forward convolution (k_conv3_fwd_pers),
restated as four kinds of actors and run under random interleavings (no GPU).

Roles and barriers, as in the kernel:
  - the TMA thread fills stage g % NS for the g-th K-step of the block (over all
    its tiles in turn); before reusing a stage it waits for `empty` of that
    stage to have completed (g / NS) times, then arrives on `full` (one arrival
    plus the transaction bytes);
  - the MMA thread takes tile i into accumulator buffer i & 1; before reusing a
    buffer (i >= 2) it waits for `tempty[buf]` to have completed i / 2 times;
    per K-step it waits for `full` of the stage to have completed g / NS + 1
    times, issues, and commits to `empty` of the stage; after the tile's last
    K-step it commits to `tfull[buf]`;
  - each of the four epilogue warps waits for `tfull[buf]` to have completed
    i / 2 + 1 times, reads the accumulators and arrives on `tempty[buf]`
    (count 4).
An mbarrier wait only sees the parity of the barrier's phase, so a wait for the
k-th completion is ambiguous if the barrier has meanwhile completed k + 2 times;
the simulation fails on that as well as on a deadlock.
"""
import random

import pytest


class _Bar:
    def __init__(self, count):
        self.count, self.arrivals, self.completed = count, 0, 0

    def arrive(self):
        self.arrivals += 1
        if self.arrivals == self.count:
            self.arrivals, self.completed = 0, self.completed + 1

    def done(self, k):
        """The k-th completion (k = 0, 1, ...) has happened, as a parity wait sees it."""
        if self.completed >= k + 2:
            raise AssertionError("a parity wait would be ambiguous")
        return self.completed >= k + 1


def _run(tile_steps, NS, seed, epi_warps=4):
    rnd = random.Random(seed)
    full = [_Bar(1) for _ in range(NS)]
    empty = [_Bar(1) for _ in range(NS)]
    tfull, tempty = [_Bar(1), _Bar(1)], [_Bar(epi_warps), _Bar(epi_warps)]
    issued, read = [], []

    def producer():
        g = 0
        for steps in tile_steps:
            for _ in range(steps):
                st = g % NS
                if g >= NS:
                    while not empty[st].done(g // NS - 1):
                        yield
                full[st].arrive()
                g += 1
                yield

    def mma():
        g = 0
        for i, steps in enumerate(tile_steps):
            buf = i & 1
            if i >= 2:
                while not tempty[buf].done(i // 2 - 1):
                    yield
            for s in range(steps):
                st = g % NS
                while not full[st].done(g // NS):
                    yield
                issued.append((i, s))
                empty[st].arrive()
                g += 1
                yield
            tfull[buf].arrive()
            yield

    def epilogue(w):
        for i in range(len(tile_steps)):
            buf = i & 1
            while not tfull[buf].done(i // 2):
                yield
            # the tile's MMAs are all done when tfull completes
            assert sum(1 for t, _ in issued if t == i) == tile_steps[i]
            read.append((w, i))
            yield
            tempty[buf].arrive()
            yield

    actors = [producer(), mma()] + [epilogue(w) for w in range(epi_warps)]
    steps = 0
    while actors:
        a = rnd.choice(actors)
        try:
            next(a)
        except StopIteration:
            actors.remove(a)
        steps += 1
        assert steps < 10 ** 6, "deadlock"
    assert len(issued) == sum(tile_steps) and len(read) == epi_warps * len(tile_steps)


@pytest.mark.parametrize("NS", [2, 3, 4])
@pytest.mark.parametrize("ntile", [1, 2, 3, 5, 8])
def test_persistent_forward_protocol_has_no_deadlock_or_ambiguity(NS, ntile):
    for seed in range(40):
        rnd = random.Random(1000 * NS + 10 * ntile + seed)
        # K-steps per tile: Ci / 16 chunks times the planes inside the volume (2 or 3)
        steps = [rnd.choice([1, 2]) * rnd.choice([2, 3]) for _ in range(ntile)]
        _run(steps, NS, seed)


def test_a_missing_buffer_wait_is_caught():
    """The same protocol without the MMA thread's wait on tempty lets the next
    tile but one overwrite a buffer that the epilogue has not read: the
    simulation must fail on some interleaving."""
    failures = 0
    for seed in range(200):
        try:
            _run_without_tempty([2, 2, 2, 2, 2], 3, seed)
        except AssertionError:
            failures += 1
    assert failures > 0


def _run_without_tempty(tile_steps, NS, seed):
    rnd = random.Random(seed)
    full = [_Bar(1) for _ in range(NS)]
    empty = [_Bar(1) for _ in range(NS)]
    tfull = [_Bar(1), _Bar(1)]
    state = {"written": [0, 0], "read": [[0] * 4, [0] * 4]}

    def producer():
        g = 0
        for steps in tile_steps:
            for _ in range(steps):
                st = g % NS
                if g >= NS:
                    while not empty[st].done(g // NS - 1):
                        yield
                full[st].arrive()
                g += 1
                yield

    def mma():
        g = 0
        for i, steps in enumerate(tile_steps):
            buf = i & 1
            # planted: no wait for the epilogue to release the buffer; writing tile i
            # into it requires every warp to have read tile i - 2
            if i >= 2:
                assert min(state["read"][buf]) >= i // 2, "buffer overwritten before it was read"
            for _ in range(steps):
                st = g % NS
                while not full[st].done(g // NS):
                    yield
                empty[st].arrive()
                g += 1
                yield
            state["written"][buf] += 1
            tfull[buf].arrive()
            yield

    def epilogue(w):
        for i in range(len(tile_steps)):
            buf = i & 1
            while not tfull[buf].done(i // 2):
                yield
            yield
            state["read"][buf][w] += 1
            yield

    actors = [producer(), mma()] + [epilogue(w) for w in range(4)]
    steps = 0
    while actors:
        a = rnd.choice(actors)
        try:
            next(a)
        except StopIteration:
            actors.remove(a)
        steps += 1
        assert steps < 10 ** 6, "deadlock"
