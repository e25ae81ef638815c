"""Discrete model of the per-tile counters of the tensor-core low-rank kernel (CPU only).

In the low-rank mode the tensor-core kernel has no grid barrier between a stage's
epilogue and the next stage's V^H X items.  Each epilogue item (row tile t of 256 rows,
trajectory group g) writes the new stage input of its rows, then one thread adds 1 to the
tile's counter with release semantics.  A V^H X item of the next stage reads the rows of
its K-range (chunks [c0, c1) of 16 rows: tiles c0 16 / 256 .. (c1 16 - 1) / 256); before
that one thread waits (acquire) until each of those tiles' counters reaches the number of
epilogue items the tile has had in all previous stages (the sum of the per-stage group
counts, which change with the number of active trajectories).  The other phases of a stage
keep their two grid barriers; one more barrier precedes the last observables.

This model runs the protocol with every CTA as a coroutine under random schedules (any
CTA may be arbitrarily slow) and checks: every V^H X item reads only tiles whose previous
epilogue items have all finished writing, never a tile that a later epilogue is writing;
nothing deadlocks; the last observables see every tile's last epilogue.  Planted protocol
bugs (a target one stage short, the last tile of a K-range not waited for, the counter
released before the write completes, no final barrier) must be caught."""
import random

import pytest

ROWS = 256
CHUNK = 16


class Barrier:
    def __init__(self, n):
        self.n, self.arrived, self.gen = n, 0, 0

    def arrive(self):
        self.arrived += 1
        g = self.gen
        if self.arrived == self.n:
            self.arrived, self.gen = 0, self.gen + 1
        return g


def run_model(seed, ctas=5, Nt=7, steps=3, bug=None):
    rng = random.Random(seed)
    nch = Nt * ROWS // CHUNK
    # per-step group counts of the epilogue (the active trajectories shrink over time)
    gcs = [rng.randint(1, 3) for _ in range(steps)]
    KS = rng.randint(1, 6)                      # K-ranges of V^H X per V^H tile
    Mt = rng.randint(1, 2)                      # V^H tiles
    counter = [0] * Nt                          # released epilogue items per tile
    done_items = [0] * Nt                       # epilogue items whose writes completed
    writing = [0] * Nt                          # epilogue items writing the tile now
    readers = [0] * Nt                          # V^H X items reading the tile now
    bar = Barrier(ctas)
    log = []

    def barrier():
        g = bar.arrive()
        while bar.gen == g:
            yield "wait"

    def cta(c):
        target = 0
        for n in range(steps):
            GC = gcs[n]
            for st in range(4):
                # A: V^H X items of this CTA
                for item in range(c, Mt * KS, ctas):
                    ks = item // Mt
                    c0, c1 = ks * nch // KS, (ks + 1) * nch // KS
                    if c1 <= c0:
                        continue
                    t0, t1 = c0 * CHUNK // ROWS, (c1 * CHUNK - 1) // ROWS
                    wait_t1 = t1 - 1 if bug == "range" and t1 > t0 else t1
                    want = target - (gcs[n - 1] if bug == "target" and st == 0 and n > 0 else 0)
                    for t in range(t0, wait_t1 + 1):
                        while counter[t] < want:
                            yield "wait"
                    for t in range(t0, t1 + 1):
                        readers[t] += 1
                    yield "run"
                    for t in range(t0, t1 + 1):
                        # every epilogue item of the previous stages has written the tile,
                        # and none of this stage is writing it
                        if done_items[t] != target or writing[t]:
                            log.append(("stale read", n, st, t, done_items[t], target))
                        readers[t] -= 1
                yield from barrier()
                yield "run"                      # B
                yield from barrier()
                # C: epilogue items (t, g) of this CTA
                for item in range(c, Nt * GC, ctas):
                    t = item % Nt
                    if readers[t]:
                        log.append(("write under a reader", n, st, t))
                    writing[t] += 1
                    if bug == "early_release":
                        counter[t] += 1
                    yield "run"                  # the rows are being written
                    writing[t] -= 1
                    done_items[t] += 1
                    if bug != "early_release":
                        counter[t] += 1
                target += GC
        if bug != "no_final_barrier":
            yield from barrier()
        # the last observables read every tile's last partial sums
        for t in range(Nt):
            if done_items[t] != target:
                log.append(("observables before the last epilogue", t, done_items[t], target))

    agents = {c: cta(c) for c in range(ctas)}
    state = {c: None for c in range(ctas)}
    spins = 0
    while agents:
        c = rng.choice(list(agents))
        try:
            r = next(agents[c])
        except StopIteration:
            del agents[c]
            continue
        spins = spins + 1 if r == "wait" else 0
        state[c] = r
        if spins > 20000:
            log.append(("deadlock",))
            break
    return log


@pytest.mark.parametrize("seed", range(60))
def test_tile_counters_read_only_finished_tiles(seed):
    assert run_model(seed, ctas=3 + seed % 5, Nt=2 + seed % 9, steps=1 + seed % 4) == []


@pytest.mark.parametrize("bug", ["target", "range", "early_release", "no_final_barrier"])
def test_planted_protocol_bugs_are_caught(bug):
    caught = sum(1 for seed in range(80) if run_model(seed, ctas=4, Nt=6, steps=3, bug=bug))
    assert caught > 0, bug
