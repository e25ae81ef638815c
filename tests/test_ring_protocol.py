"""Discrete model of the shared-memory ring protocol of the persistent kernels (CPU only).

The persistent low-rank and channel-wise kernels stream factor tiles through a ring of
`ns` shared-memory slots: a producer thread waits for slot use u - ns to be released
(mbarrier `empty[s]`, one arrival per consumer warp), arms `full[s]` with the tile's byte
count and issues a bulk copy that completes on `full[s]`; every consumer warp waits for
`full[s]` with the parity of the use, reads the tile and arrives on `empty[s]`.  A parity
wait only tells "the phase with this parity has completed" apart from "it has not" while
the barrier is at most one phase ahead of the waiter, so the protocol must never let a
barrier run two phases ahead of anyone still waiting on it.

This model executes the protocol under random schedules (copies land out of order, warps
and the producer interleave arbitrarily, an abort may be raised mid-run) and checks:
every warp reads each use's data after it landed and before the slot is rewritten, no
parity wait is ever ambiguous, nothing deadlocks, and every issued copy has landed before
the producer exits (its drain of the last ring-full of slots)."""
import random

import pytest


class MBarrier:
    """mbarrier with an expected-arrival count, a transaction byte count and a phase
    counter (phases completed so far)."""

    def __init__(self, count):
        self.count = count
        self.pending = count
        self.tx = 0
        self.completed = 0

    def _check(self):
        assert self.pending >= 0
        if self.pending == 0 and self.tx == 0:
            self.completed += 1
            self.pending = self.count

    def arrive(self):
        self.pending -= 1
        self._check()

    def arrive_expect_tx(self, nbytes):
        self.tx += nbytes
        self.pending -= 1
        self._check()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        assert self.tx >= 0
        self._check()

    def try_wait_parity(self, parity, use):
        """True once the phase of the given parity has completed.  `use` is the index of
        the completion the waiter needs (0-based); the answer is unambiguous only while the
        barrier has completed at most use + 1 phases."""
        assert self.completed <= use + 1, "parity wait ambiguous: barrier two phases ahead"
        return (self.completed & 1) != parity


def run_ring(ns, warps, uses, seed, abort_at=None, bug=None):
    rng = random.Random(seed)
    full = [MBarrier(1) for _ in range(ns)]
    empty = [MBarrier(warps) for _ in range(ns)]
    slot_data = [None] * ns
    in_flight = []                       # (slot, use, nbytes)
    abort = False

    # producer state
    p_use, p_state, drain = 0, "issue", []
    # consumer warp states: next use index
    c_use = [0] * warps

    def producer_step():
        nonlocal p_use, p_state, drain, abort
        if p_state == "issue":
            if p_use == uses or abort:
                back = min(p_use, ns)
                drain = [p_use - j for j in range(1, back + 1)]
                p_state = "drain"
                return True
            s = p_use % ns
            if p_use >= ns and bug != "no_release_wait":
                prev = p_use - ns                       # the use whose release we need
                par = (prev // ns) & 1
                if bug == "wrong_parity":
                    par ^= 1
                if not empty[s].try_wait_parity(par, prev // ns):
                    return False
            nbytes = rng.choice([16, 32, 48])
            full[s].arrive_expect_tx(nbytes)
            in_flight.append((s, p_use, nbytes))
            p_use += 1
            return True
        if p_state == "drain":
            if not drain:
                p_state = "done"
                return True
            u = drain[-1]
            s = u % ns
            if full[s].try_wait_parity((u // ns) & 1, u // ns):
                drain.pop()
                return True
            return False
        return False

    def land_step():
        if not in_flight:
            return False
        i = rng.randrange(len(in_flight))       # copies complete out of order
        s, u, nbytes = in_flight.pop(i)
        slot_data[s] = u
        full[s].complete_tx(nbytes)
        return True

    def consumer_step(w):
        nonlocal abort
        u = c_use[w]
        if u == uses or abort:
            return False
        s = u % ns
        if not full[s].try_wait_parity((u // ns) & 1, u // ns):
            return False
        assert slot_data[s] == u, f"warp {w} read use {slot_data[s]} in slot {s}, wanted {u}"
        empty[s].arrive()
        c_use[w] += 1
        if abort_at is not None and u == abort_at and w == 0:
            abort = True                        # e.g. a bounded wait elsewhere gave up
        return True

    for _ in range(10 ** 6):
        actors = [producer_step, land_step] + [lambda w=w: consumer_step(w) for w in range(warps)]
        rng.shuffle(actors)
        progressed = False
        for a in actors:
            if a():
                progressed = True
                break
        consumers_done = abort or all(u == uses for u in c_use)
        if p_state == "done" and consumers_done:
            break
        assert progressed, "deadlock"
    assert p_state == "done"
    assert not in_flight, "producer exited with copies in flight"
    if abort_at is None:
        assert all(u == uses for u in c_use)


@pytest.mark.parametrize("ns,warps", [(4, 16), (2, 3), (11, 8), (1, 2)])
@pytest.mark.parametrize("seed", range(6))
def test_ring_protocol_random_schedules(ns, warps, seed):
    run_ring(ns, warps, uses=7 * ns + 3, seed=seed)


@pytest.mark.parametrize("seed", range(6))
def test_ring_protocol_abort_drains_copies(seed):
    run_ring(4, 16, uses=40, seed=seed, abort_at=13)


@pytest.mark.parametrize("bug", ["no_release_wait", "wrong_parity"])
def test_ring_model_catches_planted_protocol_bugs(bug):
    """A producer that does not wait for the release, or waits with the parity of the
    wrong use, trips the model on some schedule."""
    caught = 0
    for seed in range(20):
        try:
            run_ring(4, 16, uses=40, seed=seed, bug=bug)
        except AssertionError:
            caught += 1
    assert caught > 0


def test_ring_model_detects_missing_release():
    """The model itself: a producer that does not wait for the release overwrites a slot
    that a warp has not read yet (or runs a barrier two phases ahead)."""
    full = MBarrier(1)
    full.arrive_expect_tx(16)
    full.complete_tx(16)                        # use 0 landed
    full.arrive_expect_tx(16)
    full.complete_tx(16)                        # use 1 in the same slot, no release wait
    with pytest.raises(AssertionError):
        full.try_wait_parity(0, 0)              # a warp still waiting for use 0


# ---------------------------------------------------------------- grid barrier ----------

def run_grid_barrier(G, barriers, seed, extra=0, budget=None, bug=None):
    """Monotonic arrival counter (no reset): barrier g (1, 2, ...) completes once the
    counter reaches g (G + extra).  Returns the per-CTA outcome ('done' or 'timeout')."""
    rng = random.Random(seed)
    counter = 0
    gen = [0] * G                    # barriers passed
    arrived = [False] * G            # arrived at the current barrier, now polling
    polls = [0] * G
    arrivals = [0] * (barriers + 1)  # CTAs that arrived at barrier g
    state = ["run"] * G
    for _ in range(10 ** 6):
        live = [c for c in range(G) if state[c] == "run"]
        if not live:
            break
        c = rng.choice(live)
        if gen[c] == barriers:
            state[c] = "done"
            continue
        g = gen[c] + 1
        if not arrived[c]:
            counter += 1             # red.release.gpu.add
            arrivals[g] += 1
            arrived[c] = True
            polls[c] = 0
            if bug == "reset" and arrivals[g] == G:
                counter = 0          # a counter reset at each barrier, as a planted bug
        target = (g if bug != "reset" else 1) * (G + extra)
        if counter >= target:        # ld.acquire.gpu poll
            assert arrivals[g] == G, f"CTA {c} left barrier {g} after {arrivals[g]} of {G} arrivals"
            gen[c] += 1
            arrived[c] = False
        else:
            polls[c] += 1
            if budget is not None and polls[c] > budget:
                state[c] = "timeout"
    return state


@pytest.mark.parametrize("G", [1, 2, 7, 152])
@pytest.mark.parametrize("seed", range(3))
def test_grid_barrier_orders_every_generation(G, seed):
    assert run_grid_barrier(G, barriers=9, seed=seed) == ["done"] * G


def test_grid_barrier_extra_arrival_times_out_everywhere():
    """The test hook's extra arrival can never come: every CTA's wait runs out its budget
    (the kernel then records TDAGW_ERR_TIMEOUT) instead of hanging or passing."""
    assert run_grid_barrier(5, barriers=3, seed=1, extra=1, budget=200) == ["timeout"] * 5


def test_grid_barrier_model_catches_a_reset_counter():
    """Resetting the counter at each barrier lets a late CTA miss the completion; the model
    reports it as a timeout (or an early exit) on some schedule."""
    outcomes = [run_grid_barrier(6, barriers=6, seed=s, budget=5000, bug="reset") for s in range(10)]
    assert any(o != ["done"] * 6 for o in outcomes)
