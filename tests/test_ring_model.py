"""A host model of the reverse pass's staging ring, run under random
interleavings of its warps and of its copies' arrivals.

The kernel stages a tile's list in batches through K buffers.  Each warp, for
every batch u in order, waits for buffer u % K to hold batch u (the phase of
its mbarrier with parity (u / K) & 1), reads it, and releases it by adding one
to the buffer's count; the warp whose addition completes the count resets it
and refills the buffer with batch u + K (if there is one), and the refill's
arrival completes the next phase once its copies land.  Every wait is bounded:
a warp whose wait runs out stops at once (it releases nothing more), and
before the block exits one thread per buffer waits for the buffer's last fill
(the drain), so that no copy is still writing into the block's shared memory.

The model checks the protocol's claims: a buffer is never refilled while a
warp still has to read its batch or while its previous fill is in flight,
every warp that does not time out reads every batch once and in order, a wait
never sees a phase of another fill (parity aliasing), no interleaving
deadlocks, and no fill is in flight when the block exits.  Planted mistakes
(a refill by the first warp out, a failed warp that keeps releasing, an exit
without the drain) must each be caught by some interleaving.
"""
import random

import pytest


class ProtocolError(AssertionError):
    pass


def check(cond, what):
    if not cond:
        raise ProtocolError(what)


def run_ring(n_warps, K, nb, seed, refill_by_first=False, timeouts=0.0, stall=0.0, failed_keeps_releasing=False,
             drain=True):
    """One interleaving.  `timeouts`: probability that a scheduled warp whose
    phase has not completed gives up its wait instead of staying blocked;
    `stall`: probability that a fill's copies land only after every bounded wait
    of the warps has run out (they land during the drain, or never while the
    block runs); the last three arguments plant mistakes."""
    rng = random.Random(seed)
    content = [None] * K          # batch held by each buffer (written when its copies land)
    phase = [0] * K               # completed phases of each buffer's barrier
    inflight = [None] * K         # batch of the fill whose copies are still in flight
    stalled = [False] * K         # that fill lands only after the warps' waits
    last_fill = [None] * K        # ring use of each buffer's last fill
    released = [0] * K            # release count of each buffer
    reading = [set() for _ in range(K)]
    seen = [[] for _ in range(n_warps)]
    failed = [False] * n_warps
    fills = 0

    def fill(s, u):
        nonlocal fills
        check(not reading[s], "refill while a warp still reads the buffer")
        check(inflight[s] is None, "two fills in flight on one buffer")
        inflight[s] = u
        stalled[s] = rng.random() < stall
        last_fill[s] = u
        fills += 1

    def land(s):
        content[s] = inflight[s]
        inflight[s] = None
        phase[s] += 1

    for u in range(min(K, nb)):   # the warps' initial fills
        fill(u, u)
    # per warp: next batch and its step (0 wait, 1 read, 2 release); None when stopped
    state = [[0, 0] for _ in range(n_warps)]

    def done(w):
        return state[w] is None or state[w][0] >= nb

    while not all(done(w) for w in range(n_warps)):
        # copies land at any time while the warps run; the block exits as soon
        # as every warp is done, whatever is still in flight
        events = [("land", s) for s in range(K) if inflight[s] is not None and not stalled[s]]
        blocked = []
        for w in range(n_warps):
            if done(w):
                continue
            u, step = state[w]
            s = u % K
            if step == 0 and not failed[w]:
                # the hardware test: try_wait.parity(p) succeeds when the parity
                # of the completed-phase count differs from p, which is right
                # only while that count is u // K or u // K + 1
                check(u // K <= phase[s] <= u // K + 1, "parity would alias")
                if (phase[s] & 1) != ((u // K) & 1):
                    events.append(("warp", w))
                else:
                    blocked.append(w)
            else:
                events.append(("warp", w))
        if timeouts:
            events += [("timeout", w) for w in blocked if rng.random() < timeouts]
        if not events:
            # nothing else can move: a bounded wait runs out
            events = [("timeout", w) for w in blocked]
        check(events, "deadlock")
        kind, i = rng.choice(events)
        if kind == "land":
            land(i)
            continue
        w = i
        if kind == "timeout":
            failed[w] = True
            if failed_keeps_releasing:
                state[w][1] = 2   # the planted mistake: count the release anyway
            else:
                state[w] = None   # stop at once
            continue
        u, step = state[w]
        s = u % K
        if failed[w]:             # (planted variant only) release without reading
            step = 2
        if step == 0:
            # the wait succeeded: the phase it waited for is the current fill
            check(phase[s] == u // K + 1, "wait satisfied by another fill's phase")
            reading[s].add(w)
            state[w][1] = 1
        elif step == 1:
            check(content[s] == u, "read a batch other than its own")
            seen[w].append(content[s])
            reading[s].discard(w)
            state[w][1] = 2
        else:
            released[s] += 1
            last = released[s] == n_warps
            if refill_by_first and released[s] == 1 and u + K < nb:
                fill(s, u + K)  # the planted mistake: refill before every warp released
            elif last:
                released[s] = 0
                if u + K < nb and not failed[w]:
                    fill(s, u + K)
            state[w] = [u + 1, 0]
    if drain and any(failed):
        # one thread per buffer waits for the buffer's last fill
        for s in range(K):
            if last_fill[s] is None:
                continue
            f = last_fill[s] // K
            check(f <= phase[s] <= f + 1, "drain's parity would alias")
            if inflight[s] is not None:
                check(inflight[s] == last_fill[s], "the drain waits for a fill other than the one in flight")
                land(s)
    check(all(x is None for x in inflight), "the block exits with a fill in flight")
    for w in range(n_warps):
        if not failed[w]:
            check(seen[w] == list(range(nb)), "a warp missed or repeated a batch")
    if not any(failed):
        check(fills == nb, "fill count")
    return any(failed)


@pytest.mark.parametrize("n_warps,K", [(4, 2), (4, 3), (2, 2), (8, 4), (4, 1), (1, 2)])
def test_ring_protocol_under_random_interleavings(n_warps, K):
    for seed in range(200):
        for nb in (0, 1, 2, 3, 5, 9):
            assert not run_ring(n_warps, K, nb, seed * 31 + nb)


@pytest.mark.parametrize("n_warps,K", [(4, 2), (4, 3), (2, 2), (8, 4), (1, 2)])
def test_ring_failure_path_leaves_no_fill_in_flight(n_warps, K):
    """Copies that stall (waits that run out before the copies land): every
    interleaving ends, no buffer ever has two fills in flight, and after the
    drain no fill is in flight when the block exits."""
    failures = 0
    for seed in range(300):
        for nb in (1, 2, 3, 5, 9):
            failures += run_ring(n_warps, K, nb, seed * 17 + nb, timeouts=0.02, stall=0.2)
    assert failures > 100  # the failure path was exercised


def test_model_catches_a_refill_before_every_release():
    """The same model with the refill issued by the first warp to release a
    buffer instead of the last: some interleaving must break it."""
    caught = 0
    for seed in range(200):
        try:
            run_ring(4, 2, 9, seed, refill_by_first=True)
        except ProtocolError:
            caught += 1
    assert caught > 0


def test_model_catches_an_exit_without_the_drain():
    """Without the drain some interleaving exits while a fill is in flight."""
    caught = 0
    for seed in range(300):
        try:
            run_ring(4, 2, 9, seed, timeouts=0.02, stall=0.2, drain=False)
        except ProtocolError as e:
            assert "in flight" in str(e)
            caught += 1
    assert caught > 0


def test_model_catches_a_failed_warp_that_keeps_releasing():
    """A warp that keeps counting releases after its wait ran out lets a round
    complete while another warp still reads the buffer or its previous fill is
    in flight."""
    caught = 0
    for seed in range(300):
        try:
            run_ring(4, 2, 9, seed, timeouts=0.02, stall=0.2, failed_keeps_releasing=True)
        except ProtocolError:
            caught += 1
    assert caught > 0
