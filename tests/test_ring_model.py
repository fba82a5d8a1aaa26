"""A host model of the reverse pass's staging ring, run under random
interleavings of its warps.

The kernel stages a tile's list in batches through K buffers.  Each warp, for
every batch u in order, waits for buffer u % K to hold batch u (the phase of
its mbarrier with parity (u / K) & 1), reads it, and releases it by adding one
to the buffer's count; the warp whose addition completes the count resets it
and refills the buffer with batch u + K (if there is one), and the refill's
arrival completes the next phase.  The model checks the protocol's claims: a
buffer is never refilled while a warp still has to read its batch, every warp
reads every batch once and in order, a wait never sees a phase of another fill
(parity aliasing), and no interleaving deadlocks.
"""
import random

import pytest


def run_ring(n_warps, K, nb, seed, refill_by_first=False):
    rng = random.Random(seed)
    content = [None] * K          # batch held by each buffer
    phase = [0] * K               # completed phases of each buffer's barrier
    released = [0] * K            # release count of each buffer
    reading = [set() for _ in range(K)]
    seen = [[] for _ in range(n_warps)]
    fills = 0

    def fill(s, batch):
        nonlocal fills
        assert not reading[s], "refill while a warp still reads the buffer"
        content[s] = batch
        phase[s] += 1
        fills += 1

    for u in range(min(K, nb)):   # the warps' initial fills
        fill(u, u)
    # per warp: next batch and its step (0 wait, 1 read, 2 release)
    state = [[0, 0] for _ in range(n_warps)]
    while True:
        runnable = []
        for w, (u, step) in enumerate(state):
            if u >= nb:
                continue
            s = u % K
            if step == 0:
                # the hardware test: try_wait.parity(p) succeeds when the parity
                # of the completed-phase count differs from p, which is right
                # only while that count is u // K or u // K + 1
                assert u // K <= phase[s] <= u // K + 1, "parity would alias"
                if (phase[s] & 1) != ((u // K) & 1):
                    runnable.append(w)
            else:
                runnable.append(w)
        if not runnable:
            break
        w = rng.choice(runnable)
        u, step = state[w]
        s = u % K
        if step == 0:
            # the wait succeeded: the phase it waited for is the current fill
            assert phase[s] == u // K + 1, "wait satisfied by another fill's phase"
            reading[s].add(w)
            state[w][1] = 1
        elif step == 1:
            assert content[s] == u
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
                if u + K < nb:
                    fill(s, u + K)
            state[w] = [u + 1, 0]
    assert all(u >= nb for u, _ in state), "deadlock"
    assert all(seq == list(range(nb)) for seq in seen)
    assert fills == nb


@pytest.mark.parametrize("n_warps,K", [(4, 2), (4, 3), (2, 2), (8, 4), (4, 1), (1, 2)])
def test_ring_protocol_under_random_interleavings(n_warps, K):
    for seed in range(200):
        for nb in (0, 1, 2, 3, 5, 9):
            run_ring(n_warps, K, nb, seed * 31 + nb)


def test_model_catches_a_refill_before_every_release():
    """The same model with the refill issued by the first warp to release a
    buffer instead of the last: some interleaving must break it."""
    caught = 0
    for seed in range(200):
        try:
            run_ring(4, 2, 9, seed, refill_by_first=True)
        except AssertionError:
            caught += 1
    assert caught > 0
