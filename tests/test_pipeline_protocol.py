"""Race check of the image-fed sketch kernel's mbarrier protocol, on the host.

The kernel's roles (tile loader, B loader, two producer groups of warps, the
MMA thread, drain warps) meet only through mbarriers that are waited on by
phase parity.  A parity wait passes when the barrier's current phase has the
other parity, so a waiter whose phase is still one behind passes early: the
failure an odd slot count causes with two producer groups.  This module
models the protocol as the kernel's comments state it (rings of SF tile
slots, SB B slots, S A slots, NB chunk-indexed full/done barriers, two
accumulator sets alternating every DR = 4 chunks) and runs it under random
interleavings of the warps, checking that every wait passes only once the
phase it stands for has completed and that every role finishes.  A model
with an odd tile-slot count must show the early pass."""
import random

import pytest


class Bar:
    """An mbarrier: `count` arrivals complete a phase."""

    def __init__(self, name, count):
        self.name, self.count = name, count
        self.done = 0        # completed phases
        self.pending = 0     # arrivals in the current phase

    def arrive(self):
        self.pending += 1
        assert self.pending <= self.count, f"{self.name}: more arrivals than its count"
        if self.pending == self.count:
            self.pending = 0
            self.done += 1

    def parity_passes(self, parity):
        # try_wait.parity: true iff the current (incomplete) phase has the
        # other parity, i.e. the last completed phase has parity `parity`
        return (self.done & 1) != parity


def model(nch, SF, SB, S, NB=8, NWARP=2, NDRAIN=2, DR=4, seed=0):
    """Runs the protocol for one CTA of `nch` chunks under a random schedule.
    Returns a list of early passes (wait name, intended phase, completed
    phases at the pass); raises on deadlock."""
    rnd = random.Random(seed)
    fullF = [Bar(f"fullF{i}", 1) for i in range(SF)]
    emptyF = [Bar(f"emptyF{i}", NWARP) for i in range(SF)]
    full = [Bar(f"full{j}", NWARP + 1) for j in range(NB)]
    done = [Bar(f"done{j}", 1) for j in range(NB)]
    accF = [Bar(f"accF{b}", 1) for b in range(2)]
    accE = [Bar(f"accE{b}", NDRAIN) for b in range(2)]
    early = []
    pending_async = []   # (bar) arrivals of copies and MMA commits, landing later

    def wait(bar, phase):
        # blocks until the parity wait passes; records a pass before `phase` completed
        while not bar.parity_passes(phase & 1):
            yield
        if bar.done < phase + 1:
            early.append((bar.name, phase, bar.done))

    def tile_loader():
        for c in range(nch):
            if c >= SF:
                yield from wait(emptyF[c % SF], c // SF - 1)
            pending_async.append(fullF[c % SF])

    def b_loader():
        for c in range(nch):
            if c >= SB:
                j = (c - SB) % NB
                yield from wait(done[j], (c - SB) // NB)
            pending_async.append(full[c % NB])   # arrive.expect_tx + the copy's bytes: one arrival

    def producer_warp(g):
        for c in range(g, nch, 2):
            yield from wait(fullF[c % SF], c // SF)
            if c >= S:
                yield from wait(done[(c - S) % NB], (c - S) // NB)
            yield
            emptyF[c % SF].arrive()
            yield
            full[c % NB].arrive()

    def mma():
        for c in range(nch):
            if c % DR == 0 and c >= 2 * DR:
                g = c // DR
                yield from wait(accE[g & 1], (g - 2) // 2)
            yield from wait(full[c % NB], c // NB)
            pending_async.append(done[c % NB])
            if c % DR == DR - 1 or c == nch - 1:
                pending_async.append(accF[(c // DR) & 1])
            yield

    def drain_warp():
        for g in range((nch + DR - 1) // DR):
            yield from wait(accF[g & 1], g // 2)
            yield
            accE[g & 1].arrive()

    roles = [tile_loader(), b_loader(), mma()]
    roles += [producer_warp(g) for g in (0, 1) for _ in range(NWARP)]
    roles += [drain_warp() for _ in range(NDRAIN)]
    live = list(roles)
    stall = 0
    while live:
        if pending_async and rnd.random() < 0.3:
            # asynchronous completions land in order per barrier, in any order across them
            pending_async.pop(rnd.randrange(len(pending_async)) if rnd.random() < 0.5 else 0).arrive()
            stall = 0
            continue
        r = rnd.choice(live)
        before = (tuple(b.done for b in fullF + emptyF + full + done + accF + accE), len(pending_async))
        try:
            next(r)
        except StopIteration:
            live.remove(r)
            stall = 0
            continue
        after = (tuple(b.done for b in fullF + emptyF + full + done + accF + accE), len(pending_async))
        stall = 0 if after != before else stall + 1
        if stall > 200000 and not pending_async:
            raise RuntimeError("deadlock")
    while pending_async:
        pending_async.pop(0).arrive()
    return early


@pytest.mark.parametrize("SF,SB,S", [(8, 8, 2), (4, 4, 4), (8, 4, 2), (4, 8, 4)])
@pytest.mark.parametrize("nch", [1, 7, 8, 9, 37])
def test_protocol_has_no_early_pass(SF, SB, S, nch):
    """The kernel's configurations (A in tensor memory: 8 tile, 8 B, 2 A
    slots; A in shared memory: 4, 4, 4) and their mixes, ragged chunk counts
    around the unrolled period of 8, many random schedules."""
    for seed in range(25):
        assert model(nch, SF, SB, S, seed=seed) == []


def test_odd_tile_slot_count_passes_early():
    """With 3 tile slots the two producer groups take turns on a slot; some
    schedule lets a group pass its fullF wait while the barrier is still one
    phase behind."""
    found = any(model(24, 3, 8, 2, seed=seed) for seed in range(200))
    assert found
