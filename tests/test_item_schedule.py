"""CPU model of the Wilson kernel's staging ring and its dynamic item schedule.

Each CTA of the persistent Wilson kernel works through items, where an item is one chain of loop
blocks for one group of tiles. Each CTA stages the items' loop blocks, chunk by chunk, through a
ring of `stages` shared-memory slots. Every slot has two mbarriers:
- a `full` barrier: one arrival plus the copy's bytes;
- an `empty` barrier: one arrival per warp.

Thread 0 (lane 0 of warp 0) is also the producer.
- Its first `stages` chunks are issued before the warps start.
- After that it refills a slot once every warp has released it.
- When it starts an item it takes a new one. The CTA's first item is its own index; later ones are
  the grid size plus a claim from the launch's counter (or the previous item plus the grid size
  when there is no counter).
- Past the last item it writes the sentinel -1 to the slot's item word and completes the slot's
  full barrier without a copy. Every warp's wait then ends.

A wait is bounded. When a wait runs out, the warp sets the error flag and the CTA's abort word and
returns. Thread 0 then waits for its own copies still in flight before the CTA exits.

This model runs that protocol on Python generators, with one generator per warp and one per copy in
flight. A random scheduler drives them, with random item costs (heavy-tailed across items), random
chunk costs and random copy latencies. It checks:
- every item of the launch is walked exactly once, by every warp, through each block and chunk of
  its chain in order;
- each chunk a warp reads is the one it expects, and stays unchanged until the warp releases it;
- no parity test is ambiguous: a waiter's barrier is never more than one phase past the phase it
  waits for;
- with no fault, every wait ends without running out, and no copy is in flight when a CTA exits;
- with waits that give up early, every warp still ends, the error flag is set, and no copy is in
  flight when a CTA exits;
- mistakes planted in the model's protocol are caught by these checks.
"""
import random

import pytest

CHUNK_BYTES = 64 * 512      # a 64-row chunk of 32 float4 lanes
TICK = ("tick",)


class ProtocolError(AssertionError):
    pass


class Barrier:
    """An mbarrier: an arrival count, a transaction byte count and a phase."""

    def __init__(self, count):
        self.count = count
        self.pending = count
        self.tx = 0
        self.phase = 0          # phases completed so far

    def _complete(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def arrive(self, expect_tx=0):
        if self.pending <= 0:
            raise ProtocolError("arrival on a barrier with no pending arrival")
        self.tx += expect_tx
        self.pending -= 1
        self._complete()

    def complete_tx(self, nbytes):
        self.tx -= nbytes
        if self.tx < 0:
            raise ProtocolError("more bytes landed than the barrier expected")
        self._complete()

    def test(self, use):
        """try_wait.parity with parity `use & 1`, for the `use`-th phase of this barrier.

        The parity test can tell phase `use` apart from phase `use + 1` only; a barrier that
        has run further ahead (or not yet reached `use`) makes the answer wrong."""
        if self.phase not in (use, use + 1):
            raise ProtocolError(f"phase {self.phase} is ambiguous for a wait on phase {use}")
        return (self.phase & 1) != (use & 1)


class Cta:
    def __init__(self, idx, warps, stages):
        self.idx = idx
        self.full = [Barrier(1) for _ in range(stages)]
        self.empty = [Barrier(warps) for _ in range(stages)]
        self.ring = [None] * stages        # what the slot holds: (item, block, chunk)
        self.chunk_item = [None] * stages  # the item word thread 0 writes with each chunk
        self.issued = 0
        self.blk = 0
        self.chunk = 0
        self.item = 0
        self.started = False
        self.done = False
        self.abort = False
        self.in_flight = 0
        self.live = warps


class Launch:
    """One launch of the kernel: `grid` CTAs of `warps` warps over the items of
    ceil(n_blocks / chain) chains x n_tg tile groups."""

    def __init__(self, seed, grid, warps, stages, cpb, chain, n_blocks, n_tg, dynamic=True,
                 give_up=0.0, bug=None, max_latency=6):
        self.rng = random.Random(seed)
        self.grid, self.warps, self.stages, self.cpb = grid, warps, stages, cpb
        self.chain, self.n_blocks, self.n_tg = chain, n_blocks, n_tg
        self.n_items = (-(-n_blocks // chain)) * n_tg
        self.dynamic, self.give_up, self.bug = dynamic, give_up, bug
        self.max_latency = max_latency
        self.counter = 0
        self.flag = None
        self.timeouts = 0
        self.walked = {}
        self.item_cta = {}
        # heavy-tailed item costs: some items are many times the typical one
        self.cost = [1 + int(self.rng.paretovariate(1.2)) % 12 for _ in range(self.n_items)]
        self.agents = []
        self.ctas = [Cta(i, warps, stages) for i in range(grid)]

    # -- the producer (thread 0)
    def blocks_in_item(self, item):
        b0 = (item // self.n_tg) * self.chain
        return min(b0 + self.chain, self.n_blocks) - b0

    def issue_next(self, cta, slot):
        if cta.blk == 0 and cta.chunk == 0:
            if not cta.started:
                item = cta.idx
                cta.started = True
            elif self.dynamic:
                item = self.counter + (0 if self.bug == "claim_without_grid" else self.grid)
                self.counter += 1                      # atomicAdd returns the old value
            else:
                item = cta.item + self.grid
            cta.item = item
            if item >= self.n_items:
                cta.chunk_item[slot] = -1
                cta.done = True
                if self.bug != "sentinel_without_arrive":
                    cta.full[slot].arrive()
                return
        cta.chunk_item[slot] = cta.item
        b = (cta.item // self.n_tg) * self.chain + cta.blk
        cta.full[slot].arrive(expect_tx=CHUNK_BYTES)
        cta.in_flight += 1
        self.spawn(self.copy(cta, slot, (cta.item, b, cta.chunk)))
        cta.issued += 1
        cta.chunk += 1
        if cta.chunk == self.cpb:
            cta.chunk = 0
            cta.blk += 1
            if cta.blk == self.blocks_in_item(cta.item):
                cta.blk = 0

    def copy(self, cta, slot, content):
        for _ in range(self.rng.randint(0, self.max_latency)):
            yield TICK
        cta.ring[slot] = content
        cta.in_flight -= 1
        cta.full[slot].complete_tx(CHUNK_BYTES)

    # -- a warp
    def warp(self, cta, w):
        S = self.stages
        kc = 0
        ok = True
        while ok:
            slot, use = kc % S, kc // S
            if not (yield ("wait", cta.full[slot], use, True)):
                self.flag = "timeout_full"
                cta.abort = True
                ok = False
                break
            item = cta.chunk_item[slot]
            if item < 0:
                break
            ok, kc = yield from self.run_item(cta, w, item, kc)
        if not ok and w == 0:
            # thread 0: let the copies it issued land before the CTA's shared memory goes away
            for q in range(kc, cta.issued):
                yield ("wait", cta.full[q % S], q // S, False)
        cta.live -= 1
        if cta.live == 0 and cta.in_flight:
            raise ProtocolError(f"CTA {cta.idx} exits with {cta.in_flight} copies in flight")

    def run_item(self, cta, w, item, kc):
        S = self.stages
        b0 = (item // self.n_tg) * self.chain
        b1 = min(b0 + self.chain, self.n_blocks)
        if w == 0:
            if item in self.item_cta:
                raise ProtocolError(f"item {item} taken by CTAs {self.item_cta[item]} and {cta.idx}")
            self.item_cta[item] = cta.idx
        for b in range(b0, b1):
            for ch in range(self.cpb):
                slot, use = kc % S, kc // S
                if not (yield ("wait", cta.full[slot], use, True)):
                    self.flag = "timeout_full"
                    cta.abort = True
                    return False, kc
                want = (item, b, ch)
                if cta.ring[slot] != want:
                    raise ProtocolError(f"warp {w} of CTA {cta.idx} wants {want}, "
                                        f"slot {slot} holds {cta.ring[slot]}")
                for _ in range(self.cost[item] * self.rng.randint(1, 3)):
                    yield TICK
                if cta.ring[slot] != want:
                    raise ProtocolError(f"slot {slot} of CTA {cta.idx} overwritten while "
                                        f"warp {w} walks it")
                self.walked.setdefault((item, w), []).append((b, ch))
                cta.empty[slot].arrive()
                if w == 0 and not cta.done:
                    if self.bug == "refill_without_empty_wait":
                        self.issue_next(cta, slot)
                    elif not (yield ("wait", cta.empty[slot], use, True)):
                        self.flag = "timeout_empty"
                        cta.abort = True
                    else:
                        self.issue_next(cta, slot)
                kc += 1
                if cta.abort:
                    return False, kc
        return True, kc

    # -- the scheduler
    def spawn(self, gen):
        self.agents.append([gen, None, True])

    def _advance(self, agent, value):
        gen = agent[0]
        try:
            agent[1] = gen.send(value) if agent[2] is False else next(gen)
            agent[2] = False
        except StopIteration:
            agent[1] = "finished"

    def run(self, max_steps=2_000_000):
        # thread 0's prologue, then __syncthreads, then the warps
        for cta in self.ctas:
            for s in range(self.stages):
                if cta.done:
                    break
                self.issue_next(cta, s)
            for w in range(self.warps):
                self.spawn(self.warp(cta, w))
        for a in self.agents:
            if a[2]:
                self._advance(a, None)
        steps = 0
        while True:
            self.agents = [a for a in self.agents if a[1] != "finished"]
            for a in self.agents:                    # agents spawned since the last step
                if a[2]:
                    self._advance(a, None)
            self.agents = [a for a in self.agents if a[1] != "finished"]
            if not self.agents:
                return
            steps += 1
            if steps > max_steps:
                raise ProtocolError("the model did not finish")
            ready, blocked = [], []
            for a in self.agents:
                req = a[1]
                if req[0] == "tick" or req[1].test(req[2]):
                    ready.append(a)
                else:
                    blocked.append(a)
            # a bounded wait may run out while its phase is still pending
            quitters = [a for a in blocked if a[1][3]]
            if self.give_up and quitters and self.rng.random() < self.give_up:
                self.timeouts += 1
                self._advance(self.rng.choice(quitters), False)
                continue
            if ready:
                self._advance(self.rng.choice(ready), True)
                continue
            # nothing can move: the bounded waits run out, one at a time
            if not quitters:
                raise ProtocolError("a wait with no limit can never end")
            self.timeouts += 1
            self._advance(self.rng.choice(quitters), False)

    # -- the checks of a fault-free launch
    def check_complete(self):
        if self.timeouts or self.flag:
            raise ProtocolError(f"{self.timeouts} waits ran out (flag {self.flag})")
        for item in range(self.n_items):
            b0 = (item // self.n_tg) * self.chain
            want = [(b, ch) for b in range(b0, min(b0 + self.chain, self.n_blocks))
                    for ch in range(self.cpb)]
            for w in range(self.warps):
                if self.walked.get((item, w)) != want:
                    raise ProtocolError(f"item {item}, warp {w}: walked "
                                        f"{self.walked.get((item, w))}, want {want}")
        extra = set(i for i, _ in self.walked) - set(range(self.n_items))
        if extra:
            raise ProtocolError(f"items past the end walked: {sorted(extra)}")
        for cta in self.ctas:
            if cta.in_flight:
                raise ProtocolError("copy in flight after the launch")


def _random_shape(rng):
    n_blocks = rng.randint(1, 9)
    chain = rng.randint(1, 4)
    n_tg = rng.randint(1, 3)
    n_items = (-(-n_blocks // chain)) * n_tg
    # the host launches min(CTAs per SM x SMs, items); a wider grid is also safe
    grid = rng.choice([rng.randint(1, n_items), rng.randint(1, n_items + 3)])
    return dict(grid=grid, warps=rng.randint(1, 4), stages=rng.randint(1, 8),
                cpb=rng.randint(1, 3), chain=chain, n_blocks=n_blocks, n_tg=n_tg)


@pytest.mark.parametrize("dynamic", [True, False])
def test_every_item_walked_once(dynamic):
    rng = random.Random(7 if dynamic else 8)
    claimed = 0
    for trial in range(400):
        shape = _random_shape(rng)
        L = Launch(seed=1000 * trial + 1, dynamic=dynamic, **shape)
        L.run()
        L.check_complete()
        claimed += L.counter > L.grid     # claims past the first wave
    assert claimed > 100 if dynamic else claimed == 0


def test_dynamic_schedule_balances_skewed_items():
    """Every ninth item costs 40 times the rest. With the counter, CTAs that finish early take
    more of the remaining items. Without it, each CTA walks a fixed stride of items."""
    L = Launch(seed=3, grid=4, warps=2, stages=2, cpb=2, chain=1, n_blocks=24, n_tg=2)
    L.cost = [40 if i % 9 == 0 else 1 for i in range(L.n_items)]
    L.run()
    L.check_complete()
    per_cta = [sum(1 for c in L.item_cta.values() if c == i) for i in range(L.grid)]
    assert sum(per_cta) == L.n_items
    # CTA 0 starts on a dear item (0, 9, 18, ... are), so it takes fewer than its fixed share
    assert per_cta[0] < L.n_items // L.grid, per_cta
    S = Launch(seed=3, grid=4, warps=2, stages=2, cpb=2, chain=1, n_blocks=24, n_tg=2,
               dynamic=False)
    S.run()
    S.check_complete()
    assert all(S.item_cta[i] == i % 4 for i in range(S.n_items))


def test_waits_that_run_out_still_end():
    """Bounded waits that give up early (at random, while the awaited phase is still pending):
    every warp ends, the error flag is set, and thread 0's drain leaves no copy in flight."""
    rng = random.Random(11)
    flagged = 0
    for trial in range(150):
        shape = _random_shape(rng)
        L = Launch(seed=trial, give_up=0.02, **shape)
        L.run()                        # ProtocolError on a copy in flight at a CTA's exit
        if L.timeouts:
            assert L.flag is not None
            flagged += 1
        else:
            L.check_complete()
    assert flagged > 20


@pytest.mark.parametrize("bug,expect", [
    ("refill_without_empty_wait", "overwritten|holds|ambiguous|no pending arrival"),
    ("claim_without_grid", "taken by CTAs"),
    ("sentinel_without_arrive", "waits ran out|can never end"),
])
def test_planted_mistakes_are_caught(bug, expect):
    import re
    rng = random.Random(21)
    caught = 0
    for trial in range(60):
        shape = _random_shape(rng)
        shape.update(warps=max(shape["warps"], 2), grid=max(2, min(shape["grid"], 4)))
        L = Launch(seed=trial, bug=bug, **shape)
        try:
            L.run()
            L.check_complete()
        except ProtocolError as e:
            assert re.search(expect, str(e)), str(e)
            caught += 1
    assert caught >= 10, caught
