"""The barrier protocol of the persistent slice GEMM (tc_gemm.cuh,
gemm_sliced_persistent), model-checked on the CPU.

Three roles share mbarriers: the TMA thread fills shared-memory stages
(full[s] completes when the copies land), the MMA thread consumes them
(commits free a stage, empty[s], and hand a finished accumulator set to the
epilogue, tfull[b]), and four epilogue warps release an accumulator set
(tempty[b], four arrivals).  A wait names the phase it needs by its parity,
so it is only correct if the barrier is never two or more phases past the
phase the waiter needs when it looks.  The model runs the roles in random
interleavings, with copies and MMA commits completing after random delays
(commits in issue order, as tcgen05 operations complete), using the same
stage, buffer and parity arithmetic as the kernel, and checks that every
role finishes, that no wait ever sees an aliased phase, that a stage is
refilled only after the MMAs that read it completed, and that an
accumulator set is overwritten only after all four epilogue warps read it."""
import random

import pytest


class Barrier:
    def __init__(self, count):
        self.count, self.pending, self.done = count, count, 0    # done = completed phases

    def arrive(self):
        self.pending -= 1
        assert self.pending >= 0
        if self.pending == 0:
            self.done += 1
            self.pending = self.count


def wait_ready(bar, phase):
    """True once the given phase has completed; fails on an aliased phase
    (the barrier two or more phases past it, which a parity wait would take
    for the phase still to come)."""
    assert bar.done - phase <= 1, (bar.done, phase)
    return bar.done > phase


def run_cta(ntiles, nkb, stages, rng, mutant=None):
    full = [Barrier(1) for _ in range(stages)]         # the expect_tx arrival; completes when the copies land
    empty = [Barrier(1) for _ in range(stages)]
    tfull = [Barrier(1) for _ in range(2)]
    tempty = [Barrier(4) for _ in range(2)]
    copies = []                                        # stages whose copies are in flight
    commits = []                                       # MMA commits in issue order
    consumed = set()                                   # K blocks whose MMAs have completed
    mma_started, reads_done = set(), {}

    def commit(bar, kblock=None):
        def fire():
            if kblock is not None:
                consumed.add(kblock)
            bar.arrive()
        commits.append(fire)

    def producer():
        it = 0
        for _tile in range(ntiles):
            for _kb in range(nkb):
                s = it % stages
                if it >= stages and mutant != "no_empty_wait":
                    while not wait_ready(empty[s], it // stages - 1):
                        yield
                    assert it - stages in consumed     # the stage's previous MMAs are done
                copies.append(s)
                it += 1
                yield

    def mma():
        it = 0
        for tl in range(ntiles):
            buf = tl & 1
            if tl >= 2 and mutant != "no_tempty_wait":
                while not wait_ready(tempty[buf], (tl >> 1) - 1):
                    yield
                assert reads_done.get(tl - 2) == 4     # every epilogue warp has read the set
            mma_started.add(tl)
            for _kb in range(nkb):
                s = it % stages
                while not wait_ready(full[s], it // stages):
                    yield
                commit(empty[s], it)
                it += 1
                yield
            commit(tfull[buf])

    def epilogue():
        for tl in range(ntiles):
            buf = tl & 1
            while not wait_ready(tfull[buf], tl >> 1):
                yield
            assert tl + 2 not in mma_started           # the set is not being overwritten
            yield                                      # reads the accumulators
            assert tl + 2 not in mma_started
            reads_done[tl] = reads_done.get(tl, 0) + 1
            tempty[buf].arrive()

    roles = [producer(), mma()] + [epilogue() for _ in range(4)]
    live = list(range(len(roles)))
    for _step in range(10 ** 6):
        if not live and not copies and not commits:
            assert reads_done == {tl: 4 for tl in range(ntiles)}
            return
        r = rng.random()
        if copies and r < 0.15:
            full[copies.pop(rng.randrange(len(copies)))].arrive()   # at most one in flight per stage
            continue
        if commits and r < 0.3:
            commits.pop(0)()                           # the oldest outstanding commit fires
            continue
        if live:
            k = rng.choice(live)
            try:
                next(roles[k])
            except StopIteration:
                live.remove(k)
    raise AssertionError("the roles did not finish (deadlock)")


@pytest.mark.parametrize("ntiles,nkb,stages", [(1, 1, 2), (1, 16, 2), (2, 3, 2), (3, 1, 2), (7, 16, 2),
                                               (6, 2, 2), (5, 5, 3), (7, 4, 4)])
def test_persistent_gemm_protocol(ntiles, nkb, stages):
    rng = random.Random(1000 * ntiles + 10 * nkb + stages)
    for _ in range(40):
        run_cta(ntiles, nkb, stages, rng)


@pytest.mark.parametrize("mutant", ["no_tempty_wait", "no_empty_wait"])
def test_model_catches_a_dropped_wait(mutant):
    """A protocol with one of its waits taken out fails the model's checks."""
    rng = random.Random(5)
    with pytest.raises(AssertionError):
        for _ in range(200):
            run_cta(6, 4, 2, rng, mutant)


def test_model_detects_an_aliased_wait():
    """The check itself: a barrier two phases past the awaited phase fails."""
    b = Barrier(1)
    b.arrive()
    b.arrive()
    with pytest.raises(AssertionError):
        wait_ready(b, 0)
