"""A host-side model of the tensor-core moment kernel's warp-role protocol
(csrc/moments_tc.cu), run under random schedules on the CPU.

Roles and barriers as in the kernel: the producer fills two chunk buffers
(chunk_ready) and reuses one once the MMAs of its previous chunk completed
(chunk_done); the former warps take the slot groups of a pass in order, wait
for a group's previous use to be released (slot_empty), form it and arrive
(slot_full); the MMA thread waits for each group, its completion releases the
group, and a commit ends each chunk and each pass (pass_done); the formers
drain a pass and release the accumulators (d_free).  Waits test the parity of
a barrier's phase, as mbarrier try_wait.parity does.

The model checks, for the kernel's pass/tile arithmetic at several k and every
accepted slot count: no schedule deadlocks, a slot group is never formed while
the MMAs of its previous use are pending, and the producer never overwrites a
chunk buffer a former may still read.  It also checks that the layout the
kernel excludes - two former teams taking alternate groups of a single slot
pair - is caught (a team can read a barrier two phases old as free).  With a
wait of the MMA thread running out (an abort), tensor memory must be freed only
after the last MMA commit has completed: the model checks the kernel's final
wait (a commit to a barrier used only for it) and catches parity waits on
pass_done, which can name an already completed phase."""
import random

import pytest


class _Bar:
    def __init__(self, count):
        self.count, self.pending, self.phase = count, count, 0

    def arrive(self):
        self.pending -= 1
        if self.pending == 0:
            self.phase += 1
            self.pending = self.count

    def done(self, parity):  # the phase of this parity has completed
        return (self.phase & 1) != parity


class _Violation(Exception):
    pass


def _tiles(k):
    """Row-product tiles and accumulator columns per tile (moments_tc_rows, moments_tc_n)."""
    kb = (k + 7) // 8
    rows = max(kb * (kb + 1) // 2 * 64, k * (k + 1) // 2 + 2 * k)
    return (rows + 127) // 128, 16 if k <= 16 else (k + 15) // 16 * 16


def _simulate(k, nslots, seed, nchunks=3, group=2, teams=1, warps_per_team=8, abort_at=None,
              final_parity="fin"):
    """abort_at: the MMA thread's wait (counted from 0) that runs out, or None.
    final_parity: the MMA thread's last wait before TMEM is freed: "fin" (the
    kernel: a commit to a barrier used once, phase 0), or a parity wait on
    pass_done at the phase of the last commit issued ("issued") or at phase
    npass - 1 ("npass"); after an abort both parity waits can name a phase that
    completed earlier."""
    ntiles, nb = _tiles(k)
    tpp = min(ntiles, (512 - 32 * nslots) // nb)
    npass = (ntiles + tpp - 1) // tpp
    ngs = nslots // group
    nformers = teams * warps_per_team
    slot_full = [_Bar(warps_per_team) for _ in range(ngs)]
    slot_empty = [_Bar(1) for _ in range(ngs)]
    chunk_ready, chunk_done = [_Bar(1), _Bar(1)], [_Bar(1), _Bar(1)]
    pass_done, d_free = _Bar(1), _Bar(nformers)
    commits = []          # tcgen05.commit arrivals, completed later in order
    reading = {}          # former -> chunk whose operands it is reading
    aborted = [False]     # the CTA-wide abort flag: after it every work wait is skipped

    def producer():
        gc = 0
        for _ in range(npass):
            for _ in range(nchunks):
                b, use = gc & 1, gc >> 1
                if use >= 1:
                    while not chunk_done[b].done((use - 1) & 1) and not aborted[0]:
                        yield False
                if not aborted[0] and any(c is not None and c != gc and (c & 1) == b for c in reading.values()):
                    raise _Violation("chunk buffer overwritten while read")
                chunk_ready[b].arrive()
                gc += 1
                yield True

    def former(w):
        team = w // warps_per_team
        gs = gph = gq = gc = 0
        for ps in range(npass):
            nt = min(tpp, ntiles - ps * tpp)
            for _ in range(nchunks):
                b = gc & 1
                while not chunk_ready[b].done((gc >> 1) & 1) and not aborted[0]:
                    yield False
                for _t in range(0, nt, group):
                    if teams == 1 or (gq & 1) == team:
                        if gq >= ngs:
                            while not slot_empty[gs].done(gph ^ 1) and not aborted[0]:
                                yield False
                        if not aborted[0] and slot_empty[gs].phase < gq // ngs:
                            raise _Violation("slot group formed before its previous use was released")
                        reading[w] = gc
                        yield True
                        reading[w] = None
                        slot_full[gs].arrive()
                    gs += 1
                    if gs == ngs:
                        gs, gph = 0, gph ^ 1
                    gq += 1
                gc += 1
            while not pass_done.done(ps & 1) and not aborted[0]:
                yield False
            d_free.arrive()
            yield True

    def mma():
        gc = s = ph = 0
        nwait = 0
        npd = 0

        def runs_out():
            nonlocal nwait
            nwait += 1
            if abort_at is not None and nwait - 1 == abort_at:
                aborted[0] = True
            return aborted[0]

        for ps in range(npass):
            nt = min(tpp, ntiles - ps * tpp)
            if ps > 0:
                if not runs_out():
                    while not d_free.done((ps - 1) & 1) and not aborted[0]:
                        yield False
            for _ in range(nchunks):
                if aborted[0]:
                    break
                for _t in range(0, nt, group):
                    if runs_out():
                        break
                    while not slot_full[s].done(ph) and not aborted[0]:
                        yield False
                    if aborted[0]:
                        break
                    commits.append(slot_empty[s])
                    s += 1
                    if s == ngs:
                        s, ph = 0, ph ^ 1
                    yield True
                commits.append(chunk_done[gc & 1])  # issued after an abort too, as in the kernel
                gc += 1
            commits.append(pass_done)
            npd += 1
            if aborted[0]:
                break
        if final_parity == "fin":
            fin = _Bar(1)  # a barrier used once: its commit follows every MMA issued
            commits.append(fin)
            while not fin.done(0):
                yield False
        else:
            parity = (npd - 1) & 1 if final_parity == "issued" else (npass - 1) & 1
            while not pass_done.done(parity):
                yield False
        # TMEM is freed here: every commit (every MMA issued) must have completed
        if commits:
            raise _Violation("tensor memory freed while MMAs were pending")

    agents = [producer(), mma()] + [former(w) for w in range(nformers)]
    for w in range(nformers):
        reading[w] = None
    rng = random.Random(seed)
    idle = 0
    while agents:
        progressed = False
        rng.shuffle(agents)
        for a in list(agents):
            try:
                progressed |= next(a)
            except StopIteration:
                agents.remove(a)
                progressed = True
        if commits and rng.random() < 0.5:
            commits.pop(0).arrive()
            progressed = True
        idle = 0 if progressed or commits else idle + 1
        if idle > 3:
            raise _Violation("deadlock")


@pytest.mark.parametrize("k", [2, 10, 16, 17, 33, 64])
@pytest.mark.parametrize("nslots", [2, 4, 6, 8])
def test_protocol_is_deadlock_and_race_free(k, nslots):
    if 512 - 32 * nslots < _tiles(k)[1]:
        pytest.skip("the kernel rejects this slot count for k")
    for seed in range(4):
        _simulate(k, nslots, seed)


def test_model_catches_two_teams_on_one_slot_pair():
    with pytest.raises(_Violation):
        for seed in range(8):
            _simulate(64, 2, seed, teams=2)


@pytest.mark.parametrize("k,nslots", [(64, 8), (64, 4), (33, 2), (10, 4)])
def test_abort_frees_tensor_memory_only_after_the_last_commit(k, nslots):
    # a wait of the MMA thread runs out at a random point: it stops issuing,
    # commits the pass it is in, and waits for that last commit before the
    # CTA frees TMEM; the other roles skip their waits from then on
    rng = random.Random(k * 100 + nslots)
    for trial in range(40):
        _simulate(k, nslots, seed=trial, abort_at=rng.randrange(0, 60))


@pytest.mark.parametrize("rule", ["npass", "issued"])
def test_model_catches_parity_waits_on_pass_done(rule):
    # after an abort, a parity wait on pass_done can pass at once: at phase
    # npass - 1 it may name an earlier pass; at the last commit issued it may
    # name the previous one when the abort came at the wait between passes and
    # two commits are pending.  Either frees TMEM under running MMAs (k = 64
    # with 8 slots has npass = 5)
    with pytest.raises(_Violation):
        for trial in range(200):
            _simulate(64, 8, seed=trial, abort_at=trial % 40, final_parity=rule)
