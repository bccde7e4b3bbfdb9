"""Host-side models of two pieces of the BF16-mixed patch passes
(csrc/gram_tc.cu, csrc/rotate_tc.cu, csrc/patch_gather.cuh), run on the CPU.

1. The column sums of pg::warp_colsum8: 32 lanes each hold 8 column values;
   three reduce-scatter shuffle steps, two butterfly steps and eight
   broadcasts must leave every lane with the 8 column sums, bit-identical
   across lanes (every caller then centres with identical means).  The model
   repeats the kernel's lane arithmetic in float32.

2. The gather ring: S stages; each producer thread commits one cp.async
   group per chunk (the first S - 1 before the loop); in iteration ci it waits
   until all but its S - 2 most recent groups have completed
   (cp.async.wait_group S - 2; groups may land in any order), passes the CTA
   barrier,
   issues chunk ci + S - 1 into stage (ci + S - 1) % S and then reads chunk
   ci from stage ci % S - including units other threads copied.  Under random
   schedules and random copy completion the model checks that a read always
   finds its chunk landed and not yet overwritten, and that the two mistakes
   the kernel avoids (issuing before the barrier, waiting one group too few)
   are caught."""
import random

import numpy as np
import pytest


# ---------------------------------------------------------------- column sums
def _colsum8(S, swap_round_b=False):
    """Lane arithmetic of warp_colsum8 in float32; S is a (32, 8) float32 array."""
    S = S.astype(np.float32)
    t = np.zeros((32, 4), np.float32)
    for l in range(32):
        p = l ^ 16
        for i in range(4):
            keep = S[l, i + 4] if l & 16 else S[l, i]
            recv = S[p, i] if p & 16 else S[p, i + 4]  # what the partner sends
            t[l, i] = np.float32(keep + recv)
    u = np.zeros((32, 2), np.float32)
    for l in range(32):
        p = l ^ 8
        for i in range(2):
            b3 = bool(l & 8) != swap_round_b
            keep = t[l, i + 2] if b3 else t[l, i]
            recv = t[p, i] if p & 8 else t[p, i + 2]
            u[l, i] = np.float32(keep + recv)
    c = np.zeros(32, np.float32)
    for l in range(32):
        p = l ^ 4
        keep = u[l, 1] if l & 4 else u[l, 0]
        recv = u[p, 0] if p & 4 else u[p, 1]
        c[l] = np.float32(keep + recv)
    c = np.array([np.float32(c[l] + c[l ^ 1]) for l in range(32)], np.float32)
    c = np.array([np.float32(c[l] + c[l ^ 2]) for l in range(32)], np.float32)
    src = [((e & 4) << 2) | ((e & 2) << 2) | ((e & 1) << 2) for e in range(8)]
    return np.array([[c[src[e]] for e in range(8)] for _ in range(32)], np.float32)


@pytest.mark.parametrize("seed", range(5))
def test_colsum8_sums_every_column_on_every_lane(seed):
    rng = np.random.default_rng(seed)
    S = rng.standard_normal((32, 8)).astype(np.float32) * np.float32(10.0) ** rng.integers(-3, 4, (32, 8))
    out = _colsum8(S)
    exact = S.astype(np.float64).sum(axis=0)
    scale = np.abs(S.astype(np.float64)).sum(axis=0)
    # 31 float32 additions: error below 31 u of the absolute sum
    assert np.all(np.abs(out[0] - exact) <= 31 * 2.0 ** -24 * scale + 1e-30)
    assert np.array_equal(out, np.broadcast_to(out[0], out.shape))  # identical on every lane


def test_colsum8_model_catches_a_swapped_step():
    S = np.random.default_rng(9).standard_normal((32, 8)).astype(np.float32)
    exact = S.astype(np.float64).sum(axis=0)
    wrong = _colsum8(S, swap_round_b=True)
    assert not np.allclose(wrong[0], exact, rtol=1e-5, atol=1e-5)


# ---------------------------------------------------------------- gather ring
class _Violation(Exception):
    pass


def _run_ring(S, nchunks, nthreads, seed, issue_before_barrier=False, wait_pending=None):
    """Random schedule of the ring protocol; raises _Violation on a bad read or reuse."""
    rng = random.Random(seed)
    wait_pending = S - 2 if wait_pending is None else wait_pending
    # stage contents per (stage, owner thread): the chunk whose copy has landed
    content = {}
    pending = [[] for _ in range(nthreads)]  # per thread: its pending groups: [(commit index, chunk or None, stage)]
    committed = [0] * nthreads
    reads_done = [-1] * nthreads             # last chunk each thread has finished reading
    # per-thread program
    prog = []
    for _ in range(nthreads):
        steps = [("issue", j) for j in range(S - 1)]
        for ci in range(nchunks):
            if issue_before_barrier:
                steps += [("issue", ci + S - 1), ("wait", ci), ("barrier", ci), ("read", ci)]
            else:
                steps += [("wait", ci), ("barrier", ci), ("issue", ci + S - 1), ("read", ci)]
        prog.append(steps)
    pc = [0] * nthreads
    at_barrier = set()

    def land(t, g):
        _, chunk, stage = pending[t][g]
        if chunk is not None:
            content[(stage, t)] = chunk
        pending[t].pop(g)

    while any(pc[t] < len(prog[t]) for t in range(nthreads)):
        # random asynchronous completions
        for t in range(nthreads):
            if pending[t] and rng.random() < 0.3:
                land(t, rng.randrange(len(pending[t])))
        runnable = [t for t in range(nthreads) if pc[t] < len(prog[t]) and t not in at_barrier]
        if not runnable:  # everyone at the barrier: release it
            at_barrier.clear()
            for t in range(nthreads):
                pc[t] += 1
            continue
        t = rng.choice(runnable)
        op, ci = prog[t][pc[t]]
        if op == "issue":
            if ci < nchunks:
                stage = ci % S
                prev = ci - S  # the stage's previous chunk
                for o in range(nthreads):
                    if prev >= 0 and reads_done[o] < prev:
                        raise _Violation(f"thread {t} overwrites stage {stage} (chunk {prev}) before thread {o} read it")
                pending[t].append((committed[t], ci, stage))
            else:
                pending[t].append((committed[t], None, None))  # an empty group
            committed[t] += 1
            pc[t] += 1
        elif op == "wait":
            # cp.async.wait_group n: every group but the n most recently
            # committed has completed (groups may land in any order)
            while pending[t] and pending[t][0][0] < committed[t] - wait_pending:
                land(t, 0)
            pc[t] += 1
        elif op == "barrier":
            at_barrier.add(t)
        elif op == "read":
            stage = ci % S
            for o in range(nthreads):  # every thread reads units any thread copied
                if content.get((stage, o)) != ci:
                    raise _Violation(f"thread {t} reads chunk {ci} from stage {stage}: "
                                     f"thread {o}'s copy holds {content.get((stage, o))}")
            reads_done[t] = ci
            pc[t] += 1


@pytest.mark.parametrize("S", [2, 3, 5, 6])
def test_gather_ring_protocol(S):
    for nchunks in (1, 2, S - 1, S, S + 1, 17):
        for seed in range(20):
            _run_ring(S, nchunks, nthreads=4, seed=seed)


def test_gather_ring_model_catches_issue_before_barrier():
    caught = False
    for seed in range(200):
        try:
            _run_ring(5, 12, nthreads=4, seed=seed, issue_before_barrier=True, wait_pending=4)
        except _Violation:
            caught = True
            break
    assert caught


def test_gather_ring_model_catches_short_wait():
    caught = False
    for seed in range(200):
        try:
            _run_ring(5, 12, nthreads=4, seed=seed, wait_pending=4)
        except _Violation:
            caught = True
            break
    assert caught
