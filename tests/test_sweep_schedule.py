"""Host-side checks of the FP32 preconditioner sweep schedule (no GPU).

The sweeps of a block-banded LU (Sec. 4.2, App. A) run as a table of tasks
built on the host (bfs_sweep_schedule): one chain for the one-ended LU, two
chains from either end plus the middle system for the two-ended ("twisted")
LU.  The GPU kernel spins on the tags of the vector slices a task multiplies,
so the table must name, for every block, the one task that writes that slice,
and the tasks must be able to run group by group in order without a cycle.
These tests check that, and that executing the table over factors stored in
the slot layout the factorisation writes solves the banded system.
"""
import numpy as np
import pytest

from paper_1709_08803_gb300 import bfs

CASES = [(M, h) for M in (3, 4, 5, 7, 8, 13, 61) for h in (0, 1, 2, 3) if h <= M - 1]


def _rows(tbl):
    out = []
    for r in tbl:
        nblk = int(r[2])
        out.append(dict(k=int(r[0]), out=int(r[1]), blocks=[(int(r[4 + p]), int(r[8 + p]), int(r[12 + p]))
                                                             for p in range(nblk)]))
    return out


def _simulate(M, tasks, ntask):
    """Run the groups in lockstep rounds; a task runs once every vector slice it
    reads has been written.  Returns the number of rounds (None on a cycle)."""
    groups = [list(range(ntask[0])), list(range(ntask[0], ntask[0] + ntask[1]))]
    done = set()
    ptr = [0, 0]
    rounds = 0
    while ptr[0] < len(groups[0]) or ptr[1] < len(groups[1]):
        ran = []
        for g in (0, 1):
            if ptr[g] < len(groups[g]):
                u = groups[g][ptr[g]]
                if all(uid in done for _, _, uid in tasks[u]["blocks"]):
                    ran.append(u)
                    ptr[g] += 1
        if not ran:
            return None
        done.update(ran)
        rounds += 1
    return rounds


@pytest.mark.parametrize("M,h", CASES)
@pytest.mark.parametrize("twisted", [0, 1])
def test_schedule_is_well_formed(M, h, twisted):
    tbl, ntask = bfs.sweep_schedule(M, h, twisted)
    tasks = _rows(tbl)
    assert len(tasks) == ntask[0] + ntask[1]
    # every slice of y and of z has exactly one writer
    wy = [u for u, t in enumerate(tasks) if t["out"] == 0]
    wz = [u for u, t in enumerate(tasks) if t["out"] == 1]
    assert sorted(tasks[u]["k"] for u in wy) == list(range(M))
    assert sorted(tasks[u]["k"] for u in wz) == list(range(M))
    writer = {(t["out"], t["k"]): u for u, t in enumerate(tasks)}
    for u, t in enumerate(tasks):
        assert len(t["blocks"]) <= min(h + 1, 4)
        for m, vec, uid in t["blocks"]:
            assert abs(m - t["k"]) <= h, "block outside the band"
            assert writer[(vec & 1, m)] == uid, "awaited tag names the wrong task"
            assert uid != u
        # the freshest vector (the group's previous task) is awaited last
        g0 = u < ntask[0]
        prev = u - 1 if (g0 and u > 0) or (not g0 and u > ntask[0]) else None
        uids = [uid for _, _, uid in t["blocks"]]
        if prev is not None and prev in uids:
            assert uids[-1] == prev
    # where a thread finds its columns of each vector: the critical one (written
    # by the group's previous task, polled last), a register-window entry (one of
    # the last two critical vectors, at the index given), or a prefetch
    for g, rng in ((0, range(ntask[0])), (1, range(ntask[0], ntask[0] + ntask[1]))):
        win = []
        for u in rng:
            prev = u - 1 if u != rng.start else None
            crit = None
            for m, vec, uid in tasks[u]["blocks"]:
                src, wi = (vec >> 2) & 3, (vec >> 4) & 3
                assert src in (0, 1, 2)
                if uid == prev:
                    assert src == 2
                    crit = uid
                elif src == 1:
                    assert wi < len(win) and win[wi] == uid
                else:
                    assert src == 0
            if crit is not None:
                win = [crit] + win[:1]
    rounds = _simulate(M, tasks, ntask)
    assert rounds is not None, "the schedule has a cycle"
    two = twisted and h >= 1 and M - h >= 2
    if two:
        assert ntask[1] > 0
        # about M dependent steps instead of 2M
        assert rounds <= M + h + 2, rounds
        # block 0 advances the tag word at its end: group 0's last task must
        # depend, through the table, on group 1's tasks (so every CTA has read
        # the launch's tag by then)
        seen, stack = set(), [ntask[0] - 1]
        while stack:
            u = stack.pop()
            for _, _, uid in tasks[u]["blocks"]:
                if uid not in seen:
                    seen.add(uid)
                    stack.append(uid)
        assert any(uid >= ntask[0] for uid in seen)
    else:
        assert ntask[1] == 0 and rounds == 2 * M


def _factor(Bk, M, h, twist):
    """Block LU of a block-banded matrix in the slot layout of the GPU factor:
    diagonal slots D^-1; one-ended: L below, W above; two-ended: top rows as
    one-ended, bottom rows W' below and U' above, middle-middle slots C^-1."""
    B = {key: v.copy() for key, v in Bk.items()}
    inv = np.linalg.inv

    def elim(k, lo, hi):
        B[(k, k)] = inv(B[(k, k)])
        for j in range(lo, hi + 1):
            B[(k, j)] = B[(k, k)] @ B[(k, j)]
        for i in range(lo, hi + 1):
            for j in range(lo, hi + 1):
                B[(i, j)] = B[(i, j)] - B[(i, k)] @ B[(k, j)]
        for i in range(lo, hi + 1):
            B[(i, k)] = B[(i, k)] @ B[(k, k)]

    if twist < 0:
        for k in range(M):
            elim(k, k + 1, min(M - 1, k + h))
        return B
    t0, t1 = twist, twist + h
    for i in range(max(t0, M - t1)):
        if i < t0:
            elim(i, i + 1, min(M - 1, i + h))
        kb = M - 1 - i
        if kb >= t1:
            elim(kb, max(0, kb - h), kb - 1)
    mid = list(range(t0, t1))
    C = np.block([[B[(a, b)] for b in mid] for a in mid])
    Ci = inv(C)
    nb = B[(0, 0)].shape[0]
    for ia, a in enumerate(mid):
        for ib, b in enumerate(mid):
            B[(a, b)] = Ci[ia * nb:(ia + 1) * nb, ib * nb:(ib + 1) * nb]
    return B


@pytest.mark.parametrize("M,h", [(3, 1), (5, 3), (8, 2), (13, 3), (12, 1), (7, 0)])
@pytest.mark.parametrize("twisted", [0, 1])
def test_schedule_solves_banded_system(M, h, twisted):
    nb = 5
    rng = np.random.default_rng(170908803 + 31 * M + h)
    Bk = {}
    for l in range(M):
        for m in range(max(0, l - h), min(M, l + h + 1)):
            Bk[(l, m)] = rng.standard_normal((nb, nb)) * 0.3 + (np.eye(nb) * 4.0 if l == m else 0.0)
    A = np.zeros((M * nb, M * nb))
    for (l, m), v in Bk.items():
        A[l * nb:(l + 1) * nb, m * nb:(m + 1) * nb] = v
    tbl, ntask = bfs.sweep_schedule(M, h, twisted)
    tasks = _rows(tbl)
    two = twisted and h >= 1 and M - h >= 2
    B = _factor(Bk, M, h, (M - h) // 2 if two else -1)
    r = rng.standard_normal(M * nb)
    y, z = {}, {}
    order = list(range(ntask[0] + ntask[1]))
    # any order the dependencies allow gives the same result: run group 1 first
    # where possible to exercise interleavings other than lockstep
    pending = order[ntask[0]:] + order[:ntask[0]]
    written = set()
    while pending:
        for u in pending:
            t = tasks[u]
            if all(uid in written for _, _, uid in t["blocks"]):
                k = t["k"]
                acc = r[k * nb:(k + 1) * nb].copy() if t["out"] == 0 else np.zeros(nb)
                for m, vec, _ in t["blocks"]:
                    v = (z if vec & 1 else y)[m]
                    acc += (1.0 if vec & 2 else -1.0) * (B[(k, m)] @ v)
                (z if t["out"] else y)[k] = acc
                written.add(u)
                pending.remove(u)
                break
        else:
            raise AssertionError("cycle")
    x = np.concatenate([z[k] for k in range(M)])
    ref = np.linalg.solve(A, r)
    assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()


def test_schedule_rejects_wide_band():
    with pytest.raises(bfs.BfsError):
        bfs.sweep_schedule(10, 4, 1)
