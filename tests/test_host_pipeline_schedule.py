"""The schedule of the pipelined host-buffer step (gbh_abi.cu, host_step), restated
on the CPU: chunks of consecutive blocks, the reach need[k] of each chunk, the
launch order on the stage-1 and stage-2 streams with their event waits, and the
face pre-pass per chunk (gbh_stage.cu, face_flux_kernel over a block range).

For every lattice and chunking tried, a happens-before check over that schedule
shows that every face-flux slot a chunk's stage reads was written once in the
same stage, by a pre-pass ordered before the read, and that no write of the
other stage can land between that write and the read."""
import itertools

import numpy as np
import pytest

from paper_2401_03378_gb300.grid import neighbour_table


def face_table(ndim, nb, periodic):
    """[nblocks][6] face neighbours (x-, x+, y-, y+, z-, z+) from the full table."""
    full = neighbour_table(ndim, nb, periodic)
    centre = 13 if ndim == 3 else 4
    step = (1, 3, 9)
    out = np.full((full.shape[0], 6), -1, dtype=np.int64)
    for d in range(ndim):
        out[:, 2 * d] = full[:, centre - step[d]]
        out[:, 2 * d + 1] = full[:, centre + step[d]]
    return out


def chunks(nblocks, wanted, sms=152):
    """Chunk starts as the host step forms them: `wanted` equal chunks, or by
    default whole waves of two CTAs per SM with the remainder last."""
    wave = 2 * sms
    K = wanted if wanted > 0 else (nblocks + wave - 1) // wave
    K = max(1, min(K, 64, nblocks))
    first = [nblocks * k // K for k in range(K + 1)]
    if wanted == 0 and wave * (K - 1) < nblocks and (K - 1) * wave > 0:
        first = [k * wave for k in range(K)] + [nblocks]
    return first


def reach(face, first):
    K = len(first) - 1
    chunk_of = np.empty(face.shape[0], dtype=np.int64)
    for k in range(K):
        chunk_of[first[k]:first[k + 1]] = k
    need = []
    for k in range(K):
        m = k
        for b in range(first[k], first[k + 1]):
            for f in range(6):
                nb = face[b, f]
                if nb >= 0:
                    m = max(m, chunk_of[nb])
        need.append(m)
    return need, chunk_of


def prepass_writes(face, lo, hi, ndim):
    """Slots (block, face) the pre-pass over blocks [lo, hi) writes."""
    w = set()
    for b in range(lo, hi):
        for f in range(2 * ndim):
            nb = face[b, f]
            if f % 2 == 0:
                if not (0 <= nb < hi):
                    w.add((b, f))              # low face solved by the block itself
            else:
                w.add((b, f))
                if nb >= lo:
                    w.add((nb, f - 1))         # the neighbour's low face
    return w


def schedule(face, first, ndim):
    """Operations with vector clocks over the two stage streams: ('pre', s, k)
    writes, ('stage', s, k) reads the slots of chunk k's blocks."""
    K = len(first) - 1
    need, _ = reach(face, first)
    ops = []
    pos = {1: 0, 2: 0}
    vc_stream = {1: {1: 0, 2: 0}, 2: {1: 0, 2: 0}}
    s1_done = {}                              # clock of stream 1 after chunk k's stage 1

    def emit(s, kind, k, extra_wait=None):
        clock = dict(vc_stream[s])
        if extra_wait is not None:
            for t, v in extra_wait.items():
                clock[t] = max(clock[t], v)
        pos[s] += 1
        clock[s] = pos[s]
        vc_stream[s] = clock
        ops.append((kind, s, k, dict(clock)))

    for k in range(K):                         # stream 1; copies (stream 0) do not touch the slots
        emit(1, "pre", k)
        emit(1, "stage", k)
        s1_done[k] = dict(vc_stream[1])
    for k in range(K):                         # stream 2 waits for stage 1 of chunks up to need[k]
        emit(2, "pre", k, extra_wait=s1_done[need[k]])
        emit(2, "stage", k)
    return ops, need


def hb(a, b):
    """a happens before b (a's position on its stream is covered by b's clock)."""
    return a[3][a[1]] <= b[3][a[1]] and a is not b


@pytest.mark.parametrize("ndim,nb,periodic,wanted", [
    (3, (4, 4, 4), (True, True, True), 64),     # one block per chunk
    (3, (4, 4, 4), (True, True, True), 5),      # uneven chunks
    (3, (4, 4, 4), (True, True, True), 3),
    (3, (4, 4, 4), (True, True, True), 0),      # default: one chunk here
    (3, (8, 8, 8), (False, False, True), 7),
    (3, (3, 2, 5), (True, False, True), 4),
    (3, (2, 2, 2), (True, True, True), 8),      # every neighbour is also the other side's
    (3, (1, 3, 4), (True, True, True), 6),      # one block across x: its own neighbour
    (3, (16, 16, 16), (False, False, False), 0),  # the benchmark: 13 waves of 304 and 144
])
def test_chunked_prepass_slots_are_ready_and_not_overwritten(ndim, nb, periodic, wanted):
    check_schedule(face_table(ndim, nb, periodic), ndim, wanted)


@pytest.mark.parametrize("wanted", [0, 3, 7, 25])
def test_batched_problems_schedule(wanted):
    """A batched context's face table: independent lattices one after another
    (block ids offset), periodic wraps inside each problem."""
    parts, off = [], 0
    for nb, per in (((3, 3, 2), (True, True, True)), ((2, 4, 3), (False, True, True)), ((1, 2, 2), (True, True, True))):
        f = face_table(3, nb, per)
        parts.append(np.where(f >= 0, f + off, f))
        off += f.shape[0]
    check_schedule(np.concatenate(parts), 3, wanted)


def check_schedule(face, ndim, wanted):
    NB = face.shape[0]
    first = chunks(NB, wanted)
    K = len(first) - 1
    ops, need = schedule(face, first, ndim)
    writes = {}
    for op in ops:
        if op[0] == "pre":
            k = op[2]
            for slot in prepass_writes(face, first[k], first[k + 1], ndim):
                writes.setdefault(slot, []).append(op)
    # the whole-range pre-pass writes each slot once: the per-chunk form covers the same slots
    full = prepass_writes(face, 0, NB, ndim)
    assert full == {(b, f) for b in range(NB) for f in range(2 * ndim)}
    for op in ops:
        if op[0] != "stage":
            continue
        kind, s, k, _ = op
        for b in range(first[k], first[k + 1]):
            for f in range(2 * ndim):
                ws = writes.get((b, f), [])
                same = [w for w in ws if w[1] == s]
                other = [w for w in ws if w[1] != s]
                # written once in this stage, before the read
                assert len(same) == 1 and hb(same[0], op), (b, f, s, len(same))
                for w in other:
                    if s == 1:
                        # stage-2 writers come after this stage-1 read
                        assert hb(op, w), (b, f, "stage-2 write before stage-1 read")
                    else:
                        # stage-1 writers come before every stage-2 writer of the slot
                        assert all(hb(w, x) for x in same), (b, f, "stage-1 write after a stage-2 write")
    assert K == len(need)


def test_face_table_matches_offsets():
    face = face_table(3, (3, 2, 2), (True, False, False))
    # block 0 at (0, 0, 0): x- wraps to block 2, x+ is block 1, y- and z- are outflow
    assert list(face[0]) == [2, 1, -1, 3, -1, 6]
    for b, f in itertools.product(range(face.shape[0]), range(6)):
        nb = face[b, f]
        if nb >= 0:
            assert face[nb, f ^ 1] == b
