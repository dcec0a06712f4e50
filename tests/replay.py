"""CPU checks of emitted instruction graphs (test infrastructure).

* ``sequential_run``: runs a program's tasks in order on one flat array per
  buffer (the sequential meaning of the program, no graph involved).
* ``replay``: executes per-node instruction graphs on virtual memories
  (one byte array per allocation), matching receives to sends by
  (task, buffer, receiver); before every device kernel it checks that each
  read accessor's allocation holds the newest data, and it returns the final
  buffer contents for comparison with ``sequential_run``.
* ``check_invariants``: structural checks of one node's graph.

The workload kernels are restated here in numpy with the same float32
operation order as the CUDA kernels (no fused multiply-add).
"""
from __future__ import annotations

import numpy as np

from paper_2503_10516_gb300 import workloads as W

NONE = 0xFFFFFFFF
EPOCH, HORIZON, ALLOC, FREE, COPY, SEND, RECEIVE, SPLIT_RECEIVE, AWAIT_RECEIVE, KERNEL = range(10)
K_DATAFLOW, K_ANTI, K_ALLOC, K_EPOCH, K_FRONT = 1, 2, 4, 8, 16

NBODY_EPS = np.float32(1e-6)
NBODY_DT = np.float32(0.01)


def item_lo(mapper, item, ext, bdims):
    """Low corner of one kernel item's mapped box, or None if clamped empty."""
    p = []
    for d in range(3):
        kind, a, b, c = mapper[d]
        if d >= bdims:
            l, h = 0, 1
        elif kind == 1:
            l, h = 0, ext[d]
        elif kind == 2:
            l, h = a, b
        else:
            off = b - (1 << 32) if b >= (1 << 31) else b
            l, h = item[a] + off - c, item[a] + off + c + 1
        l, h = max(l, 0), min(h, ext[d])
        if l >= h:
            return None
        p.append(l)
    return tuple(p)


def mix(seq, w, lin):
    h = (seq * 0x9E3779B1 + (w + 1) * 0x85EBCA77 + lin * 0xC2B2AE3D) & 0xFFFFFFFF
    h ^= h >> 15
    h = (h * 0x2C1B3C6D) & 0xFFFFFFFF
    h ^= h >> 12
    return h


class View:
    """Element access to a buffer region stored as a byte array over `box`."""

    def __init__(self, data: np.ndarray, lo, dtype: str):
        self.data, self.lo, self.dtype = data, tuple(lo), dtype

    def typed(self):
        if self.dtype == "u32":
            return self.data.view(np.uint32)[..., 0]
        if self.dtype == "f32":
            return self.data.view(np.float32)[..., 0]
        return self.data.view(np.float32)  # (..., 4)

    def sl(self, box_lo, box_hi):
        return tuple(slice(box_lo[d] - self.lo[d], box_hi[d] - self.lo[d]) for d in range(3))


def run_kernel(task: W.Task, seq: int, chunk_lo, chunk_hi, rviews, wviews, bufs):
    """Runs one workload kernel over kernel-index box [chunk_lo, chunk_hi).
    rviews[a] / wviews[a]: View for accessor a (reads / writes), or None."""
    k = task.kernel
    acc = task.accessors
    if k == W.K_NOP:
        return
    if k in (W.K_JACOBI, W.K_WAVE):
        if k == W.K_JACOBI:
            src_i, dst_i, prev_i = 0, 1, None
        else:
            prev_i, src_i, dst_i = 0, 1, 2
        H, Wd = bufs[acc[src_i].buffer].extent[:2]
        y0, y1 = chunk_lo[0], chunk_hi[0]
        x0, x1 = chunk_lo[1], chunk_hi[1]
        U = rviews[src_i].typed()
        ulo = rviews[src_i].lo
        Y, X = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
        interior = (Y > 0) & (Y < H - 1) & (X > 0) & (X < Wd - 1)

        def at(dy, dx):
            yy = np.clip(Y + dy, ulo[0], ulo[0] + U.shape[0] - 1) - ulo[0]
            xx = np.clip(X + dx, ulo[1], ulo[1] + U.shape[1] - 1) - ulo[1]
            return U[yy, xx, 0]
        c = at(0, 0)
        if k == W.K_JACOBI:
            val = ((at(-1, 0) + at(1, 0)) + (at(0, -1) + at(0, 1))) * np.float32(0.25)
        else:
            P = rviews[prev_i].typed()
            plo = rviews[prev_i].lo
            pv = P[Y - plo[0], X - plo[1], 0]
            t2 = (np.float32(2.0) * c) - pv
            t5 = (at(-1, 0) + at(1, 0)) + (at(0, -1) + at(0, 1))
            t8 = np.float32(0.25) * (t5 - np.float32(4.0) * c)
            val = t2 + t8
        out = np.where(interior, val, c).astype(np.float32)
        D = wviews[dst_i].typed()
        dlo = wviews[dst_i].lo
        D[y0 - dlo[0]:y1 - dlo[0], x0 - dlo[1]:x1 - dlo[1], 0] = out
        return
    if k == W.K_NBODY_STEP:
        Pv, Vr, Vw = rviews[0], rviews[1], wviews[1]
        P = Pv.typed()[:, 0, 0]
        n = bufs[acc[0].buffer].extent[0]
        i0, i1 = chunk_lo[0], chunk_hi[0]
        pi = P[i0 - Pv.lo[0]:i1 - Pv.lo[0]]
        ax = np.zeros(i1 - i0, np.float32)
        ay = np.zeros(i1 - i0, np.float32)
        az = np.zeros(i1 - i0, np.float32)
        for j in range(n):
            pj = P[j - Pv.lo[0]]
            dx = pj[0] - pi[:, 0]
            dy = pj[1] - pi[:, 1]
            dz = pj[2] - pi[:, 2]
            r2 = ((dx * dx + dy * dy) + dz * dz) + NBODY_EPS
            s = np.sqrt(r2)
            inv = np.float32(1.0) / (r2 * s)
            wgt = pj[3] * inv
            ax = ax + dx * wgt
            ay = ay + dy * wgt
            az = az + dz * wgt
        V = Vr.typed()[i0 - Vr.lo[0]:i1 - Vr.lo[0], 0, 0].copy()
        V[:, 0] = V[:, 0] + ax * NBODY_DT
        V[:, 1] = V[:, 1] + ay * NBODY_DT
        V[:, 2] = V[:, 2] + az * NBODY_DT
        Vw.typed()[i0 - Vw.lo[0]:i1 - Vw.lo[0], 0, 0] = V
        return
    if k == W.K_NBODY_UPDATE:
        Vv, Pr, Pw = rviews[0], rviews[1], wviews[1]
        i0, i1 = chunk_lo[0], chunk_hi[0]
        V = Vv.typed()[i0 - Vv.lo[0]:i1 - Vv.lo[0], 0, 0]
        P = Pr.typed()[i0 - Pr.lo[0]:i1 - Pr.lo[0], 0, 0].copy()
        for c in range(3):
            P[:, c] = P[:, c] + V[:, c] * NBODY_DT
        Pw.typed()[i0 - Pw.lo[0]:i1 - Pw.lo[0], 0, 0] = P
        return
    if k == W.K_GROW:
        y0, y1 = chunk_lo[0], chunk_hi[0]
        x0, x1 = chunk_lo[1], chunk_hi[1]
        if len(acc) == 1:
            Yb, Xb = np.meshgrid(np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
            val = ((Yb * 131 + Xb * 7) & 1023).astype(np.float32) * np.float32(0.5)
            D = wviews[0]
        else:
            r = task.params[0]
            Yb, Xb = np.meshgrid(np.arange(y0 + r, y1 + r), np.arange(x0, x1), indexing="ij")
            S = rviews[0]
            last = S.typed()[r - 1 - S.lo[0], x0 - S.lo[1]:x1 - S.lo[1], 0]
            val = last[None, :] * np.float32(0.5) + (Yb & 255).astype(np.float32)
            D = wviews[1]
        T = D.typed()
        T[Yb - D.lo[0], Xb - D.lo[1], 0] = val.astype(np.float32)
        return
    if k == W.K_GENERIC:
        for y in range(chunk_lo[0], chunk_hi[0]):
            for x in range(chunk_lo[1], chunk_hi[1]):
                for z in range(chunk_lo[2], chunk_hi[2]):
                    item = (y, x, z)
                    s = 0
                    for ai, a in enumerate(acc):
                        if not (a.mode & W.READ):
                            continue
                        B = bufs[a.buffer]
                        q = item_lo(a.mapper, item, B.extent, B.dims)
                        if q is None:
                            continue
                        v = rviews[ai]
                        s = (s + int(v.typed()[tuple(q[d] - v.lo[d] for d in range(3))])) & 0xFFFFFFFF
                    for ai, a in enumerate(acc):
                        if not (a.mode & W.WRITE):
                            continue
                        B = bufs[a.buffer]
                        p = item_lo(a.mapper, item, B.extent, B.dims)
                        if p is None:
                            continue
                        lin = (p[0] * B.extent[1] + p[1]) * B.extent[2] + p[2]
                        v = wviews[ai]
                        v.typed()[tuple(p[d] - v.lo[d] for d in range(3))] = (mix(seq, ai, lin) + s) & 0xFFFFFFFF
        return
    raise ValueError(f"unknown kernel {k}")


def _buf_bytes(b: W.Buffer):
    shape = tuple(b.extent) + (b.elem_size,)
    if b.init is not None:
        return np.frombuffer(np.ascontiguousarray(b.init).tobytes(), dtype=np.uint8).reshape(shape).copy()
    return np.zeros(shape, dtype=np.uint8)


def horizon_after(prog: W.Program):
    """Per task: whether a horizon follows it (every horizon_step tasks, or by
    the task graph's critical path, the brute-force generator's per-element
    bookkeeping deciding)."""
    tasks = prog.tasks
    if not prog.horizon_cp:
        return [bool(prog.horizon_step) and (i + 1) % prog.horizon_step == 0 for i in range(len(tasks))]
    from tests.brute_idag import Brute
    b = Brute(1, 1, prog.horizon_step, 0)
    for buf in prog.buffers:
        b.create_buffer(buf.dims, buf.extent[:buf.dims], buf.elem_size, False)
    return [bool(b._critical_path(t)) for t in tasks]


def task_seqs(prog: W.Program):
    """Item sequence numbers: buffers, tasks, horizons, epochs, destroys each
    consume one; a lookahead change consumes none."""
    out, seq, k = [], 0, 0
    follow = horizon_after(prog)
    for op in prog.ops:
        if op[0] == "task":
            out.append(seq)
            seq += 1
            if follow[k]:
                seq += 1
            k += 1
        elif op[0] in ("buffer", "flush", "destroy"):
            seq += 1
    return out


def sequential_run(prog: W.Program, rejected=()):
    """Final contents of every buffer when the tasks run one after another on
    whole buffers; also which elements were ever written or initialised."""
    bufs = prog.buffers
    data = [_buf_bytes(b) for b in bufs]
    known = [np.full(b.extent, b.init is not None, dtype=bool) for b in bufs]
    seqs = task_seqs(prog)
    for t, seq in zip(prog.tasks, seqs):
        if seq in rejected:
            continue
        pre = [d.copy() for d in data]
        rv = [View(pre[a.buffer], (0, 0, 0), bufs[a.buffer].dtype) for a in t.accessors]
        wv = [View(data[a.buffer], (0, 0, 0), bufs[a.buffer].dtype) for a in t.accessors]
        run_kernel(t, seq, (0, 0, 0), tuple(t.range), rv, wv, bufs)
        for a in t.accessors:
            if a.mode & W.WRITE:
                # mark written elements: run the mapper over the kernel range
                B = bufs[a.buffer]
                if a.mapper == W.one_to_one():
                    hi = [min(t.range[d], B.extent[d]) if d < B.dims else 1 for d in range(3)]
                    known[a.buffer][:hi[0], :hi[1], :hi[2]] = True
                else:
                    for y in range(t.range[0]):
                        for x in range(t.range[1]):
                            for z in range(t.range[2]):
                                p = item_lo(a.mapper, (y, x, z), B.extent, B.dims)
                                if p is not None:
                                    known[a.buffer][p] = True
    return data, known


class _Alloc:
    def __init__(self, buffer, mem, box, elem):
        self.buffer, self.mem, self.box = buffer, mem, box
        shape = tuple(box[3 + d] - box[d] for d in range(3)) + (elem,)
        self.data = np.zeros(shape, dtype=np.uint8)

    def sl(self, bx):
        return tuple(slice(bx[d] - self.box[d], bx[3 + d] - self.box[d]) for d in range(3))


def replay(prog: W.Program, graphs, rejected=(), check_reads=True):
    """Execute the graphs; returns (final contents, known mask, stats)."""
    bufs = prog.buffers
    tasks = dict(zip(task_seqs(prog), prog.tasks))
    N = len(graphs)
    allocs = [dict() for _ in range(N)]
    latest = [_buf_bytes(b) for b in bufs]
    known = [np.full(b.extent, b.init is not None, dtype=bool) for b in bufs]
    messages = {}
    stats = {"kernels": 0, "copies": 0, "copy_bytes": 0, "reads_checked": 0}

    def get_alloc(n, aid, buffer):
        if aid not in allocs[n]:
            # user allocation on M0: the buffer's host data
            B = bufs[buffer]
            a = _Alloc(buffer, 0, (0, 0, 0) + tuple(B.extent), B.elem_size)
            a.data[...] = _buf_bytes(B)
            allocs[n][aid] = a
        return allocs[n][aid]

    blocks = []
    for n, g in enumerate(graphs):
        by_seq = {}
        for i, r in enumerate(g["instrs"]):
            if r[2] == NONE:
                continue
            by_seq.setdefault(int(r[2]), []).append(i)
        blocks.append(by_seq)
    all_seqs = sorted(set(s for b in blocks for s in b))

    def boxes(g, r):
        return [tuple(int(v) for v in g["boxes"][r[7] + j]) for j in range(r[8])]

    def execute(n, i, pending):
        g = graphs[n]
        r = g["instrs"][i]
        typ, seq, a, b, c, d = (int(x) for x in r[1:7])
        if typ == ALLOC:
            bx = boxes(g, r)[0]
            allocs[n][a] = _Alloc(c, b, bx, bufs[c].elem_size)
        elif typ == FREE:
            del allocs[n][a]
        elif typ == COPY:
            src, dst = get_alloc(n, a, c), allocs[n][b]
            for bx in boxes(g, r):
                dst.data[dst.sl(bx)] = src.data[src.sl(bx)]
                stats["copy_bytes"] += src.data[src.sl(bx)].size
            stats["copies"] += 1
        elif typ == SEND:
            src = allocs[n][a]
            bx = boxes(g, r)[0]
            messages.setdefault((seq, c, b), []).append((bx, src.data[src.sl(bx)].copy()))
        elif typ in (RECEIVE, SPLIT_RECEIVE):
            dst = allocs[n][a]
            W_ = boxes(g, r)
            got = messages.get((seq, c, n), [])
            shape = bufs[c].extent
            cover = np.zeros(shape, dtype=np.int32)
            for bx, payload in got:
                dst.data[dst.sl(bx)] = payload
                cover[bx[0]:bx[3], bx[1]:bx[4], bx[2]:bx[5]] += 1
            want = np.zeros(shape, dtype=np.int32)
            for bx in W_:
                want[bx[0]:bx[3], bx[1]:bx[4], bx[2]:bx[5]] += 1
            assert np.array_equal(cover, want), f"pilots do not tile the awaited region (node {n}, seq {seq})"
        elif typ == KERNEL:
            t = tasks[seq]
            binds = g["binds"][r[9]:r[9] + r[10]]
            rv, wv = [], []
            for ai, acc in enumerate(t.accessors):
                al = int(binds[ai][0])
                if al == NONE:
                    rv.append(None)
                    wv.append(None)
                    continue
                A = get_alloc(n, al, acc.buffer)
                bx = tuple(int(v) for v in binds[ai][1:])
                if check_reads and (acc.mode & W.READ):
                    mine = A.data[A.sl(bx)]
                    ref = latest[acc.buffer][bx[0]:bx[3], bx[1]:bx[4], bx[2]:bx[5]]
                    kn = known[acc.buffer][bx[0]:bx[3], bx[1]:bx[4], bx[2]:bx[5]]
                    bad = (mine != ref).any(axis=-1) & kn
                    assert not bad.any(), (f"stale read: node {n} instr {i} seq {seq} acc {ai} "
                                           f"buffer {acc.buffer} at {np.argwhere(bad)[:3].tolist()}")
                    stats["reads_checked"] += int(kn.sum())
                rv.append(View(A.data.copy(), A.box[:3], bufs[acc.buffer].dtype))
                wv.append(View(A.data, A.box[:3], bufs[acc.buffer].dtype))
            cb = boxes(g, r)[0]
            run_kernel(t, seq, cb[:3], cb[3:], rv, wv, bufs)
            for ai, acc in enumerate(t.accessors):
                if (acc.mode & W.WRITE) and int(binds[ai][0]) != NONE:
                    bx = tuple(int(v) for v in binds[ai][1:])
                    A = allocs[n][int(binds[ai][0])]
                    pending.append((acc.buffer, bx, A.data[A.sl(bx)].copy()))
            stats["kernels"] += 1

    for s in all_seqs:
        pending = []
        halves = []
        for n in range(N):
            idx = blocks[n].get(s, [])
            cut = len(idx)
            for j, i in enumerate(idx):
                if graphs[n]["instrs"][i][1] in (RECEIVE, SPLIT_RECEIVE):
                    cut = j
                    break
            halves.append((idx[:cut], idx[cut:]))
        for n in range(N):
            for i in halves[n][0]:
                execute(n, i, pending)
        for n in range(N):
            for i in halves[n][1]:
                execute(n, i, pending)
        for b, bx, payload in pending:
            latest[b][bx[0]:bx[3], bx[1]:bx[4], bx[2]:bx[5]] = payload
            known[b][bx[0]:bx[3], bx[1]:bx[4], bx[2]:bx[5]] = True
    return latest, known, stats


# ---- structural invariants -------------------------------------------------

def _ancestors(instrs, edges):
    n = len(instrs)
    preds = [[] for _ in range(n)]
    for f, t, k in edges:
        preds[int(t)].append(int(f))
    anc = [0] * n
    for i in range(n):
        a = 0
        for p in preds[i]:
            a |= anc[p] | (1 << p)
        anc[i] = a
    return anc, preds


def _box_vol(bx):
    v = 1
    for d in range(3):
        v *= max(0, bx[3 + d] - bx[d])
    return v


def _isect(a, b):
    lo = [max(a[d], b[d]) for d in range(3)]
    hi = [min(a[3 + d], b[3 + d]) for d in range(3)]
    return tuple(lo + hi) if all(lo[d] < hi[d] for d in range(3)) else None


def check_invariants(prog: W.Program, g: dict, node: int):
    """Structural invariants of one node's instruction graph (Sec. 3)."""
    instrs, edges, boxes, binds = g["instrs"], g["edges"], g["boxes"], g["binds"]
    tasks = dict(zip(task_seqs(prog), prog.tasks))
    n = len(instrs)
    assert n >= 1 and instrs[0][1] == EPOCH
    # edges point backwards, grouped by successor in emission order, sorted
    last = (-1, -1)
    has_pred = [False] * n
    for f, t, k in edges:
        assert f < t, "edge must point to an earlier instruction"
        assert (t, f) > last, "edges sorted by (successor, predecessor) and unique"
        last = (t, f)
        assert k != 0
        has_pred[t] = True
    assert all(has_pred[1:]), "every instruction after the first epoch has a predecessor"
    anc, preds = _ancestors(instrs, edges)
    # receives have no dataflow predecessors (Sec. 4.2)
    kinds = {}
    for f, t, k in edges:
        kinds[(int(f), int(t))] = int(k)
    for i, r in enumerate(instrs):
        if r[1] in (RECEIVE, SPLIT_RECEIVE):
            for p in preds[i]:
                assert not (kinds[(p, i)] & K_DATAFLOW), "receive with a dataflow predecessor"
    # allocations: disjoint per (buffer, memory), never shrink, accesses inside
    live = {}
    alloc_seq = {}  # allocation -> submission that allocated it
    accesses = []  # (instr, alloc, box, writes)

    def bx_of(r, j=0):
        return tuple(int(v) for v in boxes[r[7] + j])
    for i, r in enumerate(instrs):
        typ = int(r[1])
        a, b, c = int(r[3]), int(r[4]), int(r[5])
        if typ == ALLOC:
            box = bx_of(r)
            live[a] = (c, b, box)
            alloc_seq[a] = int(r[2])
            accesses.append((i, a, box, True))
        elif typ == FREE:
            assert a in live, "free of an unknown allocation"
            ob, om, obox = live.pop(a)
            # a resize frees an older allocation: a live allocation of (buffer,
            # memory) now holds its box (a host staging allocation is freed by
            # the submission that made it)
            if int(r[2]) in tasks and alloc_seq.get(a) != int(r[2]):
                assert any(lb == ob and lm == om and _isect(lbox, obox) == obox
                           for lb, lm, lbox in live.values()), "allocation shrank on resize"
            accesses.append((i, a, obox, True))
        elif typ == COPY:
            for j in range(r[8]):
                bx = bx_of(r, j)
                if a in live:
                    assert _isect(live[a][2], bx) == bx
                accesses.append((i, a, bx, False))
                assert b in live and _isect(live[b][2], bx) == bx, "copy outside its destination allocation"
                accesses.append((i, b, bx, True))
        elif typ == SEND:
            bx = bx_of(r)
            accesses.append((i, a, bx, False))
        elif typ in (RECEIVE, SPLIT_RECEIVE):
            for j in range(r[8]):
                bx = bx_of(r, j)
                assert _isect(live[a][2], bx) == bx
                accesses.append((i, a, bx, True))
        elif typ == KERNEL:
            t = tasks[int(r[2])]
            for ai, acc in enumerate(t.accessors):
                bd = binds[r[9] + ai]
                if bd[0] == NONE:
                    continue
                al = int(bd[0])
                bx = tuple(int(v) for v in bd[1:])
                if al in live:
                    lb, lm, lbox = live[al]
                    assert lb == acc.buffer and lm == b, "accessor bound to the wrong buffer or memory"
                    assert _isect(lbox, bx) == bx, "accessor not inside one allocation"
                if acc.mode & W.READ:
                    accesses.append((i, al, bx, False))
                if acc.mode & W.WRITE:
                    accesses.append((i, al, bx, True))
        # live allocations of one (buffer, memory) are pairwise disjoint after each instruction
        if typ in (KERNEL, SEND):
            groups = {}
            for oid, (ob, om, obox) in live.items():
                groups.setdefault((ob, om), []).append(obox)
            for lst in groups.values():
                for x in range(len(lst)):
                    for y in range(x + 1, len(lst)):
                        assert _isect(lst[x], lst[y]) is None, "overlapping live allocations"
    # no two conflicting accesses unordered in the DAG
    by_alloc = {}
    for acc in accesses:
        by_alloc.setdefault(acc[1], []).append(acc)
    for al, lst in by_alloc.items():
        for x in range(len(lst)):
            for y in range(x + 1, len(lst)):
                i1, _, b1, w1 = lst[x]
                i2, _, b2, w2 = lst[y]
                if i1 == i2 or not (w1 or w2):
                    continue
                if _isect(b1, b2) is None:
                    continue
                lo, hi = min(i1, i2), max(i1, i2)
                assert (anc[hi] >> lo) & 1, f"unordered conflicting accesses {lo} and {hi} on allocation {al}"
    return True
