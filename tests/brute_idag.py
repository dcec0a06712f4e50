"""Per-element brute-force instruction-graph generator (test pin for the oracle).

Same lowering rules as the oracle, but every region is a dense boolean array
over the buffer's elements and every region map a dense per-element array;
range mappers are evaluated item by item and unioned, chunk membership is
decided row by row, and box lists are read off dense masks with an open-run
sweep over real coordinates. Only for tiny buffers (a few hundred elements).
Emits the same record layout as the oracle so graphs compare exactly.
"""
from __future__ import annotations

import numpy as np

NONE = 0xFFFFFFFF
REMOTE = 0xFFFFFFFE
HOST = 0xFFFFFFFE
LOOKAHEAD_HORIZONS = 0xFFFFFFFE  # lookahead value selecting the horizon-count heuristic
EPOCH, HORIZON, ALLOC, FREE, COPY, SEND, RECEIVE, SPLIT_RECEIVE, AWAIT_RECEIVE, KERNEL = range(10)
K_DATAFLOW, K_ANTI, K_ALLOC, K_EPOCH, K_FRONT = 1, 2, 4, 8, 16
M_READ, M_WRITE = 1, 2


# ---- masks and boxes ------------------------------------------------------

def box_mask(shape, box):
    m = np.zeros(shape, dtype=bool)
    lo, hi = box[:3], box[3:]
    if all(lo[d] < hi[d] for d in range(3)):
        m[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = True
    return m


def _rects2d(m2):
    """Canonical rectangles of a 2D mask: open-run sweep over rows."""
    out = []
    open_ = {}
    for j in range(m2.shape[0]):
        row = m2[j]
        runs = set()
        k = 0
        while k < row.shape[0]:
            if row[k]:
                s = k
                while k < row.shape[0] and row[k]:
                    k += 1
                runs.add((s, k))
            else:
                k += 1
        for r in list(open_):
            if r not in runs:
                out.append((open_.pop(r), j) + r)
        for r in runs:
            if r not in open_:
                open_[r] = j
    for r, s in open_.items():
        out.append((s, m2.shape[0]) + r)
    return out


def boxes_of(mask):
    """Canonical box list of a 3D mask: maximal runs along the fastest dim,
    identical runs merged over rows, identical rectangles merged over slabs."""
    out = []
    open_ = {}
    for i in range(mask.shape[0]):
        rects = set(_rects2d(mask[i]))
        for r in list(open_):
            if r not in rects:
                s = open_.pop(r)
                out.append((s, r[0], r[2], i, r[1], r[3]))
        for r in rects:
            if r not in open_:
                open_[r] = i
    for r, s in open_.items():
        out.append((s, r[0], r[2], mask.shape[0], r[1], r[3]))
    out.sort()
    return [tuple(int(v) for v in b) for b in out]


def bbox_of_mask(m):
    idx = np.nonzero(m)
    lo = [int(x.min()) for x in idx]
    hi = [int(x.max()) + 1 for x in idx]
    return tuple(lo + hi)


# ---- program semantics evaluated per element ------------------------------

def chunk_rows(E0, C):
    """chunk index of every row, by testing each chunk's row interval."""
    owner = [-1] * E0
    for y in range(E0):
        for c in range(C):
            if (c * E0) // C <= y < ((c + 1) * E0) // C:
                owner[y] = c
                break
    return owner


def item_box(mapper, item, bshape, bdims):
    """Mapped box of one kernel item (a single index point), clamped."""
    lo, hi = [], []
    for d in range(3):
        ext = bshape[d]
        kind, a, b, c = mapper[d]
        if d >= bdims:
            l, h = 0, 1
        elif kind == 1:
            l, h = 0, ext
        elif kind == 2:
            l, h = a, b
        else:
            off = b - (1 << 32) if b >= (1 << 31) else b
            l, h = item[a] + off - c, item[a] + off + c + 1
        l, h = max(l, 0), min(h, ext)
        if l >= h:
            return None
        lo.append(l)
        hi.append(h)
    return tuple(lo + hi)


class BruteNode:
    def __init__(self, nid, lookahead):
        self.id = nid
        self.instrs, self.edges, self.boxes, self.binds, self.diags = [], [], [], [], []
        self.types = [EPOCH]
        self.instrs.append([0, EPOCH, NONE, NONE, NONE, NONE, NONE, 0, 0, 0, 0])
        self.front = {0}
        self.epoch = 0
        self.last_horizon = None
        self.next_msg = 0
        self.lookahead = lookahead
        self.queue = []
        self.h_after = 0   # horizons queued since the last allocating task
        self.allocs = []   # dicts
        self.bstate = {}   # buffer -> (prod, pmem, mask) int64 arrays


class Brute:
    def __init__(self, nodes, devices, horizon_step, lookahead):
        self.N, self.D, self.hstep = nodes, devices, horizon_step
        self.bufs = []
        self.own = {}  # buffer -> (owner, repl) arrays
        self.nodes = [BruteNode(n, lookahead) for n in range(nodes)]
        self.seq = 0
        self.ntasks = 0
        self.rejected = []
        self.stage_d2d = False  # device-to-device copies staged in host memory
        self.horizon_cp = False  # horizons by the task graph's critical path
        self.t_last = {}         # buffer -> per-element task that last wrote it (-1: none)
        self.t_read = {}         # buffer -> {task: elements it read since their last write}
        self.depth = []          # per task: depth in the task graph
        self.cpl = 0
        self.cpl_h = 0

    # -- items --
    def create_buffer(self, dims, extent, elem, init):
        shape = tuple(int(extent[d]) if d < dims else 1 for d in range(3))
        bid = len(self.bufs)
        self.bufs.append({"dims": dims, "shape": shape, "init": bool(init), "live": True})
        self.own[bid] = (np.full(shape, HOST if init else NONE, dtype=np.int64),
                         np.full(shape, 0xFFFFFFFF, dtype=np.int64))
        self._broadcast("create", bid)
        return bid

    def destroy_buffer(self, b):
        self.bufs[b]["live"] = False
        self._broadcast("destroy", b)

    def set_lookahead(self, L):
        for n in self.nodes:
            if L == LOOKAHEAD_HORIZONS and n.queue:
                self._flush(n)
            n.lookahead = L
            n.h_after = 0
            if n.queue and self._queued(n) > n.lookahead:
                self._flush(n)

    def flush(self):
        self._broadcast("epoch", 0)

    def _broadcast(self, kind, arg):
        s = self.seq
        self.seq += 1
        for n in self.nodes:
            self._deliver(n, {"kind": kind, "seq": s, "arg": arg})

    def submit(self, task):
        seq = self.seq
        self.seq += 1
        kdims, krange, C = task.dims, list(task.range), task.chunks
        M = self.N * self.D
        chunks = []
        if C >> 16:
            # a grid of Cy x Cx chunks: grid rows to nodes, then each node's
            # chunks (row-major) to its devices, both by block assignment
            Cy, Cx = C & 0xFFFF, C >> 16
            owner_row, owner_col = chunk_rows(krange[0], Cy), chunk_rows(krange[1], Cx)
            node_of = [(iy * self.N) // Cy for iy in range(Cy)]
            for iy in range(Cy):
                n = node_of[iy]
                grid_rows = [r for r in range(Cy) if node_of[r] == n]
                K = len(grid_rows) * Cx
                for ix in range(Cx):
                    rows = [y for y in range(krange[0]) if owner_row[y] == iy]
                    cols = [x for x in range(krange[1]) if owner_col[x] == ix]
                    if not rows or not cols:
                        continue
                    j = grid_rows.index(iy) * Cx + ix
                    chunks.append({"index": iy * Cx + ix, "node": n, "mem": 2 + (j * self.D) // K,
                                   "box": (rows[0], cols[0], 0, rows[-1] + 1, cols[-1] + 1, krange[2]),
                                   "rows": rows, "cols": cols})
        else:
            owner_row = chunk_rows(krange[0], C)
            for c in range(C):
                rows = [y for y in range(krange[0]) if owner_row[y] == c]
                if not rows:
                    continue
                g = (c * M) // C
                chunks.append({"index": c, "node": g // self.D, "mem": 2 + g % self.D,
                               "box": (rows[0], 0, 0, rows[-1] + 1, krange[1], krange[2]), "rows": rows,
                               "cols": list(range(krange[1]))})
        accs = task.accessors
        # mapped masks: union over the chunk's items of each item's mapped box
        for ch in chunks:
            ch["masks"] = []
            for a in accs:
                buf = self.bufs[a.buffer]
                m = np.zeros(buf["shape"], dtype=bool)
                for y in ch["rows"]:
                    for x in ch["cols"]:
                        for z in range(krange[2]):
                            bx = item_box(a.mapper, (y, x, z), buf["shape"], buf["dims"])
                            if bx is not None:
                                m |= box_mask(buf["shape"], bx)
                ch["masks"].append(m)
        bad = False
        for i in range(len(chunks)):
            for j in range(i + 1, len(chunks)):
                for ai, a in enumerate(accs):
                    for bi, b in enumerate(accs):
                        if (a.mode & M_WRITE) and (b.mode & M_WRITE) and a.buffer == b.buffer:
                            if (chunks[i]["masks"][ai] & chunks[j]["masks"][bi]).any():
                                bad = True
        if bad:
            self.rejected.append(seq)
        else:
            per = [{"seq": seq, "task": task, "chunks": [c for c in chunks if c["node"] == n],
                    "remote": [c for c in chunks if c["node"] != n], "push": {}, "await": {}}
                   for n in range(self.N)]
            for b in sorted({a.buffer for a in accs}):
                owner, repl = self.own[b]
                shape = self.bufs[b]["shape"]
                missing = []
                for m in range(self.N):
                    R = np.zeros(shape, dtype=bool)
                    for ch in chunks:
                        if ch["node"] != m:
                            continue
                        for ai, a in enumerate(accs):
                            if a.buffer == b and (a.mode & M_READ):
                                R |= ch["masks"][ai]
                    missing.append(R & (((repl >> m) & 1) == 0))
                for m in range(self.N):
                    if not missing[m].any():
                        continue
                    per[m]["await"][b] = missing[m].copy()
                    for o in range(self.N):
                        g = missing[m] & (owner == o)
                        if g.any():
                            per[o]["push"][(b, m)] = g
                for m in range(self.N):
                    repl[missing[m]] |= (1 << m)
                for ch in chunks:
                    for ai, a in enumerate(accs):
                        if a.buffer == b and (a.mode & M_WRITE):
                            owner[ch["masks"][ai]] = ch["node"]
                            repl[ch["masks"][ai]] = 1 << ch["node"]
            for n in range(self.N):
                self._deliver(self.nodes[n], {"kind": "task", "seq": seq, "nt": per[n]})
        fire = self._critical_path(task)
        self.ntasks += 1
        if (fire if self.horizon_cp else (self.hstep and self.ntasks % self.hstep == 0)):
            self._broadcast("horizon", 0)
        return 0 if not bad else -2

    def _critical_path(self, task):
        """Task-graph depth of this task from per-element last writers and
        readers; True when the longest path grew by horizon_step since the
        last horizon."""
        me = len(self.depth)
        masks = []
        for a in task.accessors:
            buf = self.bufs[a.buffer]
            m = np.zeros(buf["shape"], dtype=bool)
            for y in range(task.range[0]):
                for x in range(task.range[1]):
                    for z in range(task.range[2]):
                        bx = item_box(a.mapper, (y, x, z), buf["shape"], buf["dims"])
                        if bx is not None:
                            m |= box_mask(buf["shape"], bx)
            masks.append(m)
        deepest = 0
        for a, m in zip(task.accessors, masks):
            last = self.t_last.setdefault(a.buffer, np.full(self.bufs[a.buffer]["shape"], -1, dtype=np.int64))
            readers = self.t_read.setdefault(a.buffer, {})
            for u in np.unique(last[m]):
                if u >= 0:
                    deepest = max(deepest, self.depth[int(u)])
            if a.mode & M_WRITE:
                for u, rm in readers.items():
                    if (rm & m).any():
                        deepest = max(deepest, self.depth[u])
        self.depth.append(deepest + 1)
        for a, m in zip(task.accessors, masks):
            if a.mode & M_READ:
                readers = self.t_read[a.buffer]
                readers[me] = readers.get(me, np.zeros_like(m)) | m
        for a, m in zip(task.accessors, masks):
            if a.mode & M_WRITE:
                for u in self.t_read[a.buffer]:
                    self.t_read[a.buffer][u] = self.t_read[a.buffer][u] & ~m
                self.t_last[a.buffer][m] = me
        self.cpl = max(self.cpl, deepest + 1)
        if self.hstep and self.cpl >= self.cpl_h + self.hstep:
            self.cpl_h = self.cpl
            return True
        return False

    # -- lookahead queue --
    def _queued(self, n):
        return sum(1 for x in n.queue if x["kind"] == "task")

    def _flush(self, n):
        while n.queue:
            it = n.queue.pop(0)
            look = [q["nt"] for q in n.queue if q["kind"] == "task"]
            self._process(n, it, look)

    def _deliver(self, n, it):
        horizons = n.lookahead == LOOKAHEAD_HORIZONS
        if not n.queue:
            if it["kind"] == "task" and self._allocating(n, it["nt"]):
                n.queue.append(it)
                n.h_after = 0
                if not horizons and self._queued(n) > n.lookahead:
                    self._flush(n)
            else:
                self._process(n, it, [])
            return
        if horizons:
            # compile once two horizons follow the last task that the queue
            # would not make room for
            if it["kind"] == "task" and self._allocating_queued(n, it["nt"]):
                n.h_after = 0
            n.queue.append(it)
            if it["kind"] == "horizon":
                n.h_after += 1
            if it["kind"] in ("epoch", "destroy") or n.h_after >= 2:
                self._flush(n)
            return
        n.queue.append(it)
        if it["kind"] in ("epoch", "destroy") or self._queued(n) > n.lookahead:
            self._flush(n)

    # -- requirements / allocations --
    def _reqs(self, nt):
        out = []
        task = nt["task"]
        for ch in nt["chunks"]:
            for ai, a in enumerate(task.accessors):
                if ch["masks"][ai].any():
                    out.append((a.buffer, ch["mem"], ch["masks"][ai]))
        for (b, t), g in sorted(nt["push"].items()):
            out.append((b, 1, box_mask(g.shape, bbox_of_mask(g))))
        for b, g in sorted(nt["await"].items()):
            out.append((b, 1, box_mask(g.shape, bbox_of_mask(g))))
        return out

    def _find_alloc(self, n, b, m, mask):
        for al in n.allocs:
            if al["live"] and al["buffer"] == b and al["mem"] == m and not (mask & ~al["mask"]).any():
                return al["id"]
        return None

    def _allocating(self, n, nt):
        return any(self._find_alloc(n, b, m, mk) is None for b, m, mk in self._reqs(nt))

    def _allocating_queued(self, n, nt):
        queued = [r for q in n.queue if q["kind"] == "task" for r in self._reqs(q["nt"])]
        for b, m, mk in self._reqs(nt):
            if self._find_alloc(n, b, m, mk) is not None:
                continue
            if not any(qb == b and qm == m and not (mk & ~qmk).any() for qb, qm, qmk in queued):
                return True
        return False

    # -- emission --
    def _emit(self, n, rec, masks, accesses, extra, binds=None):
        iid = len(n.instrs)
        deps = dict(extra)
        for aid, R, mode in accesses:
            al = n.allocs[aid]
            inside = R & al["mask"]
            ws = set(int(v) for v in np.unique(al["writers"][inside]))
            if mode & M_READ:
                for w in ws:
                    deps[w] = deps.get(w, 0) | (K_ALLOC if n.types[w] == ALLOC else K_DATAFLOW)
            if mode & M_WRITE:
                for w in ws:
                    deps[w] = deps.get(w, 0) | (K_ALLOC if n.types[w] == ALLOC else K_ANTI)
                for x, rm in al["readers"].items():
                    if (rm & R).any():
                        deps[x] = deps.get(x, 0) | K_ANTI
        if not deps:
            deps[n.epoch] = K_EPOCH
        for p in sorted(deps):
            n.edges.append([p, iid, deps[p]])
            n.front.discard(p)
        n.front.add(iid)
        boxes = []
        for m in masks:
            boxes.extend(boxes_of(m) if isinstance(m, np.ndarray) else [m])
        r = [iid] + rec + [len(n.boxes), len(boxes), len(n.binds), len(binds) if binds else 0]
        n.boxes.extend(boxes)
        if binds:
            n.binds.extend(binds)
        n.instrs.append(r)
        n.types.append(rec[0])
        for aid, R, mode in accesses:
            if mode & M_READ:
                al = n.allocs[aid]
                al["readers"][iid] = al["readers"].get(iid, np.zeros_like(R)) | (R & al["mask"])
        for aid, R, mode in accesses:
            if mode & M_WRITE:
                al = n.allocs[aid]
                al["writers"][R & al["mask"]] = iid
                for x in list(al["readers"]):
                    al["readers"][x] = al["readers"][x] & ~R
                    if not al["readers"][x].any():
                        del al["readers"][x]
        return iid

    def _apply(self, n, h):
        for al in n.allocs:
            if not al["live"]:
                continue
            w = al["writers"]
            w[(w < h) & al["mask"]] = h
            merged = None
            for x in list(al["readers"]):
                if x < h:
                    merged = al["readers"].pop(x) if merged is None else merged | al["readers"].pop(x)
            if merged is not None:
                al["readers"][h] = al["readers"].get(h, np.zeros_like(merged)) | merged
        for b, (prod, pmem, mask) in n.bstate.items():
            sel = (prod < h) & (prod != NONE) & (prod != REMOTE)
            prod[sel] = h
        n.epoch = h

    def _new_alloc(self, n, b, m, box, writer, user=False):
        shape = self.bufs[b]["shape"]
        mk = box_mask(shape, box)
        w = np.full(shape, -1, dtype=np.int64)
        w[mk] = writer
        al = {"id": len(n.allocs), "buffer": b, "mem": m, "box": box, "mask": mk, "live": True,
              "user": user, "writers": w, "readers": {}}
        n.allocs.append(al)
        return al["id"]

    def _free_deps(self, n, al):
        deps = {}
        for w in np.unique(al["writers"][al["mask"]]):
            deps[int(w)] = deps.get(int(w), 0) | K_ALLOC
        for x in al["readers"]:
            deps[x] = deps.get(x, 0) | K_ALLOC
        return deps

    def _alloc_phase(self, n, it, look):
        nt = it["nt"]
        reqs = self._reqs(nt)
        keys = sorted({(b, m) for b, m, _ in reqs})
        for b, m in keys:
            shape = self.bufs[b]["shape"]
            cl = [{"mask": box_mask(shape, bbox_of_mask(mk)), "own": True, "abs": []}
                  for bb, mm, mk in reqs if bb == b and mm == m and self._find_alloc(n, b, m, mk) is None]
            if not cl:
                continue
            for q in look:
                for bb, mm, mk in self._reqs(q):
                    if bb == b and mm == m and self._find_alloc(n, b, m, mk) is None:
                        cl.append({"mask": box_mask(shape, bbox_of_mask(mk)), "own": False, "abs": []})
            changed = True
            while changed:
                changed = False
                for i in range(len(cl)):
                    for j in range(i + 1, len(cl)):
                        if (cl[i]["mask"] & cl[j]["mask"]).any():
                            u = cl[i]["mask"] | cl[j]["mask"]
                            cl[i] = {"mask": box_mask(shape, bbox_of_mask(u)), "own": cl[i]["own"] or cl[j]["own"],
                                     "abs": cl[i]["abs"] + cl[j]["abs"]}
                            del cl[j]
                            changed = True
                            break
                    if changed:
                        break
                if changed:
                    continue
                taken = {a for c in cl for a in c["abs"]}
                for c in cl:
                    for al in n.allocs:
                        if al["live"] and al["buffer"] == b and al["mem"] == m and al["id"] not in taken \
                                and (c["mask"] & al["mask"]).any():
                            u = c["mask"] | al["mask"]
                            c["mask"] = box_mask(shape, bbox_of_mask(u))
                            c["abs"].append(al["id"])
                            changed = True
                            break
                    if changed:
                        break
            mine = sorted([c for c in cl if c["own"]], key=lambda c: bbox_of_mask(c["mask"]))
            for c in mine:
                bb = bbox_of_mask(c["mask"])
                aid = len(n.allocs)
                iid = self._emit(n, [ALLOC, it["seq"], aid, m, b, NONE], [bb], [], {})
                self._new_alloc(n, b, m, bb, iid)
                prod, pmem, mask = n.bstate[b]
                for old in sorted(c["abs"]):
                    oal = n.allocs[old]
                    live = oal["mask"] & (((mask >> m) & 1) == 1)
                    if live.any():
                        self._emit(n, [COPY, it["seq"], old, aid, b, 1], [live],
                                   [(old, live, M_READ), (aid, live, M_WRITE)], {})
                    self._emit(n, [FREE, it["seq"], old, m, b, NONE], [], [], self._free_deps(n, oal))
                    oal["live"] = False

    def _coherence(self, n, seq, b, m, dst, need):
        prod, pmem, mask = n.bstate[b]
        stale = need & (((mask >> m) & 1) == 0) & (prod != NONE)
        assert not (stale & (prod == REMOTE)).any(), "read of remotely written data that was never received"
        keys = sorted({(int(p), int(q)) for p, q in zip(prod[stale], pmem[stale])})
        copied = np.zeros_like(need)
        for p, q in keys:
            g = stale & (prod == p) & (pmem == q)
            for al in list(n.allocs):
                if not al["live"] or al["buffer"] != b or al["mem"] != q:
                    continue
                part = g & al["mask"]
                if not part.any():
                    continue
                if self.stage_d2d and q >= 2 and m >= 2:
                    # through a fresh host allocation over the region's bounding box
                    bb = bbox_of_mask(part)
                    hid = len(n.allocs)
                    iid = self._emit(n, [ALLOC, seq, hid, 1, b, NONE], [bb], [], {})
                    self._new_alloc(n, b, 1, bb, iid)
                    self._emit(n, [COPY, seq, al["id"], hid, b, 0], [part],
                               [(al["id"], part, M_READ), (hid, part, M_WRITE)], {})
                    self._emit(n, [COPY, seq, hid, dst, b, 0], [part],
                               [(hid, part, M_READ), (dst, part, M_WRITE)], {})
                    h = n.allocs[hid]
                    self._emit(n, [FREE, seq, hid, 1, b, NONE], [], [], self._free_deps(n, h))
                    h["live"] = False
                else:
                    self._emit(n, [COPY, seq, al["id"], dst, b, 0], [part],
                               [(al["id"], part, M_READ), (dst, part, M_WRITE)], {})
                copied |= part
        mask[copied] |= (1 << m)

    def _compile(self, n, it, look):
        nt = it["nt"]
        task = nt["task"]
        seq = it["seq"]
        accs = task.accessors
        self._alloc_phase(n, it, look)
        for (b, t), P in sorted(nt["push"].items()):
            dst = self._find_alloc(n, b, 1, box_mask(P.shape, bbox_of_mask(P)))
            self._coherence(n, seq, b, 1, dst, P)
            prod, pmem, mask = n.bstate[b]
            keys = sorted({(int(p), int(q)) for p, q in zip(prod[P], pmem[P])})
            for p, q in keys:
                for bx in boxes_of(P & (prod == p) & (pmem == q)):
                    self._emit(n, [SEND, seq, dst, t, b, n.next_msg], [bx],
                               [(dst, box_mask(P.shape, bx), M_READ)], {})
                    n.next_msg += 1
        for b, W in sorted(nt["await"].items()):
            dst = self._find_alloc(n, b, 1, box_mask(W.shape, bbox_of_mask(W)))
            cons = []
            for ch in nt["chunks"]:
                for ai, a in enumerate(accs):
                    if a.buffer == b and (a.mode & M_READ):
                        r = ch["masks"][ai] & W
                        if r.any():
                            cons.append(r)
            whole = len(cons) <= 1 or all((r == W).all() for r in cons)
            prod, pmem, mask = n.bstate[b]
            if whole:
                iid = self._emit(n, [RECEIVE, seq, dst, NONE, b, NONE], [W], [(dst, W, M_WRITE)], {})
                prod[W], pmem[W], mask[W] = iid, 1, 2
            else:
                sid = self._emit(n, [SPLIT_RECEIVE, seq, dst, NONE, b, NONE], [W], [(dst, W, M_WRITE)], {})
                covered = np.zeros_like(W)
                for r in cons:
                    part = r & ~covered
                    if not part.any():
                        continue
                    aid = self._emit(n, [AWAIT_RECEIVE, seq, dst, sid, b, NONE], [part], [], {sid: K_DATAFLOW})
                    n.allocs[dst]["writers"][part] = aid
                    prod[part], pmem[part], mask[part] = aid, 1, 2
                    covered |= part
        for ch in nt["chunks"]:
            for ai, a in enumerate(accs):
                mk = ch["masks"][ai]
                if not (a.mode & M_READ) or not mk.any():
                    continue
                prod, pmem, mask = n.bstate[a.buffer]
                if (mk & (prod == NONE)).any():
                    n.diags.append([seq, ch["index"], ai])
                dst = self._find_alloc(n, a.buffer, ch["mem"], mk)
                self._coherence(n, seq, a.buffer, ch["mem"], dst, mk)
        for ch in nt["chunks"]:
            accesses, binds = [], []
            for ai, a in enumerate(accs):
                mk = ch["masks"][ai]
                if not mk.any():
                    binds.append([NONE, 0, 0, 0, 0, 0, 0])
                    continue
                al = self._find_alloc(n, a.buffer, ch["mem"], mk)
                binds.append([al] + list(bbox_of_mask(mk)))
                accesses.append((al, mk, a.mode))
            kid = self._emit(n, [KERNEL, seq, ch["index"], ch["mem"], task.kernel, NONE], [ch["box"]],
                             accesses, {}, binds)
            for ai, a in enumerate(accs):
                mk = ch["masks"][ai]
                if (a.mode & M_WRITE) and mk.any():
                    prod, pmem, mask = n.bstate[a.buffer]
                    prod[mk], pmem[mk], mask[mk] = kid, ch["mem"], 1 << ch["mem"]
        for ch in nt["remote"]:
            for ai, a in enumerate(accs):
                mk = ch["masks"][ai]
                if (a.mode & M_WRITE) and mk.any():
                    prod, pmem, mask = n.bstate[a.buffer]
                    prod[mk], pmem[mk], mask[mk] = REMOTE, 0, 0

    def _process(self, n, it, look):
        k = it["kind"]
        if k == "create":
            b = it["arg"]
            shape = self.bufs[b]["shape"]
            if self.bufs[b]["init"]:
                self._new_alloc(n, b, 0, (0, 0, 0) + shape, n.epoch, user=True)
                n.bstate[b] = (np.full(shape, n.epoch, dtype=np.int64), np.zeros(shape, dtype=np.int64),
                               np.full(shape, 1, dtype=np.int64))
            else:
                n.bstate[b] = (np.full(shape, NONE, dtype=np.int64), np.zeros(shape, dtype=np.int64),
                               np.zeros(shape, dtype=np.int64))
        elif k == "task":
            self._compile(n, it, look)
        elif k in ("horizon", "epoch"):
            fd = {f: K_FRONT for f in n.front}
            iid = self._emit(n, [EPOCH if k == "epoch" else HORIZON, it["seq"], NONE, NONE, NONE, NONE], [], [], fd)
            n.front = {iid}
            if k == "epoch":
                self._apply(n, iid)
                n.last_horizon = None
            else:
                if n.last_horizon is not None:
                    self._apply(n, n.last_horizon)
                n.last_horizon = iid
        elif k == "destroy":
            b = it["arg"]
            ids = sorted([al["id"] for al in n.allocs if al["live"] and al["buffer"] == b],
                         key=lambda i: (n.allocs[i]["mem"], i))
            for i in ids:
                al = n.allocs[i]
                if not al["user"]:
                    self._emit(n, [FREE, it["seq"], i, al["mem"], b, NONE], [], [], self._free_deps(n, al))
                al["live"] = False
            del n.bstate[b]

    def graph(self, node):
        n = self.nodes[node]

        def arr(x, w):
            return np.array(x, dtype=np.uint32).reshape(-1, w)
        return {"instrs": arr(n.instrs, 11), "edges": arr(n.edges, 3), "boxes": arr(n.boxes, 6),
                "binds": arr(n.binds, 7), "diags": arr(n.diags, 3)}
