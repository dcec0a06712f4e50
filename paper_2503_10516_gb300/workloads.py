"""Seeded synthetic programs for the lowering engine (inputs only).

This module describes programs — buffers, tasks with range-mapped accessors,
flushes — and draws their initial buffer contents from fixed seeds. It holds
none of the lowering arithmetic: chunking, mapper evaluation and everything
after it live in the CUDA engine and, separately, in the test oracle.

Shapes follow the paper's applications (Sec. 5): a 5-point stencil
(WaveSim), an all-pairs N-body step (Listing 1), and a buffer whose accessed
region grows row by row (RSim); plus Listing 2 and random small programs.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Tuple

import numpy as np

# Access modes (Sec. 2.1: read_only, write_only + no_init, read_write).
READ, WRITE, READ_WRITE = 1, 2, 3

# Workload kernels run by device-kernel instructions at execute time.
K_NOP, K_JACOBI, K_WAVE, K_NBODY_STEP, K_NBODY_UPDATE, K_GROW, K_GENERIC = 0, 1, 2, 3, 4, 5, 6
K_SHIFT = 7  # reads accessor 0 at item + (params 0-2 as int32), writes the value to accessor 1 at item

TASK_HDR = 11
ACC_W = 14
MAX_ACC = 8

# Lookahead values: a task-count window, or the paper's horizon-count
# heuristic (Sec. 4.3), or compile only at epochs.
LOOKAHEAD_HORIZONS = 0xFFFFFFFE
LOOKAHEAD_INFINITE = 0xFFFFFFFF

MapDim = Tuple[int, int, int, int]  # (kind, a, b, c): 0 affine(k, offset, radius), 1 all, 2 fixed[a, b)


def affine(k: int, offset: int = 0, radius: int = 0) -> MapDim:
    return (0, k, offset & 0xFFFFFFFF, radius)


def all_dim() -> MapDim:
    return (1, 0, 0, 0)


def fixed(lo: int, hi: int) -> MapDim:
    return (2, lo, hi, 0)


def one_to_one() -> List[MapDim]:
    return [affine(0), affine(1), affine(2)]


def neighborhood(*r: int) -> List[MapDim]:
    rr = list(r) + [r[-1]] * (3 - len(r))
    return [affine(0, 0, rr[0]), affine(1, 0, rr[1]), affine(2, 0, rr[2])]


def all_mapper() -> List[MapDim]:
    return [all_dim(), all_dim(), all_dim()]


def row_slice() -> List[MapDim]:
    return [affine(0), all_dim(), all_dim()]


def col_slice() -> List[MapDim]:
    return [all_dim(), affine(1), all_dim()]


def transposed() -> List[MapDim]:
    return [affine(1), affine(0), affine(2)]


def fixed_box(lo, hi) -> List[MapDim]:
    lo = list(lo) + [0] * (3 - len(lo))
    hi = list(hi) + [1] * (3 - len(hi))
    return [fixed(lo[d], hi[d]) for d in range(3)]


@dataclasses.dataclass
class Accessor:
    buffer: int
    mode: int
    mapper: List[MapDim]


@dataclasses.dataclass
class Task:
    dims: int
    range: Tuple[int, int, int]
    chunks: int
    kernel: int
    accessors: List[Accessor]
    params: Tuple[int, int, int, int] = (0, 0, 0, 0)

    def flat(self) -> np.ndarray:
        w = np.zeros(TASK_HDR + ACC_W * MAX_ACC, dtype=np.uint32)
        w[0] = self.dims
        w[1:4] = self.range
        w[4] = self.chunks
        w[5] = self.kernel
        w[6] = len(self.accessors)
        w[7:11] = self.params
        for i, a in enumerate(self.accessors):
            o = TASK_HDR + ACC_W * i
            w[o] = a.buffer
            w[o + 1] = a.mode
            for d in range(3):
                w[o + 2 + 4 * d: o + 6 + 4 * d] = a.mapper[d]
        return w


@dataclasses.dataclass
class Buffer:
    dims: int
    extent: Tuple[int, int, int]
    elem_size: int
    init: Optional[np.ndarray]  # host data (row-major, elem_size bytes per element) or None
    dtype: str = "f32"          # "f32", "f32x4" or "u32": how execute's kernels read it


@dataclasses.dataclass
class Program:
    """A program: configuration plus an ordered list of operations.

    ops entries: ("buffer", Buffer) | ("task", Task) | ("flush",) |
    ("destroy", buffer_id) | ("lookahead", L)
    """
    name: str
    nodes: int
    devices: int
    horizon_step: int
    lookahead: int
    ops: list
    stage_d2d: bool = False  # device-to-device copies staged in host memory
    horizon_cp: bool = False  # horizons by the task graph's critical path, not every horizon_step tasks

    @property
    def buffers(self) -> List[Buffer]:
        return [o[1] for o in self.ops if o[0] == "buffer"]

    @property
    def tasks(self) -> List[Task]:
        return [o[1] for o in self.ops if o[0] == "task"]


def f32_to_u32(x: float) -> int:
    return int(np.array([x], dtype=np.float32).view(np.uint32)[0])


def _uniform(rng, shape) -> np.ndarray:
    return rng.random(shape, dtype=np.float32)


# ---- the paper-shaped configurations ---------------------------------------

def jacobi_program(n: int = 256, steps: int = 8, nodes: int = 2, devices: int = 2, chunks: int = 4,
                   lookahead: int = 0, horizon_step: int = 4, seed: int = 0x5EED) -> Program:
    """5-point Jacobi on one n x n fp32 buffer plus an output buffer; buffers swap every step."""
    rng = np.random.default_rng(seed)
    a = Buffer(2, (n, n, 1), 4, _uniform(rng, (n, n)))
    b = Buffer(2, (n, n, 1), 4, None)
    ops = [("buffer", a), ("buffer", b)]
    src, dst = 0, 1
    for _ in range(steps):
        ops.append(("task", Task(2, (n, n, 1), chunks, K_JACOBI,
                                 [Accessor(src, READ, neighborhood(1)), Accessor(dst, WRITE, one_to_one())])))
        src, dst = dst, src
    ops.append(("flush",))
    return Program(f"jacobi{n}", nodes, devices, horizon_step, lookahead, ops)


def wave_program(n: int = 8192, steps: int = 1000, nodes: int = 4, devices: int = 4, chunks: int = 64,
                 lookahead: int = 8, horizon_step: int = 4, seed: int = 0x5EED + 1) -> Program:
    """WaveSim-shaped 2D wave stencil over three rotating n x n fp32 buffers."""
    rng = np.random.default_rng(seed)
    bufs = [Buffer(2, (n, n, 1), 4, _uniform(rng, (n, n))),
            Buffer(2, (n, n, 1), 4, _uniform(rng, (n, n))),
            Buffer(2, (n, n, 1), 4, None)]
    ops = [("buffer", b) for b in bufs]
    prev, cur, nxt = 0, 1, 2
    for _ in range(steps):
        ops.append(("task", Task(2, (n, n, 1), chunks, K_WAVE,
                                 [Accessor(prev, READ, one_to_one()), Accessor(cur, READ, neighborhood(1)),
                                  Accessor(nxt, WRITE, one_to_one())])))
        prev, cur, nxt = cur, nxt, prev
    ops.append(("flush",))
    return Program(f"wave{n}", nodes, devices, horizon_step, lookahead, ops)


def nbody_program(n: int = 1 << 20, steps: int = 200, nodes: int = 8, devices: int = 4, chunks: int = 128,
                  lookahead: int = 4, horizon_step: int = 4, seed: int = 0x5EED + 2) -> Program:
    """All-pairs N-body (Listing 1): positions and velocities as float4, two tasks per step."""
    rng = np.random.default_rng(seed)
    p = rng.standard_normal((n, 4), dtype=np.float32)
    p[:, 3] = 1.0
    v = rng.standard_normal((n, 4), dtype=np.float32) * np.float32(0.01)
    v[:, 3] = 0.0
    ops = [("buffer", Buffer(1, (n, 1, 1), 16, p, "f32x4")), ("buffer", Buffer(1, (n, 1, 1), 16, v, "f32x4"))]
    for _ in range(steps):
        ops.append(("task", Task(1, (n, 1, 1), chunks, K_NBODY_STEP,
                                 [Accessor(0, READ, all_mapper()), Accessor(1, READ_WRITE, one_to_one())])))
        ops.append(("task", Task(1, (n, 1, 1), chunks, K_NBODY_UPDATE,
                                 [Accessor(1, READ, one_to_one()), Accessor(0, READ_WRITE, one_to_one())])))
    ops.append(("flush",))
    return Program(f"nbody{n}", nodes, devices, horizon_step, lookahead, ops)


def growing_program(rows_max: int = 256, cols: int = 64, nodes: int = 1, devices: int = 2, chunks: int = 2,
                    lookahead: int = 0, horizon_step: int = 4, seed: int = 0x5EED + 4,
                    grow: Tuple[int, int] = (1, 64)) -> Program:
    """RSim-shaped growing access: each step appends rows after reading every earlier row."""
    rng = np.random.default_rng(seed)
    two_d = cols > 1
    ext = (rows_max, cols, 1) if two_d else (rows_max, 1, 1)
    buf = Buffer(2 if two_d else 1, ext, 4, None)
    ops = [("buffer", buf)]
    first = min(rows_max, int(rng.integers(grow[0], grow[1] + 1)))
    ops.append(("task", Task(buf.dims, (first, ext[1], 1), chunks, K_GROW,
                             [Accessor(0, WRITE, one_to_one())], params=(0, 0, 0, 0))))
    r = first
    while r < rows_max:
        add = min(rows_max - r, int(rng.integers(grow[0], grow[1] + 1)))
        # kernel range = the new rows; reads all earlier rows, writes the new ones
        t = Task(buf.dims, (add, ext[1], 1), chunks, K_GROW,
                 [Accessor(0, READ, fixed_box((0, 0), (r, ext[1]))),
                  Accessor(0, WRITE, [affine(0, r), affine(1), affine(2)])], params=(r, 0, 0, 0))
        ops.append(("task", t))
        r += add
    ops.append(("flush",))
    return Program(f"grow{rows_max}x{cols}", nodes, devices, horizon_step, lookahead, ops)


def served_streams(count: int = 64, seed: int = 0x5EED + 5, lookahead: int = 0,
                   max_elems: int = 1 << 27) -> List[Program]:
    """Growing-row program streams for served lowering: each has one fp32
    buffer, 2D (3 in 4 streams: 2048-8192 columns, 2048-16384 rows) or 1D
    (4096-16384 elements), at most max_elems elements; its accessed prefix
    grows by a random 1-64 rows per task (each task reads every earlier row).
    Stream 0 has the largest buffer, 16384 x 8192 = 2^27 elements. One node,
    two devices, two chunks per task."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        if i == 0:
            rows, cols = 16384, 8192
        elif rng.random() < 0.75:
            cols = int(rng.choice([2048, 4096, 8192]))
            rows = int(rng.choice([2048, 4096, 8192, 16384]))
        else:
            rows, cols = int(rng.choice([4096, 8192, 16384])), 1
        while rows * cols > max_elems:
            rows //= 2
        out.append(growing_program(rows_max=rows, cols=cols, devices=2, chunks=2, lookahead=lookahead,
                                   seed=int(seed * 1000 + i), grow=(1, 64)))
    return out


def listing2_program(n: int = 16, lookahead: int = 0, nodes: int = 1, devices: int = 1, chunks: int = 1) -> Program:
    """Listing 2: a one_to_one no_init write followed by a neighborhood({1,1}) read."""
    b = Buffer(2, (n, n, 1), 4, None, "u32")
    out = Buffer(2, (n, n, 1), 4, None, "u32")
    ops = [("buffer", b), ("buffer", out),
           ("task", Task(2, (n, n, 1), chunks, K_GENERIC, [Accessor(0, WRITE, one_to_one())])),
           ("task", Task(2, (n, n, 1), chunks, K_GENERIC,
                         [Accessor(0, READ, neighborhood(1, 1)), Accessor(1, WRITE, one_to_one())])),
           ("flush",)]
    return Program("listing2", nodes, devices, 4, lookahead, ops)


def nbody_example_program(n: int = 64, iterations: int = 4, lookahead: int = 0) -> Program:
    """The Sec. 3.6 worked example: N-body on 2 nodes x 2 devices, one chunk per device."""
    rng = np.random.default_rng(7)
    p = rng.standard_normal((n, 4), dtype=np.float32)
    v = rng.standard_normal((n, 4), dtype=np.float32)
    ops = [("buffer", Buffer(1, (n, 1, 1), 16, p, "f32x4")), ("buffer", Buffer(1, (n, 1, 1), 16, v, "f32x4"))]
    for _ in range(iterations):
        ops.append(("task", Task(1, (n, 1, 1), 4, K_NBODY_STEP,
                                 [Accessor(0, READ, all_mapper()), Accessor(1, READ_WRITE, one_to_one())])))
        ops.append(("task", Task(1, (n, 1, 1), 4, K_NBODY_UPDATE,
                                 [Accessor(1, READ, one_to_one()), Accessor(0, READ_WRITE, one_to_one())])))
    ops.append(("flush",))
    return Program("nbody_example", 2, 2, 2, lookahead, ops)


# ---- random small programs (brute-force and parity cases) ------------------

def random_program(seed: int, max_extent: int = 12, max_tasks: int = 10, allow_3d: bool = True,
                   allow_bad: bool = True, max_nodes: int = 3, max_devices: int = 2,
                   uninit_reads: bool = False, horizon_lookahead: bool = False, split2d: bool = False) -> Program:
    """A small random program over all mapper kinds.

    Writes go through one_to_one or transposed mappers only (injective), and a
    buffer written by a task is read by that task only through the same
    read_write accessor, so every task has a well-defined sequential meaning.
    Buffers without host data are written before they are read unless
    ``uninit_reads``. With ``allow_bad`` a few tasks carry overlapping writes
    (an all-mapper write) and must be rejected. With ``split2d`` most tasks of
    two or more dimensions are split along dims 0 and 1 (1-3 chunks each; the
    column count in num_chunks' high 16 bits).
    """
    rng = np.random.default_rng(seed)
    nodes = int(rng.integers(1, max_nodes + 1))
    devices = int(rng.integers(1, max_devices + 1))
    hstep = int(rng.integers(1, 5))
    look = int(rng.choice([0, 0, 1, 2, 4, 0xFFFFFFFF]))
    if horizon_lookahead:
        look = int(rng.choice([LOOKAHEAD_HORIZONS, LOOKAHEAD_HORIZONS, 0, 2]))
    ops = []
    bufs: List[Buffer] = []
    written = []
    nb = int(rng.integers(1, 4))
    for _ in range(nb):
        dims = int(rng.choice([1, 2, 2, 3] if allow_3d else [1, 2, 2]))
        hi = max_extent if dims < 3 else max(2, max_extent // 2)
        ext = [int(rng.integers(1, hi + 1)) for _ in range(dims)] + [1] * (3 - dims)
        has_init = bool(rng.random() < 0.6)
        init = rng.integers(0, 2**32, size=int(np.prod(ext)), dtype=np.uint64).astype(np.uint32) if has_init else None
        b = Buffer(dims, tuple(ext), 4, init, "u32")
        bufs.append(b)
        written.append(has_init)
        ops.append(("buffer", b))
    ntasks = int(rng.integers(1, max_tasks + 1))
    for _ in range(ntasks):
        r = rng.random()
        if r < 0.05:
            ops.append(("flush",))
            continue
        if r < 0.08:
            choices = [0, 1, 3, 0xFFFFFFFF] + ([LOOKAHEAD_HORIZONS] * 3 if horizon_lookahead else [])
            ops.append(("lookahead", int(rng.choice(choices))))
            continue
        # pick the written buffer
        wb = int(rng.integers(0, len(bufs)))
        B = bufs[wb]
        trans = B.dims == 2 and rng.random() < 0.2
        ext = list(B.extent)
        kr = [ext[1], ext[0], 1] if trans else list(ext)
        if rng.random() < 0.3:
            kr = [int(rng.integers(1, kr[d] + 1)) if d < B.dims else 1 for d in range(3)]
        kdims = B.dims
        chunks = int(rng.integers(1, 7))
        if split2d and kdims >= 2 and rng.random() < 0.7:
            chunks = int(rng.integers(1, 4)) | (int(rng.integers(1, 4)) << 16)
        accs = []
        cy, cx = chunks & 0xFFFF, chunks >> 16
        # an overlapping write needs two non-empty chunks
        bad = allow_bad and rng.random() < 0.06 and ((cy > 1 and kr[0] > 1) or (cx > 1 and kr[1] > 1))
        rw = (not trans) and written[wb] and rng.random() < 0.4
        if bad:
            accs.append(Accessor(wb, WRITE, all_mapper()))
        else:
            accs.append(Accessor(wb, READ_WRITE if rw else WRITE, transposed() if trans else one_to_one()))
        nread = int(rng.integers(0, 3))
        for _ in range(nread):
            rb = int(rng.integers(0, len(bufs)))
            if rb == wb:
                continue
            if not written[rb] and not uninit_reads:
                continue
            Rb = bufs[rb]
            kind = rng.random()
            if kind < 0.25:
                m = one_to_one()
            elif kind < 0.5:
                m = neighborhood(*[int(x) for x in rng.integers(1, 3, size=3)])
            elif kind < 0.6:
                m = all_mapper()
            elif kind < 0.7:
                lo = [int(rng.integers(0, Rb.extent[d])) for d in range(3)]
                hi = [int(rng.integers(lo[d] + 1, Rb.extent[d] + 2)) for d in range(3)]
                m = [fixed(lo[d], hi[d]) for d in range(3)]
            elif kind < 0.8:
                m = row_slice()
            elif kind < 0.9:
                m = col_slice()
            else:
                m = transposed()
            accs.append(Accessor(rb, READ, m))
        ops.append(("task", Task(kdims, tuple(kr), chunks, K_GENERIC, accs)))
        if not bad and not trans and kr[:B.dims] == ext[:B.dims]:
            written[wb] = True
        elif not bad:
            # partial or transposed writes: count as initialised only if they cover the buffer
            if trans and kr[0] == ext[1] and kr[1] == ext[0]:
                written[wb] = True
        if rng.random() < 0.05 and len(bufs) > 1:
            d = len(bufs) - 1
            if all(o[0] != "destroy" or o[1] != d for o in ops):
                ops.append(("destroy", d))
                break
    ops.append(("flush",))
    return Program(f"random{seed}", nodes, devices, hstep, look, ops)


def batch_programs(count: int = 512, seed: int = 0x5EED + 3, max_tasks: int = 2000, scale: float = 1.0) -> List[Program]:
    """Uneven batch: 1-8 buffers of mixed 1D/2D/3D shape, 2^10-2^24 elements,
    1-128 chunks, 2-32 virtual memories, lookahead 0-16. ``scale`` shrinks the
    task counts for quick runs."""
    rng = np.random.default_rng(seed)
    progs = []
    for p in range(count):
        sub = int(rng.integers(0, 2**31))
        r = np.random.default_rng(sub)
        M = int(r.integers(2, 33))
        devices = int(r.choice([d for d in (1, 2, 4, 8) if d <= M]))
        nodes = max(1, M // devices)
        nbuf = int(r.integers(1, 9))
        ops = []
        shapes = []
        for _ in range(nbuf):
            dims = int(r.integers(1, 4))
            logn = int(r.integers(10, 25))
            if dims == 1:
                ext = (1 << logn, 1, 1)
            elif dims == 2:
                a = logn // 2
                ext = (1 << a, 1 << (logn - a), 1)
            else:
                a = logn // 3
                b = (logn - a) // 2
                ext = (1 << a, 1 << b, 1 << (logn - a - b))
            shapes.append((dims, ext))
            ops.append(("buffer", Buffer(dims, ext, 4, None, "u32")))
        ntasks = max(2, int(int(r.integers(10, max_tasks + 1)) * scale))
        chunks = int(r.integers(1, 129))
        written = [False] * nbuf
        for _ in range(ntasks):
            wb = int(r.integers(0, nbuf))
            dims, ext = shapes[wb]
            accs = [Accessor(wb, WRITE if not written[wb] else int(r.choice([WRITE, READ_WRITE])), one_to_one())]
            for _ in range(int(r.integers(0, 3))):
                rb = int(r.integers(0, nbuf))
                if rb == wb or not written[rb]:
                    continue
                kind = r.random()
                if kind < 0.3:
                    m = one_to_one()
                elif kind < 0.6:
                    m = neighborhood(int(r.integers(1, 5)))
                elif kind < 0.7:
                    m = row_slice()
                elif kind < 0.8:
                    m = col_slice()
                elif kind < 0.9:
                    m = transposed()
                else:
                    m = all_mapper()
                accs.append(Accessor(rb, READ, m))
            ops.append(("task", Task(dims, ext, chunks, K_GENERIC, accs)))
            written[wb] = True
        ops.append(("flush",))
        progs.append(Program(f"batch{p}", nodes, devices, 4, int(r.integers(0, 17)), ops))
    return progs
