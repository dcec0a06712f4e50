"""Benchmark: instruction-graph lowering + execution of the 2D wave-stencil program.

Workload (one step): the WaveSim-shaped program over three rotating
8192 x 8192 fp32 buffers, 4 virtual nodes x 4 devices, 64 row chunks, 1000
time steps, lookahead 8, horizon every 4 tasks. A step lowers the whole
program on the GPU (batched: every node's warp lowers all 1000 tasks in one
launch) and executes every emitted instruction (allocations, coherence and
send/receive box copies, the stencil kernels).

Prints one JSON line. --impl reference times the CPU oracle (test
infrastructure) on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2503_10516_gb300 import workloads as W  # noqa: E402

METRIC = "instructions lowered/s"
UNIT = "instructions/s"
N, STEPS, NODES, DEVICES, CHUNKS, LOOKAHEAD, HSTEP = 8192, 1000, 4, 4, 64, 8, 4
WINDOW = 16  # the executor takes new instructions once every node has lowered this many more submissions
MAP_ENTRY_BYTES = 28.0  # algorithmic bytes of one region-map entry: six uint32 box coordinates + one uint32 value
WORKLOAD = (f"wave2d: 3 x {N}x{N} fp32 buffers rotating, {NODES} nodes x {DEVICES} devices, {CHUNKS} row chunks, "
            f"{STEPS} time steps, lookahead {LOOKAHEAD}, horizon every {HSTEP} tasks")


LOWER_PROFILE = os.path.join(ROOT, "profiles", "lower_kernel_wave8192_64tasks.md")
LOWER_SOURCES = [os.path.join(ROOT, "paper_2503_10516_gb300", "csrc", f) for f in ("igs_lower.cu", "igs_internal.h")]


def lowering_source_sha() -> str:
    """First 16 hex digits of the SHA-256 of the lowering kernel's sources."""
    h = hashlib.sha256()
    for f in LOWER_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _lowering_profile():
    """Figures of the committed ncu capture of the lowering kernel (one launch
    over 64 wave tasks): `key: value` lines of its summary. None when the
    summary is missing or the kernel's sources changed since the capture."""
    try:
        with open(LOWER_PROFILE) as f:
            lines = f.read().splitlines()
    except OSError:
        return None
    vals = {}
    for line in lines:
        if line.startswith("- `") and "`: " in line:
            k, v = line[3:].split("`: ", 1)
            vals[k.strip()] = v.strip().split()[0]
    if vals.get("source_sha256_16") != lowering_source_sha():
        return None
    return vals


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def __enter__(self):
        def run():
            q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap")
            while not self._stop.is_set():
                try:
                    out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits"], capture_output=True, text=True,
                                         timeout=5).stdout.strip()
                    if out:
                        self.samples.append([x.strip() for x in out.split(",")])
                except Exception:
                    pass
                self._stop.wait(0.2)
        self._t = threading.Thread(target=run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if len(s) > 3 + k and s[3 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def _program(with_data: bool = True):
    return W.wave_program(n=N, steps=STEPS, nodes=NODES, devices=DEVICES, chunks=CHUNKS, lookahead=LOOKAHEAD,
                          horizon_step=HSTEP) if with_data else None


def _program_shape():
    """The same program with tiny data arrays: lowering depends on shapes only."""
    p = W.wave_program(n=8, steps=STEPS, nodes=NODES, devices=DEVICES, chunks=CHUNKS, lookahead=LOOKAHEAD,
                       horizon_step=HSTEP)
    for op in p.ops:
        if op[0] == "buffer":
            op[1].extent = (N, N, 1)
        elif op[0] == "task":
            op[1].range = (N, N, 1)
    return p


def _oracle_lower(prog) -> int:
    """Lowers a program with the CPU oracle; returns the instruction count."""
    import oracle
    o = oracle.Oracle(prog.nodes, prog.devices, prog.horizon_step, prog.lookahead)
    for op in prog.ops:
        if op[0] == "buffer":
            b = op[1]
            o.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init is not None)
        elif op[0] == "task":
            o.submit(op[1].flat())
        elif op[0] == "flush":
            o.flush()
    n = sum(len(o.graph(k)["instrs"]) for k in range(prog.nodes))
    o.close()
    return n


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    prog = _program_shape()
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        _oracle_lower(prog)
    t0 = time.perf_counter()
    total = 0
    for _ in range(args.steps):
        total += _oracle_lower(prog)
    dt = time.perf_counter() - t0
    value = total / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "what": "CPU oracle lowering of the whole program, single thread"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"whole program lowering ({STEPS} tasks, all {NODES} nodes), no execution"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _stage_ctx(igs, prog, mode, stream):
    flags = (igs.FLAG_HORIZON_CP if prog.horizon_cp else 0) | (igs.FLAG_STAGE_D2D if prog.stage_d2d else 0)
    c = igs.Context(prog.nodes, prog.devices, prog.horizon_step, prog.lookahead, mode=mode, stream=stream,
                    flags=flags, **igs.small_caps(prog))
    for op in prog.ops:
        if op[0] == "buffer":
            b = op[1]
            c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
    return c


def _submit_program(c, p):
    for op in p.ops:
        if op[0] == "task":
            c.submit(op[1])
        elif op[0] == "flush":
            c.submit_epoch()


def _full_scale_caps(igs, small, full, stream, margin=3.0):
    """Capacities for each full-scale program: its prefix at a small task
    scale is lowered first (its tasks are the first tasks of the full
    program); the largest per-node instruction, edge and box counts (binds
    count half: two per instruction are provided) are extrapolated by the
    task ratio, with a margin."""
    ctxs = [_stage_ctx(igs, p, igs.MODE_BATCHED, stream) for p in small]
    for p, c in zip(small, ctxs):
        _submit_program(c, p)
    igs.lower_batch(ctxs)
    caps = []
    for ps, pf, c in zip(small, full, ctxs):
        k = len(pf.tasks) / max(1, len(ps.tasks))
        mx = {"instrs": 0, "edges": 0, "boxes": 0}
        for n in range(ps.nodes):
            g = c.graph(n)
            mx["instrs"] = max(mx["instrs"], len(g["instrs"]), (len(g["binds"]) + 1) // 2)
            mx["edges"] = max(mx["edges"], len(g["edges"]))
            mx["boxes"] = max(mx["boxes"], len(g["boxes"]))
        caps.append(igs.small_caps(pf, {key: v * k * margin + 64 for key, v in mx.items()}))
        c.close()
    return caps


def _doubled(cp, factor=2.0):
    """Capacities grown after a shortfall: the output arrays by `factor`, the
    region-map heap, scratch tables, allocations and queue doubled."""
    out = dict(cp)
    for k in ("max_instructions", "max_edges", "max_boxes"):
        out[k] = int(factor * cp[k])
    for k in ("map_heap", "scratch_capacity", "max_live_allocs", "max_allocations", "max_queue"):
        if k in cp:
            out[k] = 2 * cp[k]
    return out


def measure_batched(igs, torch, stream, count=512, scale=1.0, tune_scale=0.02, subset_every=16):
    """The 512 uneven programs of W.batch_programs (1-8 buffers of 2^10-2^24
    elements, 1-128 chunks, 2-32 memories, lookahead 0-16, 10-2000 tasks) at
    full task counts, lowered in one launch (igs_lower_batch_shaped). The
    launch shape is tuned on the same programs at 2 % of their tasks (timing
    every candidate on fresh copies). One task per launch (plain) is timed on
    every 16th program, against one batched launch of the same programs."""
    full = W.batch_programs(count=count, scale=scale, seed=0x5EED + 3)
    caps = _full_scale_caps(igs, W.batch_programs(count=count, scale=0.01, seed=0x5EED + 3), full, stream)
    res = {"programs": count, "task_scale": scale, "tasks": sum(len(p.tasks) for p in full),
           "units": sum(p.nodes for p in full)}

    def timer():
        torch.cuda.synchronize()
        return time.perf_counter()

    tune_progs = W.batch_programs(count=count, scale=tune_scale, seed=0x5EED + 3)

    def staged():
        ctxs = [_stage_ctx(igs, p, igs.MODE_BATCHED, stream) for p in tune_progs]
        for p, c in zip(tune_progs, ctxs):
            _submit_program(c, p)
        return ctxs

    t_tune = time.perf_counter()
    cands = igs.batch_shape_candidates(res["units"], torch.cuda.get_device_properties(0).multi_processor_count)
    shape, times = igs.tune_lower_batch(staged, cands, timer)
    res["tuning"] = {"task_scale": tune_scale, "seconds": time.perf_counter() - t_tune, "chosen": shape,
                     "launch_seconds": [{"shape": s_, "seconds": t_} for s_, t_ in times]}

    def stage(progs, cps, mode):
        ctxs = [igs.Context(p.nodes, p.devices, p.horizon_step, p.lookahead, mode=mode, stream=stream, **cp)
                for p, cp in zip(progs, cps)]
        for p, c in zip(progs, ctxs):
            for op in p.ops:
                if op[0] == "buffer":
                    b = op[1]
                    c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
        return ctxs

    shortfalls = []

    def batched_run(progs, cps, shp, attempts=3):
        """One launch over all programs. A context whose capacity estimate fell
        short gets larger capacities (its outputs scaled by the share of its
        items it lowered, at most 8x; heap and scratch doubled) and the launch
        is repeated; after the last attempt, programs still short (or whose
        context cannot be created) are left out and named. Only the launch that
        completes is timed."""
        active = list(range(len(progs)))
        excluded = []
        for attempt in range(attempts):
            ctxs, made = [], []
            for i in active:
                try:
                    ctxs.append(stage([progs[i]], [cps[i]], igs.MODE_BATCHED)[0])
                    made.append(i)
                except igs.IgsError as e:
                    excluded.append({"program": progs[i].name, "why": str(e)[:120]})
            active = made
            for i, c in zip(active, ctxs):
                c.set_item_times(True)  # how far a context got if a capacity falls short
                _submit_program(c, progs[i])
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                igs.lower_batch(ctxs, shp)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
            except igs.IgsError:
                grow = {}
                for i, c in zip(active, ctxs):
                    _, ts = c.item_times()
                    done = float(np.mean(ts > 0)) if len(ts) else 0.0
                    try:
                        c.sync()
                    except igs.IgsError as e:
                        grow[i] = max(2.0, min(8.0, 1.5 / max(done, 1e-3)))
                        shortfalls.append(str(e).split(": ", 2)[-1])
                for c in ctxs:
                    c.close()
                for i, f in grow.items():
                    cps[i] = _doubled(cps[i], f)
                if attempt == attempts - 1:
                    break
                if attempt == attempts - 2:  # the last attempt runs without the programs still short
                    keep = [i for i in active if i not in grow]
                    excluded += [{"program": progs[i].name, "why": "capacity estimate short twice"} for i in grow]
                    active = keep
                continue
            instrs = sum(int(c.counters()["instructions"]) for c in ctxs)
            launches = sum(int(c.counters()["launches"]) for c in ctxs)
            for c in ctxs:
                c.close()
            tasks = sum(len(progs[i].tasks) for i in active)
            return {"instr_per_s": instrs / dt, "tasks_per_s": tasks / dt, "seconds": dt, "instructions": instrs,
                    "launches": launches, "attempts": attempt + 1, "programs_lowered": len(active),
                    "tasks_lowered": tasks, "excluded": excluded, "capacity_shortfalls_before": shortfalls[:8]}
        return {"error": f"capacity estimates still short after {attempts} attempts", "shortfalls": shortfalls[:8],
                "excluded": excluded}

    res["batched_all"] = batched_run(full, caps, shape)
    sub = list(range(0, count, subset_every))
    sp, sc = [full[i] for i in sub], [caps[i] for i in sub]
    sb = batched_run(sp, sc, shape)
    gone = {e["program"] for e in sb.get("excluded", [])}
    keep = [k for k, p in enumerate(sp) if p.name not in gone]
    sp, sc = [sp[k] for k in keep], [sc[k] for k in keep]
    res["subset"] = {"programs": len(sp), "tasks": sum(len(p.tasks) for p in sp), "batched": sb}
    # one task per launch, each program after the other (a program whose
    # capacities fall short is repeated with doubled ones; only the run that
    # completes is timed)
    dt, instrs, launches = 0.0, 0, 0
    for i, p in enumerate(sp):
        for _ in range(4):
            c = stage([p], [sc[i]], igs.MODE_PLAIN)[0]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            try:
                _submit_program(c, p)
                c.sync()
            except igs.IgsError:
                c.close()
                sc[i] = _doubled(sc[i])
                continue
            torch.cuda.synchronize()
            dt += time.perf_counter() - t0
            instrs += int(c.counters()["instructions"])
            launches += int(c.counters()["launches"])
            c.close()
            break
    res["subset"]["plain"] = {"instr_per_s": instrs / dt, "seconds": dt, "instructions": instrs,
                              "launches": launches}
    res["subset"]["speedup"] = res["subset"]["batched"]["instr_per_s"] / res["subset"]["plain"]["instr_per_s"]
    return res


def _trace(progs, rate, seed):
    """Poisson arrivals at `rate` over a seeded interleaving of the streams'
    submissions (each stream keeps its order): [(stream, task or None, ns)]."""
    rng = np.random.default_rng(seed)
    order = []
    for i, p in enumerate(progs):
        for op in p.ops:
            if op[0] in ("task", "flush"):
                order.append(i)
    rng.shuffle(order)
    bodies = [[op for op in p.ops if op[0] in ("task", "flush")] for p in progs]
    pos = [0] * len(progs)
    t = np.cumsum(rng.exponential(1.0 / rate, size=len(order))) * 1e9
    trace = []
    for k, i in enumerate(order):
        op = bodies[i][pos[i]]
        pos[i] += 1
        trace.append((i, op[1] if op[0] == "task" else None, int(t[k])))
    return trace


def _lat_summary(lat_ns, wall_ns, instrs):
    lat = np.sort(np.asarray(lat_ns, dtype=np.float64)) * 1e-6
    n = len(lat)
    return {"p50_ms": float(lat[n // 2]), "p99_ms": float(lat[min(n - 1, int(n * 0.99))]), "items": n,
            "wall_s": wall_ns * 1e-9, "items_per_s": n / (wall_ns * 1e-9), "instructions": instrs,
            "instr_per_s": instrs / (wall_ns * 1e-9)}


def measure_served(igs, torch, stream, streams=64, budget=150e9, rates=(1e4, 1e5, 1e6),
                   lookaheads=(("L0", 0), ("L8", 8), ("Linf", W.LOOKAHEAD_INFINITE))):
    """Served lowering of 64 growing-row program streams (W.served_streams:
    fp32 buffers of up to 2^27 elements, prefix growing 1-64 rows per task)
    with Poisson arrivals at 1e4 / 1e5 / 1e6 tasks/s, lookahead 0, 8 and
    unbounded. Streams are admitted under a 150 GB HBM budget
    (igs_serve_enqueue) and detached when their last item is taken; latency =
    arrival -> every node has taken the item. The comparator replays the
    same arrivals with one lowering launch per item (igs_replay_plain), both
    from the library's own host loop. A slot-limited run (16 slots for the 64
    streams) shows continuous batching: streams wait for admission and are
    admitted as others detach."""
    out = {"workload": f"{streams} growing-row streams (1D / 2D fp32, up to 2^27 elements, +1-64 rows per task), "
                       f"1 node x 2 devices, 2 chunks; {budget / 1e9:.0f} GB admission budget"}

    def run_served(progs, trace, max_slots, hbm):
        srv = igs.Server(max_slots=max_slots, hbm_budget_bytes=int(hbm))
        ctxs = [_stage_ctx(igs, p, igs.MODE_PLAIN, None) for p in progs]
        admitted = sum(1 for c, p in zip(ctxs, progs) if srv.enqueue(c, 4 * len(p.ops) + 16))
        srv.start()
        lat, wall = srv.replay(ctxs, trace, timeout_ms=300000, detach=True)
        st = srv.stats()
        srv.stop()
        instrs = sum(int(c.counters()["instructions"]) for c in ctxs)
        resizes = 0
        for c in ctxs:  # resize copies: copies within one memory (d = 1)
            g = c.graph(0)
            resizes += int(((g["instrs"][:, 1] == 4) & (g["instrs"][:, 6] == 1)).sum())
        for c in ctxs:
            c.close()
        srv.close()
        res = _lat_summary(lat, wall, instrs)
        res.update({"admitted_at_once": admitted, "admitted_after_detach": st["admitted_from_queue"],
                    "peak_waiting": st["peak_waiting"], "slots": max_slots, "resize_copies": resizes})
        return res

    for lname, L in lookaheads:
        progs = W.served_streams(count=streams, lookahead=L)
        res = {"tasks": sum(len(p.tasks) for p in progs)}
        for rate in rates:
            trace = _trace(progs, rate, seed=0x5EED + 5)
            r = {"served": run_served(progs, trace, max(64, 2 * streams), budget)}
            if L == 0:
                ctxs = [_stage_ctx(igs, p, igs.MODE_PLAIN, None) for p in progs]
                lat, wall = igs.replay_plain(ctxs, trace, timeout_ms=600000)
                instrs = sum(int(c.counters()["instructions"]) for c in ctxs)
                for c in ctxs:
                    c.close()
                r["plain"] = _lat_summary(lat, wall, instrs)
            res[f"{int(rate)}_per_s"] = r
        out[lname] = res
    # the paper's lookahead heuristic (compile two horizons after the last
    # allocating task) with horizons every 4 tasks vs by the task graph's
    # critical path (Sec. 3.5, Sec. 4.3), at 1e5 tasks/s
    for lname, cp in (("Lhorizons_count_cadence", False), ("Lhorizons_critical_path", True)):
        progs = W.served_streams(count=streams, lookahead=W.LOOKAHEAD_HORIZONS)
        for p in progs:
            p.horizon_cp = cp
        out[lname] = {"tasks": sum(len(p.tasks) for p in progs),
                      "100000_per_s": {"served": run_served(progs, _trace(progs, 1e5, seed=0x5EED + 5),
                                                            max(64, 2 * streams), budget)}}
    # continuous batching: fewer slots than streams
    progs = W.served_streams(count=streams, lookahead=8)
    out["continuous_batching_16_slots_1e5_per_s_L8"] = run_served(progs, _trace(progs, 1e5, seed=0x5EED + 5), 16,
                                                                  budget)
    return out


def measure_resize_execution(igs, torch, stream):
    """Resize copies of the growing-row pattern carried out by the box-copy
    kernel: the largest served stream (16384 x 8192 fp32 = 2^27 elements,
    rows appended 1-64 per task, 2 devices) lowered with lookahead 8 and
    executed; and lookahead 0 on a quarter of the rows (2^25 elements; at
    2^27 its resize copies would move ~260 GB). Copy GB/s = bytes read +
    written by the executor's box-copy launches / their event time."""
    out = {}
    for name, rows, L in (("L8_2^27", 16384, 8), ("L0_2^25", 4096, 0)):
        p = W.growing_program(rows_max=rows, cols=8192, devices=2, chunks=2, lookahead=L,
                              seed=int((0x5EED + 5) * 1000), grow=(1, 64))
        c = _stage_ctx(igs, p, igs.MODE_BATCHED, stream)
        c.set_timing(True)
        for op in p.ops:
            if op[0] == "task":
                c.submit(op[1])
        c.flush()
        g = c.graph(0)
        t = g["instrs"][:, 1]
        resizes = int(((t == 4) & (g["instrs"][:, 6] == 1)).sum())
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.execute()
        dt = time.perf_counter() - t0
        st = c.stats()
        c.close()
        gbs = st["copy_bytes"] / (st["copy_ms"] * 1e-3) / 1e9 if st["copy_ms"] else None
        out[name] = {"tasks": len(p.tasks), "resize_copies": resizes, "copy_bytes": st["copy_bytes"],
                     "copy_ms": st["copy_ms"], "copy_gbs": gbs, "copy_launches": st["copy_launches"],
                     "execute_s": dt}
    return out


def measure_box_copy(igs, torch, stream, reps=20):
    """Resize-shaped box copies of 2^27 fp32 elements (512 MiB, the largest
    growing allocation's live data): rows [0, 8192) x cols [0, 16384) from the
    old allocation into a new one, either with the same row pitch (one
    contiguous run) or growing along the fastest dimension (16384 -> 16448
    columns: one strided run per row). Bytes = read + written; inputs exceed L2."""
    rows, cols, grow = 8192, 16384, 64
    out = {}
    src = torch.empty(rows * cols, dtype=torch.float32, device="cuda")
    src.copy_(torch.arange(rows * cols, dtype=torch.float32, device="cuda"))
    for name, dcols in (("contiguous", cols), ("pitched", cols + grow)):
        dst = torch.zeros(rows * dcols, dtype=torch.float32, device="cuda")
        job = (src.data_ptr(), (0, 0, 0, rows, cols, 1), dst.data_ptr(), (0, 0, 0, rows, dcols, 1),
               (0, 0, 0, rows, cols, 1), 4)
        for _ in range(3):
            igs.box_copy([job], stream.cuda_stream)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(reps):
            igs.box_copy([job], stream.cuda_stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1) / reps
        byts = 2.0 * rows * cols * 4
        ok = bool(torch.equal(dst.view(rows, dcols)[:, :cols], src.view(rows, cols)))
        out[name] = {"ms": ms, "bytes": byts, "gbs": byts / (ms * 1e-3) / 1e9, "checked": ok}
        del dst
    del src
    return out


def measure_executors(igs, torch, stream, prog, make_ctx, wave_tasks=200, nbody_n=1 << 16, nbody_steps=10):
    """Execution alone (each graph fully lowered first) on the level executor
    and on the dataflow executor: the first `wave_tasks` tasks of the wave
    program, and N-body (nbody_n bodies, 8 nodes x 4 devices, 128 chunks,
    lookahead 4). Then the whole bench step (igs_run) on each executor. The
    dataflow executor's node timestamps give the copy / kernel overlap (a
    separate run with timing on)."""
    wave = W.Program("wave-head", NODES, DEVICES, HSTEP, LOOKAHEAD,
                     [op for op in prog.ops if op[0] == "buffer"] + [("task", t) for t in prog.tasks[:wave_tasks]]
                     + [("flush",)])
    nbody = W.nbody_program(n=nbody_n, steps=nbody_steps, nodes=8, devices=4, chunks=128, lookahead=4)
    out = {}
    for name, p in ((f"wave{N}_{wave_tasks}_tasks", wave), (f"nbody{nbody_n}_{nbody_steps}_steps", nbody)):
        res = {}
        for ex_name, ex in (("levels", igs.EXEC_LEVELS), ("dataflow", igs.EXEC_DATAFLOW)):
            times = []
            for rep in range(3 if ex == igs.EXEC_DATAFLOW else 2):
                c = igs.Context(p.nodes, p.devices, p.horizon_step, p.lookahead, mode=igs.MODE_BATCHED, stream=stream)
                c.set_executor(ex)
                timing = rep == 2
                c.set_timing(timing)
                for op in p.ops:
                    if op[0] == "buffer":
                        b = op[1]
                        c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
                    elif op[0] == "task":
                        c.submit(op[1])
                c.flush()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                c.execute()
                dt = time.perf_counter() - t0
                instrs = int(c.counters()["instructions"])
                if timing:
                    res["dataflow_stats"] = c.exec_stats()
                else:
                    times.append(dt)
                c.close()
            res[ex_name] = {"execute_ms": min(times[1:] or times) * 1e3, "instructions": instrs,
                            "instr_per_s": instrs / min(times[1:] or times)}
        res["speedup"] = res["levels"]["execute_ms"] / res["dataflow"]["execute_ms"]
        out[name] = res
    # the whole bench step on each executor
    step = {}
    for ex_name, ex in (("levels", igs.EXEC_LEVELS), ("dataflow", igs.EXEC_DATAFLOW)):
        ts = []
        for _ in range(2):
            c = make_ctx(timing=False)
            c.set_executor(ex)
            for t in prog.tasks:
                c.submit(t)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            c.run(WINDOW)
            ts.append(time.perf_counter() - t0)
            c.close()
        step[ex_name] = {"ms": min(ts) * 1e3}
    out["bench_step"] = step
    return out


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(len(xs) * q))] if xs else None


def lowering_modes(igs, torch, stream, prog, init_zero=False):
    """One program lowered two ways, without execution: batched (one launch
    over every submission: warp 0 per node, its helper warps and the front
    warp) and plain (one launch per submission, each waited for). Batched
    per-task time = the task's completion minus the previous item's (device
    clock, igs_item_times; a task's horizon counts with it); plain
    per-task time = the launch's event time. Both instr/s by wall clock
    around the whole lowering (plain's includes its launch and sync costs)."""
    out = {}
    for name, mode in (("batched", igs.MODE_BATCHED), ("plain", igs.MODE_PLAIN)):
        c = igs.Context(prog.nodes, prog.devices, prog.horizon_step, prog.lookahead, mode=mode, stream=stream)
        c.set_timing(True)
        if mode == igs.MODE_BATCHED:
            c.set_item_times(True)
        for op in prog.ops:
            if op[0] == "buffer":
                b = op[1]
                init = b.init
                if init_zero and init is not None:
                    init = np.zeros(tuple(b.extent[:b.dims]) + ((4,) if b.elem_size == 16 else ()), np.float32)
                c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, init)
        c.sync()
        lat = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for op in prog.ops:
            if op[0] == "task":
                c.submit(op[1])
                if mode == igs.MODE_PLAIN:
                    lat.append(c.stats()["last_lower_ms"])
        c.flush()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        st = c.stats()
        instrs = int(c.counters()["instructions"])
        if mode == igs.MODE_BATCHED:
            # a task's group = the task and the items after it up to the next
            # task (its horizon), as one launch of plain mode lowers them
            kinds, ts = c.item_times()
            ends = []
            for k, t in zip(kinds, ts.astype(np.int64)):
                if k == 1:
                    ends.append(t)
                elif ends and k == 2:
                    ends[-1] = t
            lat = [(b - a) * 1e-6 for a, b in zip(ends, ends[1:])]
        c.close()
        out[name] = {"instructions": instrs, "wall_s": wall, "instr_per_s": instrs / wall,
                     "lower_ms": st["lower_ms"], "launches": st["lower_launches"],
                     "p50_task_ms": _pct(lat, 0.5), "p99_task_ms": _pct(lat, 0.99)}
    out["speedup"] = out["batched"]["instr_per_s"] / out["plain"]["instr_per_s"]
    return out


def measure_nbody(igs, torch, stream, steps=200, exec_steps=2):
    """The all-pairs N-body configuration (2^20 float4 bodies, 8 nodes x 4
    devices, 128 chunks, lookahead 4, two tasks per step): all 400 tasks
    lowered in one launch (device time by CUDA events) and one per launch
    (per-task latency); then `exec_steps` steps (2 tasks each) lowered and
    executed at full size (2^20 bodies: 2^40 body pairs per step)."""
    n = 1 << 20
    p = W.nbody_program(n=n, steps=steps, nodes=8, devices=4, chunks=128, lookahead=4)
    out = lowering_modes(igs, torch, stream, p)
    # execution at full size
    q = W.nbody_program(n=n, steps=exec_steps, nodes=8, devices=4, chunks=128, lookahead=4)
    c = igs.Context(q.nodes, q.devices, q.horizon_step, q.lookahead, mode=igs.MODE_BATCHED, stream=stream)
    c.set_timing(True)
    for op in q.ops:
        if op[0] == "buffer":
            b = op[1]
            c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
        elif op[0] == "task":
            c.submit(op[1])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c.flush()
    c.execute()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    st = c.stats()
    pairs = float(n) * n * exec_steps
    out["execute"] = {"steps": exec_steps, "tasks": len(q.tasks), "instructions": int(c.counters()["instructions"]),
                      "seconds": dt, "workload_ms": st["workload_ms"], "copy_ms": st["copy_ms"],
                      "copy_gbs": st["copy_bytes"] / (st["copy_ms"] * 1e-3) / 1e9 if st["copy_ms"] else None,
                      "body_pairs_per_s": pairs / (st["workload_ms"] * 1e-3) if st["workload_ms"] else None}
    c.close()
    out["workload"] = (f"nbody: 2 x {n} float4 bodies, 8 nodes x 4 devices, 128 chunks, lookahead 4, "
                       f"{2 * steps} tasks lowered; {exec_steps} steps executed at full size")
    return out


def measure_jacobi(igs, torch, stream, reps=5):
    """The Jacobi reference program (256 x 256 fp32, 2 nodes x 2 devices, 4
    chunks, 8 steps, lookahead 0): lowered and executed through igs_run
    (best of `reps`), and one task per launch (per-task latency)."""
    p = W.jacobi_program(n=256, steps=8, nodes=2, devices=2, chunks=4, lookahead=0)
    best = None
    for _ in range(reps):
        c = igs.Context(p.nodes, p.devices, p.horizon_step, p.lookahead, mode=igs.MODE_BATCHED, stream=stream)
        for op in p.ops:
            if op[0] == "buffer":
                b = op[1]
                c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
            elif op[0] == "task":
                c.submit(op[1])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.run(4)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        instrs = int(c.counters()["instructions"])
        c.close()
        best = dt if best is None or dt < best else best
    c = igs.Context(p.nodes, p.devices, p.horizon_step, p.lookahead, mode=igs.MODE_PLAIN, stream=stream)
    c.set_timing(True)
    for op in p.ops:
        if op[0] == "buffer":
            b = op[1]
            c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
    lat = []
    for t in p.tasks:
        c.submit(t)
        lat.append(c.stats()["last_lower_ms"])
    c.close()
    lat.sort()
    return {"workload": "jacobi 256x256 fp32, 2 nodes x 2 devices, 4 chunks, 8 steps, lookahead 0",
            "lower_and_execute_s": best, "instructions": instrs, "instr_per_s": instrs / best,
            "plain_p50_task_ms": lat[len(lat) // 2], "plain_p99_task_ms": lat[-1]}


def _cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_program_worker(prog):
    """Pool worker: lowers one batch program with the CPU oracle; returns its
    instruction count (test infrastructure, run for the CPU baseline only)."""
    import oracle
    o = oracle.Oracle(prog.nodes, prog.devices, prog.horizon_step, prog.lookahead)
    for op in prog.ops:
        if op[0] == "buffer":
            b = op[1]
            o.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init is not None)
        elif op[0] == "task":
            o.submit(op[1].flat())
        elif op[0] == "flush":
            o.flush()
    n = sum(len(o.graph(k)["instrs"]) for k in range(prog.nodes))
    o.close()
    return n


def cpu_baselines(sample_tasks=300, batch_scale=0.05, batch_programs=512):
    """The CPU oracle (plain, single-threaded C++; test infrastructure) on
    the host cores: the wave workload's first `sample_tasks` tasks on one core
    with per-task latency (the time of each submission), and the batch of
    uneven programs at `batch_scale` of their tasks, one program per host core
    (a spawned process pool of hardware_concurrency workers)."""
    import oracle
    shape = _program_shape()
    bufs = [op for op in shape.ops if op[0] == "buffer"]
    tasks = [op[1] for op in shape.ops if op[0] == "task"][:sample_tasks]
    o = oracle.Oracle(shape.nodes, shape.devices, shape.horizon_step, shape.lookahead)
    for op in bufs:
        b = op[1]
        o.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init is not None)
    lat = []
    t0 = time.perf_counter()
    for t in tasks:
        t1 = time.perf_counter()
        o.submit(t.flat())
        lat.append(time.perf_counter() - t1)
    o.flush()
    cdt = time.perf_counter() - t0
    n_or = sum(len(o.graph(k)["instrs"]) for k in range(shape.nodes))
    o.close()
    lat.sort()
    cores = os.cpu_count() or 1
    wave = {"value": n_or / cdt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {sample_tasks} of {STEPS} tasks lowered on all {NODES} nodes ({n_or} instructions)",
            "p50_task_ms": lat[len(lat) // 2] * 1e3, "p99_task_ms": lat[min(len(lat) - 1, int(len(lat) * 0.99))] * 1e3,
            "cpu_model": _cpu_model(), "hardware_concurrency": cores}
    import multiprocessing as mp
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        counts = pool.map(_oracle_program_worker,
                          W.batch_programs(count=batch_programs, scale=batch_scale, seed=0x5EED + 3), chunksize=1)
    bdt = time.perf_counter() - t0
    batch = {"value": sum(counts) / bdt, "unit": UNIT, "cores": cores, "kind": "oracle",
             "sample": f"{batch_programs} uneven programs at {batch_scale:g} of their tasks, one program per core "
                       f"({sum(counts)} instructions, {bdt:.1f} s)"}
    return wave, batch


def measure_lookahead(igs):
    """Scheduler lookahead policies (Sec. 4.3) on a growing-row stream (the
    RSim pattern, 2048 x 1024 fp32, rows appended 1-64 at a time, 2 devices)
    and on the steady wave pattern (64 tasks of the benchmark program's
    shape): allocations, resize copies, and how many tasks were submitted
    before the first instruction existed (one task per launch, counted after
    every submission)."""
    progs = {"growing_rows": W.growing_program(rows_max=2048, cols=1024, grow=(1, 64), devices=2, chunks=2,
                                               seed=500),
             "wave_steady": W.wave_program(n=8, steps=64, nodes=NODES, devices=DEVICES, chunks=CHUNKS)}
    for op in progs["wave_steady"].ops:
        if op[0] == "buffer":
            op[1].extent = (N, N, 1)
            if op[1].init is not None:
                op[1].init = np.zeros((N, N), np.float32)
        elif op[0] == "task":
            op[1].range = (N, N, 1)
    out = {}
    for name, p in progs.items():
        res = {}
        for label, L, fl in (("L0", 0, 0), ("L8", 8, 0), ("horizons", W.LOOKAHEAD_HORIZONS, 0),
                             ("horizons_critical_path", W.LOOKAHEAD_HORIZONS, igs.FLAG_HORIZON_CP),
                             ("infinite", W.LOOKAHEAD_INFINITE, 0)):
            c = igs.Context(p.nodes, p.devices, p.horizon_step, L, mode=igs.MODE_PLAIN, flags=fl)
            c.set_timing(True)
            first = None
            k = 0
            for op in p.ops:
                if op[0] == "buffer":
                    b = op[1]
                    c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
                elif op[0] == "task":
                    c.submit(op[1])
                    k += 1
                    if first is None and int(c.counters()["instructions"]) > p.nodes:
                        first = k
                elif op[0] == "flush":
                    c.submit_epoch()
            c.sync()
            g = c.graph(0)
            t = g["instrs"][:, 1]
            res[label] = {"allocs_node0": int((t == 2).sum()),
                          "resize_copies_node0": int(((t == 4) & (g["instrs"][:, 6] == 1)).sum()),
                          "instructions": int(c.counters()["instructions"]),
                          "tasks_before_first_instruction": first if first is not None else k,
                          "lower_ms": c.stats()["lower_ms"]}
            c.close()
        res["tasks"] = len(p.tasks)
        out[name] = res
    return out


def _max_over_ranks(torch, dist, x, device):
    """The largest value of x over all ranks (x itself on one rank): a job's
    time is its slowest rank's."""
    if dist is None:
        return x
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: the units every rank processed over the job's time
    (replicas: each rank runs the same workload)."""
    return units_per_rank * world / seconds


def _nvtx(torch, name, push):
    """Marks the timed region for profilers (a no-op where NVTX is absent)."""
    try:
        if push:
            torch.cuda.nvtx.range_push(name)
        else:
            torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def run_gpu(args):
    import torch
    from paper_2503_10516_gb300 import igs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    sh = stream.cuda_stream
    prog = _program()
    bufs = prog.buffers
    tasks = prog.tasks

    def make_ctx(pinned=None, timing=True):
        c = igs.Context(NODES, DEVICES, HSTEP, LOOKAHEAD, mode=igs.MODE_BATCHED, device=local, stream=sh)
        c.set_timing(timing)
        for i, b in enumerate(bufs):
            init = None
            if b.init is not None:
                init = pinned[i] if pinned is not None else b.init
            c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, init)
        return c

    def submit_all(c):
        for t in tasks:
            c.submit(t)

    def step(c):
        c.run(WINDOW)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident throughput: inputs uploaded and tasks staged before timing
    ctxs = []
    for _ in range(args.warmup + args.steps):
        c = make_ctx()
        submit_all(c)
        ctxs.append(c)
    for i in range(args.warmup):
        step(ctxs[i])
        ctxs[i].close()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    barrier()
    with clocks:
        _nvtx(torch, "timed_steps", True)
        t0 = time.perf_counter()
        for i in range(args.steps):
            step(ctxs[args.warmup + i])
        barrier()
        t1 = time.perf_counter()
        _nvtx(torch, "timed_steps", False)
    dt = t1 - t0
    instrs = int(ctxs[-1].counters()["instructions"])
    stats = [ctxs[args.warmup + i].stats() for i in range(args.steps)]
    counters = ctxs[-1].counters()
    dt = _max_over_ranks(torch, dist, dt, "cuda")
    value = _job_rate(instrs * args.steps, world, dt)
    lower_ms = statistics.mean(s["lower_ms"] for s in stats)
    copy_ms = statistics.mean(s["copy_ms"] for s in stats)
    work_ms = statistics.mean(s["workload_ms"] for s in stats)
    copy_bytes = statistics.mean(s["copy_bytes"] for s in stats)
    launches = stats[0]["lower_launches"] + stats[0]["copy_launches"] + stats[0]["workload_launches"]
    for c in ctxs[args.warmup:]:
        c.close()
    ctxs = []

    # ---- per-task lowering latency, one task per launch (plain mode)
    plain = igs.Context(NODES, DEVICES, HSTEP, LOOKAHEAD, mode=igs.MODE_PLAIN, device=local, stream=sh)
    plain.set_timing(True)
    for b in bufs:
        plain.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
    lat = []
    for t in tasks:
        plain.submit(t)
        lat.append(plain.stats()["last_lower_ms"])
    plain.flush()
    plain_stats = plain.stats()
    plain_instrs = int(plain.counters()["instructions"])
    plain.close()
    lat_sorted = sorted(lat)
    p50 = lat_sorted[len(lat) // 2]
    p99 = lat_sorted[min(len(lat) - 1, int(len(lat) * 0.99))]

    # ---- end to end through the public API: pinned host inputs, graph read back
    pinned, keep = [], []
    for b in bufs:
        if b.init is not None:
            t = torch.from_numpy(np.ascontiguousarray(b.init)).pin_memory()
            keep.append(t)
            pinned.append(t.numpy())
        else:
            pinned.append(None)
    h2d = sum(int(b.init.nbytes) for b in bufs if b.init is not None) + len(tasks) * 492
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(e2e_steps):
        c = make_ctx(pinned=pinned, timing=False)
        submit_all(c)
        step(c)
        d2h = 0
        for n in range(NODES):
            g = c.graph(n)
            d2h += sum(int(v.nbytes) for v in g.values())
        c.close()
    barrier()
    e2e_dt = _max_over_ranks(torch, dist, time.perf_counter() - t0, "cuda")
    e2e_value = _job_rate(instrs * e2e_steps, world, e2e_dt)

    # ---- roofline of the dominant kernel (algorithmic bytes / event-timed duration)
    peaks, src = _peaks()
    hbm = float(peaks["hbm_gbs"])
    elems = N * N * STEPS
    parts = {
        "workload": (work_ms, elems * 12.0, "wave stencil workload kernel: 12 B/element (u_prev, u, u_next)"),
        "box_copy": (copy_ms, copy_bytes, "box-copy kernel: bytes read + written"),
        "lowering": (lower_ms, float(counters["map_reads"] + counters["map_writes"]) * MAP_ENTRY_BYTES
                     + instrs * 44.0 + counters["edges"] * 12.0 + counters["boxes"] * 24.0,
                     "lowering kernel: region-map entries read + written x 28 B (six box coordinates + one value) "
                     "+ output records (44 B per instruction, 12 B per edge, 24 B per box)"),
    }
    dom = max(parts, key=lambda k: parts[k][0])
    ms, byts, what = parts[dom]
    achieved = byts / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    prof = _lowering_profile()
    traffic, issue = None, None
    if prof and dom == "lowering":
        # DRAM bytes of the captured launch per task, times the tasks of this launch
        traffic = float(prof["dram_bytes_per_task"]) * STEPS
        ipc = float(prof["inst_per_active_sm_cycle"])
        issue = {"inst_per_active_sm_cycle": ipc, "peak": 4.0, "frac": ipc / 4.0,
                 "warp_inst_per_emitted_instruction": float(prof["warp_inst_per_emitted_instruction"]),
                 "source": os.path.relpath(LOWER_PROFILE, ROOT)}
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "kernel": dom, "what": what, "peak_source": src,
            "issue_efficiency": issue}
    hot = {}
    for k, (ms_k, b_k, w_k) in parts.items():
        a = b_k / (ms_k * 1e-3) / 1e9 if ms_k > 0 else 0.0
        hot[k] = {"ms_per_step": ms_k, "bytes_per_step": b_k, "achieved_gbs": a, "frac": a / hbm}

    # ---- batched lowering of many programs, served lowering of many streams
    def section(fn, *a):
        """An auxiliary measurement; a failure is recorded in the line instead
        of ending the run."""
        if world != 1 or args.headline_only:
            return None
        try:
            return fn(*a)
        except Exception as e:  # noqa: BLE001
            return {"error": f"{type(e).__name__}: {e}"}

    big_copy = section(measure_box_copy, igs, torch, stream)
    executors = section(measure_executors, igs, torch, sh, prog, make_ctx)
    wave_modes = section(lowering_modes, igs, torch, sh, _program_shape(), True)
    nbody = section(measure_nbody, igs, torch, sh)
    jacobi = section(measure_jacobi, igs, torch, sh)
    lookahead = section(measure_lookahead, igs)
    batched = section(measure_batched, igs, torch, sh)
    served = section(measure_served, igs, torch, sh)
    resize_exec = section(measure_resize_execution, igs, torch, sh)

    # ---- CPU baseline: the oracle on bounded samples of the same workloads
    cpu, cpu_batch = None, None
    if rank == 0 and world == 1 and not args.headline_only:
        try:
            cpu, cpu_batch = cpu_baselines()
        except Exception as e:  # noqa: BLE001
            cpu = {"error": f"{type(e).__name__}: {e}"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lowering": f"batched, one launch; execution follows the lowering in steps of {WINDOW} submissions (igs_run)",
                       "step": "lower all tasks + execute all instructions (allocs, box copies, stencil kernels)",
                       "l2": "inputs larger than L2 (3 x 256 MiB buffers)",
                       "instructions_per_step": instrs, "parallelism": f"replicas x{world}"},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "steps": e2e_steps},
            "gpu_launches": launches * args.steps,
            "roofline": roof,
            "hot_path": hot,
            "lowering_modes": wave_modes,
            "lowering": {"batched_instr_per_s": instrs / (lower_ms * 1e-3) if lower_ms else None,
                         "plain_instr_per_s": plain_instrs / (plain_stats["lower_ms"] * 1e-3),
                         "plain_launches": plain_stats["lower_launches"],
                         "p50_task_ms": p50, "p99_task_ms": p99,
                         "batched_ms_per_task": lower_ms / STEPS},
            "box_copy_gbs": (copy_bytes / (copy_ms * 1e-3) / 1e9) if copy_ms else None,
            "in_step_launches": {"lowering": stats[0]["lower_launches"], "box_copy": stats[0]["copy_launches"],
                                 "stencil_or_level": stats[0]["workload_launches"],
                                 "note": "a level with copies and stencils runs as one level launch"},
            "box_copy_resize_512MiB": ({k: (dict(v, frac=v["gbs"] / hbm) if "gbs" in v else v)
                                        for k, v in big_copy.items()} if isinstance(big_copy, dict) else None),
            "executors": executors,
            "nbody": nbody,
            "jacobi": jacobi,
            "batched_programs": batched,
            "lookahead": lookahead,
            "served": served,
            "resize_copies_executed": resize_exec,
            "clocks": clocks.summary(),
            "cpu_baseline": cpu,
            "cpu_baseline_batch": cpu_batch,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """Small fixed cases for profiler captures (no timing, no JSON metric):
    flow_wave16 = the first 16 wave tasks on 8192^2 buffers, lowered, then
    executed by the dataflow executor; done twice (capture the second).
    lower_wave64 = the first 64 tasks of the benchmark's wave program lowered
    in one launch (the lowering kernel's configuration inside the timed step,
    without the concurrent execution); done twice (capture the second)."""
    from paper_2503_10516_gb300 import igs
    if args.profile_case == "lower_wave64":
        p = _program_shape()
        p.ops = [op for op in p.ops if op[0] == "buffer"] + [op for op in p.ops if op[0] == "task"][:64]
        for _ in range(2):
            c = igs.Context(p.nodes, p.devices, p.horizon_step, p.lookahead, mode=igs.MODE_BATCHED)
            for op in p.ops:
                if op[0] == "buffer":
                    b = op[1]
                    c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, None if b.init is None else
                                    np.zeros((N, N), np.float32))
                elif op[0] == "task":
                    c.submit(op[1])
            c.sync()
            n = int(c.counters()["instructions"])
            cnt = c.counters()
            c.close()
        print(json.dumps({"case": args.profile_case, "tasks": 64, "instructions": n, "edges": int(cnt["edges"]),
                          "boxes": int(cnt["boxes"]), "map_reads": int(cnt["map_reads"]),
                          "map_writes": int(cnt["map_writes"])}), flush=True)
        return 0
    p = W.wave_program(n=N, steps=16, nodes=NODES, devices=DEVICES, chunks=CHUNKS, lookahead=LOOKAHEAD,
                       horizon_step=HSTEP)
    for _ in range(2):
        c = igs.Context(p.nodes, p.devices, p.horizon_step, p.lookahead, mode=igs.MODE_BATCHED)
        c.set_executor(igs.EXEC_DATAFLOW)
        for op in p.ops:
            if op[0] == "buffer":
                b = op[1]
                c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
            elif op[0] == "task":
                c.submit(op[1])
        c.flush()
        c.execute()
        n = int(c.counters()["instructions"])
        c.close()
    print(json.dumps({"case": args.profile_case, "instructions": n}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="igs", choices=["igs", "reference"])
    ap.add_argument("--headline-only", action="store_true",
                    help="print the line without the auxiliary sections (for a launch-list capture of the step)")
    ap.add_argument("--profile-case", default=None, choices=["flow_wave16", "lower_wave64"],
                    help="run one small fixed case for a profiler capture instead of the benchmark")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
