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
WORKLOAD = (f"wave2d: 3 x {N}x{N} fp32 buffers rotating, {NODES} nodes x {DEVICES} devices, {CHUNKS} row chunks, "
            f"{STEPS} time steps, lookahead {LOOKAHEAD}, horizon every {HSTEP} tasks")


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
    c = igs.Context(prog.nodes, prog.devices, prog.horizon_step, prog.lookahead, mode=mode, stream=stream,
                    **igs.small_caps(prog))
    for op in prog.ops:
        if op[0] == "buffer":
            b = op[1]
            c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
    return c


def measure_batched(igs, torch, stream, count=512, scale=0.01):
    """Uneven programs (1-8 buffers of 2^10-2^24 elements, 1-128 chunks, 2-32
    memories, lookahead 0-16; task counts scaled down): one launch over all
    of them vs one task per launch. The batch shape is picked first by
    timing every candidate on a fresh copy of the batch."""
    progs = W.batch_programs(count=count, scale=scale, seed=0x5EED + 3)
    res = {}

    def staged():
        ctxs = [_stage_ctx(igs, p, igs.MODE_BATCHED, stream) for p in progs]
        for p, c in zip(progs, ctxs):
            for op in p.ops:
                if op[0] == "task":
                    c.submit(op[1])
                elif op[0] == "flush":
                    c.submit_epoch()
        return ctxs

    def timer():
        torch.cuda.synchronize()
        return time.perf_counter()

    # the batch shape (one block per unit, or a work queue of persistent
    # blocks in submission / longest-first order) is picked by timing
    units = sum(p.nodes for p in progs)
    t_tune = time.perf_counter()
    cands = igs.batch_shape_candidates(units, torch.cuda.get_device_properties(0).multi_processor_count)
    shape, times = igs.tune_lower_batch(staged, cands, timer)
    res["tuning"] = {"units": units, "seconds": time.perf_counter() - t_tune, "chosen": shape,
                     "launch_seconds": [{"shape": s, "seconds": t} for s, t in times]}
    for mode_name, mode in (("plain", igs.MODE_PLAIN), ("batched", igs.MODE_BATCHED)):
        ctxs = [_stage_ctx(igs, p, mode, stream) for p in progs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for p, c in zip(progs, ctxs):
            for op in p.ops:
                if op[0] == "task":
                    c.submit(op[1])
                elif op[0] == "flush":
                    c.submit_epoch()
        if mode == igs.MODE_BATCHED:
            igs.lower_batch(ctxs, shape)
        else:
            for c in ctxs:
                c.sync()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        instrs = sum(int(c.counters()["instructions"]) for c in ctxs)
        launches = sum(int(c.counters()["launches"]) for c in ctxs)
        res[mode_name] = {"instr_per_s": instrs / dt, "seconds": dt, "instructions": instrs, "launches": launches}
        if mode == igs.MODE_BATCHED:
            # the longest unit bounds the launch: the slowest program's mean
            # per-node lowering time (SM cycles at the sampled clock)
            cyc = max(c.profile()["total"] / p.nodes for p, c in zip(progs, ctxs))
            res[mode_name]["slowest_program_node_cycles"] = cyc
        for c in ctxs:
            c.close()
    res["programs"] = count
    res["task_scale"] = scale
    res["speedup"] = res["batched"]["instr_per_s"] / res["plain"]["instr_per_s"]
    return res


def measure_served(igs, torch, stream, streams=64, rate=1e4, rows_max=2048, cols=1024, lookahead=0):
    """Growing-row program streams (rows appended 1-64 at a time, each task
    reading every earlier row) submitting with Poisson arrivals; per-task
    latency = arrival -> every node of its program has lowered it; the
    arrivals are replayed by the library's own host loop (igs_serve_replay),
    so the rate is not limited by Python. Compared
    with one task per launch under the same arrivals (the host submits a task
    when it arrives or when the previous launch has returned, then waits for
    its launch); the plain path's unloaded per-launch time is reported too."""
    rng = np.random.default_rng(0x5EED + 5)
    progs = [W.growing_program(rows_max=rows_max, cols=cols, grow=(1, 64), devices=2, chunks=2,
                               lookahead=lookahead, seed=500 + i) for i in range(streams)]
    order = []
    for i, p in enumerate(progs):
        for op in p.ops:
            if op[0] in ("task", "flush"):
                order.append(i)
    rng.shuffle(order)
    gaps = rng.exponential(1.0 / rate, size=len(order))
    bodies = [[op for op in p.ops if op[0] in ("task", "flush")] for p in progs]
    out = {}
    # served
    srv = igs.Server(max_slots=max(32, 2 * streams))
    ctxs = [_stage_ctx(igs, p, igs.MODE_PLAIN, None) for p in progs]
    for c, p in zip(ctxs, progs):
        assert srv.attach(c, 4 * len(p.ops) + 16) == 0
    srv.start()
    # the library's own submission loop replays the arrivals (igs_serve_replay)
    pos = [0] * streams
    trace, t_ns = [], 0.0
    for k, i in enumerate(order):
        t_ns += gaps[k] * 1e9
        op = bodies[i][pos[i]]
        pos[i] += 1
        trace.append((i, op[1] if op[0] == "task" else None, int(t_ns)))
    lat_ns, wall_ns = srv.replay(ctxs, trace, timeout_ms=120000)
    lat = list(np.asarray(lat_ns, dtype=np.float64) * 1e-9)
    for c in ctxs:
        srv.detach(c)
    srv.stop()
    instrs = sum(int(c.counters()["instructions"]) for c in ctxs)
    for c in ctxs:
        c.close()
    srv.close()
    lat.sort()
    out["served"] = {"p50_ms": lat[len(lat) // 2] * 1e3, "p99_ms": lat[int(len(lat) * 0.99)] * 1e3,
                     "tasks": len(lat), "instructions": instrs, "wall_s": wall_ns * 1e-9,
                     "tasks_per_s": len(lat) / (wall_ns * 1e-9), "instr_per_s": instrs / (wall_ns * 1e-9)}
    # one task per launch under the same arrivals: the host submits each task
    # when it arrives (or when the previous launch has returned, if later) and
    # waits for its launch; latency from arrival to completion
    ctxs = [_stage_ctx(igs, p, igs.MODE_PLAIN, None) for p in progs]
    pos = [0] * streams
    lat, service = [], []
    t_next = time.perf_counter()
    for k, i in enumerate(order):
        t_next += gaps[k]
        while time.perf_counter() < t_next:
            pass
        op = bodies[i][pos[i]]
        pos[i] += 1
        t0 = time.perf_counter()
        if op[0] == "task":
            ctxs[i].submit(op[1])
        else:
            ctxs[i].submit_epoch()
        ctxs[i].sync()
        t1 = time.perf_counter()
        lat.append(t1 - t_next)
        service.append(t1 - t0)
    for c in ctxs:
        c.close()
    lat.sort()
    service.sort()
    out["plain"] = {"p50_ms": lat[len(lat) // 2] * 1e3, "p99_ms": lat[int(len(lat) * 0.99)] * 1e3,
                    "unloaded_p50_ms": service[len(service) // 2] * 1e3,
                    "unloaded_p99_ms": service[int(len(service) * 0.99)] * 1e3}
    out["streams"] = streams
    out["rate_tasks_per_s"] = rate
    out["workload"] = f"{streams} streams, growing {rows_max}x{cols} fp32 rows, 2 devices, lookahead {lookahead}"
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


def measure_nbody_lowering(igs, torch, stream, tasks=100):
    """The all-pairs N-body configuration (2^20 float4 bodies, 8 nodes x 4
    devices, 128 chunks, lookahead 4, two tasks per step): the first `tasks`
    tasks lowered in one launch (device time by CUDA events), and the same
    tasks one per launch (per-task latency)."""
    n = 1 << 20
    p = W.nbody_program(n=n, steps=tasks // 2, nodes=8, devices=4, chunks=128, lookahead=4)
    out = {}
    for name, mode in (("batched", igs.MODE_BATCHED), ("plain", igs.MODE_PLAIN)):
        c = igs.Context(p.nodes, p.devices, p.horizon_step, p.lookahead, mode=mode, stream=stream)
        c.set_timing(True)
        for op in p.ops:
            if op[0] == "buffer":
                b = op[1]
                c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
        lat = []
        for op in p.ops:
            if op[0] == "task":
                c.submit(op[1])
                if mode == igs.MODE_PLAIN:
                    lat.append(c.stats()["last_lower_ms"])
        c.flush()
        st = c.stats()
        instrs = int(c.counters()["instructions"])
        out[name] = {"instructions": instrs, "lower_ms": st["lower_ms"], "launches": st["lower_launches"],
                     "instr_per_s": instrs / (st["lower_ms"] * 1e-3)}
        if lat:
            lat.sort()
            out[name]["p50_task_ms"] = lat[len(lat) // 2]
            out[name]["p99_task_ms"] = lat[min(len(lat) - 1, int(len(lat) * 0.99))]
        c.close()
    out["workload"] = f"nbody: 2 x {n} float4 bodies, 8 nodes x 4 devices, 128 chunks, lookahead 4, first {tasks} tasks"
    return out


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
        for label, L in (("L0", 0), ("L8", 8), ("horizons", W.LOOKAHEAD_HORIZONS), ("infinite", W.LOOKAHEAD_INFINITE)):
            c = igs.Context(p.nodes, p.devices, p.horizon_step, L, mode=igs.MODE_PLAIN)
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
        "lowering": (lower_ms, float(counters["map_reads"] + counters["map_writes"]) * 40.0
                     + instrs * 44.0 + counters["edges"] * 12.0 + counters["boxes"] * 24.0,
                     "lowering kernel: region-map entries read + written x 40 B + output records"),
    }
    dom = max(parts, key=lambda k: parts[k][0])
    ms, byts, what = parts[dom]
    achieved = byts / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": None, "kernel": dom, "what": what, "peak_source": src}
    hot = {}
    for k, (ms_k, b_k, w_k) in parts.items():
        a = b_k / (ms_k * 1e-3) / 1e9 if ms_k > 0 else 0.0
        hot[k] = {"ms_per_step": ms_k, "bytes_per_step": b_k, "achieved_gbs": a, "frac": a / hbm}

    # ---- batched lowering of many programs, served lowering of many streams
    big_copy = measure_box_copy(igs, torch, stream)
    executors = measure_executors(igs, torch, sh, prog, make_ctx) if world == 1 else None
    nbody = measure_nbody_lowering(igs, torch, sh) if world == 1 else None
    lookahead = measure_lookahead(igs) if world == 1 else None
    batched = measure_batched(igs, torch, sh) if world == 1 else None
    served = {f"{int(r)}_per_s": measure_served(igs, torch, sh, rate=r) for r in (1e4, 1e5, 1e6)} \
        if world == 1 else None

    # ---- CPU baseline: the oracle on a bounded sample of the same workload
    cpu = None
    if rank == 0 and world == 1:
        shape = _program_shape()
        sample_tasks = 300
        shape.ops = [op for op in shape.ops if op[0] == "buffer"] + \
            [op for op in shape.ops if op[0] == "task"][:sample_tasks] + [("flush",)]
        t0 = time.perf_counter()
        n_or = _oracle_lower(shape)
        cdt = time.perf_counter() - t0
        cpu = {"value": n_or / cdt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"first {sample_tasks} of {STEPS} tasks lowered on all {NODES} nodes ({n_or} instructions)"}

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
            "lowering": {"batched_instr_per_s": instrs / (lower_ms * 1e-3) if lower_ms else None,
                         "plain_instr_per_s": plain_instrs / (plain_stats["lower_ms"] * 1e-3),
                         "plain_launches": plain_stats["lower_launches"],
                         "p50_task_ms": p50, "p99_task_ms": p99,
                         "batched_ms_per_task": lower_ms / STEPS},
            "box_copy_gbs": (copy_bytes / (copy_ms * 1e-3) / 1e9) if copy_ms else None,
            "box_copy_resize_512MiB": {k: dict(v, frac=v["gbs"] / hbm) for k, v in big_copy.items()},
            "executors": executors,
            "nbody_lowering": nbody,
            "batched_programs": batched,
            "lookahead": lookahead,
            "served": served,
            "clocks": clocks.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """Small fixed cases for profiler captures (no timing, no JSON metric):
    flow_wave16 = the first 16 wave tasks on 8192^2 buffers, lowered, then
    executed by the dataflow executor; done twice (capture the second)."""
    from paper_2503_10516_gb300 import igs
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
    ap.add_argument("--profile-case", default=None, choices=["flow_wave16"],
                    help="run one small fixed case for a profiler capture instead of the benchmark")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
