"""The benchmark's own workload at full size, in the launch configuration the
benchmark times (one lowering launch for all 1000 tasks through igs_run,
execution following in windows of 16 submissions): sampled 4 x 4 patches of
the final wave field equal an exact float32 recomputation of each patch's
light cone on the CPU (the wave update in the same operation order, over the
(2*1000 + 4)^2 initial values the patch depends on), on both executors."""
import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N, STEPS, NODES, DEVICES, CHUNKS, LOOKAHEAD, HSTEP, WINDOW = 8192, 1000, 4, 4, 64, 8, 4, 16
PATCH = 4
# patch corners: the middle of the field, and rows straddling the boundary
# between nodes 0 and 1 (row 2048) and a device boundary (row 2048 + 128)
SAMPLES = [(4094, 4094), (2046, 3000), (2174, 6000)]


def _cone(u_prev, u, y0, x0, steps):
    """Final values of the PATCH x PATCH patch at (y0, x0) after `steps` wave
    updates from the initial fields, computed on the shrinking light cone
    (every point stays in the interior: no border rule)."""
    r = steps
    p = u_prev[y0 - r:y0 + PATCH + r, x0 - r:x0 + PATCH + r].astype(np.float32)
    c = u[y0 - r:y0 + PATCH + r, x0 - r:x0 + PATCH + r].astype(np.float32)
    for _ in range(steps):
        cc = c[1:-1, 1:-1]
        t2 = (np.float32(2.0) * cc) - p[1:-1, 1:-1]
        t5 = (c[:-2, 1:-1] + c[2:, 1:-1]) + (c[1:-1, :-2] + c[1:-1, 2:])
        t8 = np.float32(0.25) * (t5 - np.float32(4.0) * cc)
        p, c = cc, (t2 + t8).astype(np.float32)
    return c


@pytest.fixture(scope="module")
def program_and_expected():
    p = W.wave_program(n=N, steps=STEPS, nodes=NODES, devices=DEVICES, chunks=CHUNKS, lookahead=LOOKAHEAD,
                       horizon_step=HSTEP)
    u_prev, u = p.buffers[0].init.reshape(N, N), p.buffers[1].init.reshape(N, N)
    want = {s: _cone(u_prev, u, s[0], s[1], STEPS) for s in SAMPLES}
    last = [op[1] for op in p.ops if op[0] == "task"][-1]
    out_buffer = last.accessors[2].buffer
    return p, want, out_buffer


@pytest.mark.parametrize("executor", [0, 1])
def test_wave_8192_bench_configuration_sampled(program_and_expected, executor):
    from paper_2503_10516_gb300 import igs
    p, want, ob = program_and_expected
    c = igs.Context(NODES, DEVICES, HSTEP, LOOKAHEAD, mode=igs.MODE_BATCHED)
    c.set_executor(executor)
    for b in p.buffers:
        c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
    for t in p.tasks:
        c.submit(t)
    c.submit_epoch()
    c.run(WINDOW)
    for (y0, x0), w in want.items():
        got = c.read_buffer(ob, (y0, x0, 0), (y0 + PATCH, x0 + PATCH, 1), 4).view(np.float32).reshape(PATCH, PATCH)
        assert np.array_equal(got, w), f"patch at ({y0}, {x0}) differs (executor {executor})"
    c.close()


NB = 1 << 20
BODIES = [0, 1, 4095, 8192, 123457, NB // 2, NB - 2, NB - 1]


def _nbody_bodies(P, V, idx):
    """Velocity and position of bodies idx after one step: the sum over all
    bodies in index order, in float32, each term as the kernel forms it."""
    eps, dt = np.float32(1e-6), np.float32(0.01)
    out_v, out_p = [], []
    for i in idx:
        pi = P[i]
        dx = P[:, 0] - pi[0]
        dy = P[:, 1] - pi[1]
        dz = P[:, 2] - pi[2]
        r2 = ((dx * dx + dy * dy) + dz * dz) + eps
        inv = np.float32(1.0) / (r2 * np.sqrt(r2))
        wgt = P[:, 3] * inv
        acc = [np.add.accumulate((d * wgt).astype(np.float32), dtype=np.float32)[-1] for d in (dx, dy, dz)]
        v = V[i].copy()
        for c in range(3):
            v[c] = v[c] + acc[c] * dt
        p = P[i].copy()
        for c in range(3):
            p[c] = p[c] + v[c] * dt
        out_v.append(v)
        out_p.append(p)
    return np.array(out_v, np.float32), np.array(out_p, np.float32)


@pytest.mark.parametrize("executor", [0, 1])
def test_nbody_1m_configuration_one_step_sampled(executor):
    """The all-pairs N-body configuration at full size (2^20 float4 bodies,
    8 nodes x 4 devices, 128 chunks, lookahead 4), one step (both tasks):
    sampled bodies' velocity and position equal a float32 sequential j-sum."""
    from paper_2503_10516_gb300 import igs
    p = W.nbody_program(n=NB, steps=1, nodes=8, devices=4, chunks=128, lookahead=4)
    P0 = p.buffers[0].init.reshape(NB, 4).astype(np.float32)
    V0 = p.buffers[1].init.reshape(NB, 4).astype(np.float32)
    want_v, want_p = _nbody_bodies(P0, V0, BODIES)
    c = igs.Context(p.nodes, p.devices, p.horizon_step, p.lookahead, mode=igs.MODE_BATCHED)
    c.set_executor(executor)
    for b in p.buffers:
        c.create_buffer(b.dims, b.extent[:b.dims], b.elem_size, b.init)
    for t in p.tasks:
        c.submit(t)
    c.flush()
    c.execute()
    for k, i in enumerate(BODIES):
        v = c.read_buffer(1, (i, 0, 0), (i + 1, 1, 1), 16).view(np.float32).reshape(4)
        q = c.read_buffer(0, (i, 0, 0), (i + 1, 1, 1), 16).view(np.float32).reshape(4)
        assert np.array_equal(v, want_v[k]), f"velocity of body {i} (executor {executor})"
        assert np.array_equal(q, want_p[k]), f"position of body {i} (executor {executor})"
    c.close()
