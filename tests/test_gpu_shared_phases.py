"""Phases shared by helper warps (push / await per buffer; coherence planned
per (buffer, memory) and applied per table; the kernel phase planned per
chunk, or split per device when a written buffer is also read through another
accessor) give the oracle's graphs and the sequential contents, and are
really taken (the profile counts the shared phases)."""
import numpy as np
import pytest

from paper_2503_10516_gb300 import workloads as W
from tests.harness import assert_same_graph, feed, oracle_graphs
from tests.replay import sequential_run

pytestmark = pytest.mark.gpu


def _two_stale_buffers(nodes=2, devices=4, steps=4, lookahead=0):
    """Tasks that read two buffers with a halo, both last written with a
    different chunking: every device has stale halo rows in both."""
    rng = np.random.default_rng(11)
    n = 24
    a = W.Buffer(2, (n, 16, 1), 4, rng.integers(0, 2**32, n * 16, dtype=np.uint64).astype(np.uint32), "u32")
    b = W.Buffer(2, (n, 16, 1), 4, rng.integers(0, 2**32, n * 16, dtype=np.uint64).astype(np.uint32), "u32")
    o = W.Buffer(2, (n, 16, 1), 4, None, "u32")
    ops = [("buffer", a), ("buffer", b), ("buffer", o)]
    for s in range(steps):
        ops.append(("task", W.Task(2, (n, 16, 1), 8, W.K_GENERIC,
                                   [W.Accessor(0, W.READ_WRITE, W.one_to_one())])))
        ops.append(("task", W.Task(2, (n, 16, 1), 6, W.K_GENERIC,
                                   [W.Accessor(1, W.READ_WRITE, W.one_to_one())])))
        ops.append(("task", W.Task(2, (n, 16, 1), 8, W.K_GENERIC,
                                   [W.Accessor(2, W.WRITE, W.one_to_one()),
                                    W.Accessor(0, W.READ, W.neighborhood(1, 1)),
                                    W.Accessor(1, W.READ, W.neighborhood(2, 1))])))
    ops.append(("flush",))
    return W.Program(f"two-stale-{nodes}x{devices}-L{lookahead}", nodes, devices, 3, lookahead, ops)


class _Staged:
    def __init__(self, prog):
        from paper_2503_10516_gb300 import igs
        self.g = igs.GpuImpl(prog, mode=igs.MODE_BATCHED)
        self.ctx = self.g.ctx

    def __getattr__(self, name):
        return getattr(self.g, name)

    def flush(self):
        self.ctx.submit_epoch()


def _read_own_writes(nodes=2, devices=3, steps=3, lookahead=0):
    """Each task writes a buffer one-to-one and reads it again with a halo
    through a second accessor: kernels of one device depend on one another,
    so the kernel phase keeps its per-device split."""
    rng = np.random.default_rng(12)
    n = 24
    a = W.Buffer(2, (n, 16, 1), 4, rng.integers(0, 2**32, n * 16, dtype=np.uint64).astype(np.uint32), "u32")
    ops = [("buffer", a)]
    for s in range(steps):
        ops.append(("task", W.Task(2, (n, 16, 1), 9 - s, W.K_GENERIC,
                                   [W.Accessor(0, W.READ_WRITE, W.one_to_one()),
                                    W.Accessor(0, W.READ, W.neighborhood(1, 1))])))
    ops.append(("flush",))
    return W.Program(f"read-own-writes-{nodes}x{devices}-L{lookahead}", nodes, devices, 3, lookahead, ops)


def _overlapping_consumers(nodes=2, devices=3, steps=3, lookahead=0):
    """Every chunk reads all of one buffer (its consumers on one memory
    overlap: planned in order by one worker) and a halo of another (its
    consumers overlap nothing on their memory: spread over the workers)."""
    rng = np.random.default_rng(13)
    n = 30
    a = W.Buffer(2, (n, 8, 1), 4, rng.integers(0, 2**32, n * 8, dtype=np.uint64).astype(np.uint32), "u32")
    b = W.Buffer(2, (n, 8, 1), 4, rng.integers(0, 2**32, n * 8, dtype=np.uint64).astype(np.uint32), "u32")
    o = W.Buffer(2, (n, 8, 1), 4, None, "u32")
    ops = [("buffer", a), ("buffer", b), ("buffer", o)]
    for s in range(steps):
        ops.append(("task", W.Task(2, (n, 8, 1), 5, W.K_GENERIC, [W.Accessor(0, W.READ_WRITE, W.one_to_one())])))
        ops.append(("task", W.Task(2, (n, 8, 1), 7, W.K_GENERIC, [W.Accessor(1, W.READ_WRITE, W.one_to_one())])))
        ops.append(("task", W.Task(2, (n, 8, 1), 12, W.K_GENERIC,
                                   [W.Accessor(2, W.WRITE, W.one_to_one()),
                                    W.Accessor(0, W.READ, W.all_mapper()),
                                    W.Accessor(1, W.READ, W.neighborhood(1, 0))])))
    ops.append(("flush",))
    return W.Program(f"overlapping-consumers-{nodes}x{devices}-L{lookahead}", nodes, devices, 3, lookahead, ops)


def _check(prog, pipelined, contents=True):
    from paper_2503_10516_gb300 import igs
    ref, rej = oracle_graphs(prog)
    if pipelined:
        g = _Staged(prog)
        feed(g, prog)
        g.ctx.run(2)
    else:
        g = igs.GpuImpl(prog, mode=igs.MODE_PLAIN)
        feed(g, prog)
        g.ctx.execute()
    assert g.rejected() == rej
    for n in range(prog.nodes):
        assert_same_graph(g.graph(n), ref[n], f"{prog.name} node {n}")
    want, known = sequential_run(prog, set(rej)) if contents else (None, None)
    gone = {op[1] for op in prog.ops if op[0] == "destroy"}
    for b, buf in enumerate(prog.buffers):
        if b in gone or not contents:
            continue
        got = g.ctx.read_buffer(b, (0, 0, 0), buf.extent, buf.elem_size)
        k = known[b]
        assert np.array_equal(got[k], want[b][k]), f"{prog.name}: buffer {b} differs"
    shared = g.ctx.profile()["n_shared_phases"]
    g.ctx.close()
    return shared


@pytest.mark.parametrize("pipelined", [False, True])
@pytest.mark.parametrize("shape", [(2, 4, 0), (1, 3, 2), (3, 2, 1)])
def test_two_stale_buffers(shape, pipelined):
    nodes, devices, look = shape
    assert _check(_two_stale_buffers(nodes, devices, lookahead=look), pipelined) > 0


@pytest.mark.parametrize("seed", range(24))
def test_random_programs_with_helpers(seed):
    """One task per launch on nodes with several devices runs the shared
    phases; random programs over all mappers."""
    p = W.random_program(90_000 + seed, max_extent=12, max_tasks=12, max_nodes=2, max_devices=4)
    if p.devices < 2:
        p.devices = 2
    _check(p, pipelined=bool(seed % 2))


@pytest.mark.parametrize("pipelined", [False, True])
@pytest.mark.parametrize("shape", [(2, 3, 0), (1, 4, 2)])
def test_written_buffer_read_again_keeps_device_split(shape, pipelined):
    """Graphs only: the chunks read what other chunks of the same task write,
    which the sequential replay does not order."""
    nodes, devices, look = shape
    assert _check(_read_own_writes(nodes, devices, lookahead=look), pipelined, contents=False) > 0


@pytest.mark.parametrize("pipelined", [False, True])
@pytest.mark.parametrize("shape", [(2, 3, 0), (1, 4, 1), (3, 2, 0)])
def test_overlapping_consumers_on_one_memory(shape, pipelined):
    nodes, devices, look = shape
    assert _check(_overlapping_consumers(nodes, devices, lookahead=look), pipelined) > 0
