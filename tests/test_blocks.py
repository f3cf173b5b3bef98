"""A grid decomposed into blocks (CPU): the host logic of the multi-rank path.

Every block is stepped by the oracle here (the CUDA kernels of the same
operations are checked on the GPU in test_gpu_blocks.py); the decomposition,
the two-phase halo exchange, the message matching and the global time step
are the package's.  A decomposed run must reproduce the single-grid oracle
run bit for bit: each cell's update reads the same values in the same order,
and the global smax is the maximum of the same edge speeds.

Pinned: in-process exchange over 1..3 x 1..3 blocks with every boundary kind
and periodic directions split over two blocks (both sides facing one peer),
and the same run as 2 and 4 gloo ranks exchanging through torch.distributed.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import paper_1308_1464_gb300 as mc
from paper_1308_1464_gb300.blocks import Block, Decomposition, DistTransport, Stepper, split

torch = pytest.importorskip("torch")

P, X, W, G = mc.BC_PERIODIC, mc.BC_EXTRAP, mc.BC_WALL, mc.BC_GIVEN
ORACLE_ID = {mc.ACOUSTICS: oracle.ACOUSTICS, mc.SWE_ROE: oracle.SWE, mc.EULER_ROE: oracle.EULER,
             mc.ADVECTION: oracle.ADVECTION}


def oracle_problem(p):
    return oracle.Problem(ORACLE_ID[p.solver], p.mx, p.my, p.dx, p.dy, limiter=p.limiter,
                          order=p.order, transverse=p.transverse, efix=p.efix,
                          bc=tuple(int(b) for b in p.bc), param=tuple(p.param))


class OracleOps:
    """A block's operations on the CPU: numpy slicing for the strips, the
    oracle for ghost fills and steps.  States are (meqn, my + 4, mx + 4)."""

    def __init__(self, p):
        self.p = p
        self.op = oracle_problem(p)
        bc = [int(b) for b in p.bc]
        self.fill_ops = [oracle_problem(p), oracle_problem(p)]
        self.fill_ops[0].bc = (bc[0], bc[1], G, G)     # x phase only
        self.fill_ops[1].bc = (G, G, bc[2], bc[3])     # y phase only

    def halo_elems(self, side):
        p = self.p
        return p.meqn * (p.my * 2 if side < 2 else 2 * (p.mx + 4))

    def alloc(self, n):
        return torch.zeros(int(n), dtype=torch.float64)

    def copy(self, src, dst):
        dst.copy_(src)

    def _region(self, side, ghost):
        mx, my = self.p.mx, self.p.my
        if side < 2:
            i = (0 if not ghost else -2) if side == 0 else (mx - 2 if not ghost else mx)
            return slice(2, 2 + my), slice(2 + i, 4 + i)
        j = (0 if not ghost else -2) if side == 2 else (my - 2 if not ghost else my)
        return slice(2 + j, 4 + j), slice(0, mx + 4)

    def pack(self, q, side, buf):
        rj, ri = self._region(side, False)
        buf.copy_(torch.from_numpy(np.ascontiguousarray(q[:, rj, ri]).reshape(-1)))

    def unpack(self, buf, side, q):
        rj, ri = self._region(side, True)
        q[:, rj, ri] = buf.numpy().reshape(q[:, rj, ri].shape)

    def fill_dir(self, q, direction):
        q[...] = oracle.bc_fill(self.fill_ops[direction], q)

    def step(self, q_in, q_out, dt):
        out, smax, flags = oracle.step(self.op, q_in, dt)
        assert flags == 0
        q_out[...] = out
        return smax

    def max_speed(self, q):
        return oracle.max_cell_speed(self.op, q)


def initial(solver, mx, my, seed=3):
    rng = np.random.default_rng(seed)
    if solver == mc.ADVECTION:
        return rng.uniform(0, 1, (1, my, mx))
    if solver == mc.ACOUSTICS:
        return np.stack([rng.uniform(-1, 1, (my, mx)), 0.3 * rng.uniform(-1, 1, (my, mx)),
                         0.3 * rng.uniform(-1, 1, (my, mx))])
    if solver == mc.SWE_ROE:
        return np.stack([1 + 0.5 * rng.uniform(0, 1, (my, mx)), 0.2 * rng.uniform(-1, 1, (my, mx)),
                         0.2 * rng.uniform(-1, 1, (my, mx))])
    rho = 1 + 0.5 * rng.uniform(0, 1, (my, mx))
    return np.stack([rho, 0.3 * rho * rng.uniform(-1, 1, (my, mx)),
                     0.3 * rho * rng.uniform(-1, 1, (my, mx)), 2.5 + rng.uniform(0, 1, (my, mx))])


PARAM = {mc.ACOUSTICS: (1.0, 4.0), mc.SWE_ROE: (9.81,), mc.EULER_ROE: (1.4,), mc.ADVECTION: (1.0, -0.7)}


def global_problem(solver, mx, my, bc, transverse=1, limiter=mc.LIM_MC):
    return mc.Problem.make(solver, mx, my, 1.0 / mx, 1.0 / my, dtype=mc.F64, limiter=limiter,
                           transverse=transverse, bc=bc, param=PARAM[solver])


def scatter(decomp, q):
    """Block states (with empty ghosts) cut from a global interior."""
    out = []
    for r in range(decomp.nblocks):
        e = decomp.extent(r)
        a = np.zeros((q.shape[0], e.my + 4, e.mx + 4))
        a[:, 2:-2, 2:-2] = q[:, e.j0: e.j0 + e.my, e.i0: e.i0 + e.mx]
        out.append(a)
    return out


def gather(decomp, qs, nplane):
    p = decomp.problem
    g = np.full((nplane, p.my, p.mx), np.nan)
    for r, a in enumerate(qs):
        e = decomp.extent(r)
        g[:, e.j0: e.j0 + e.my, e.i0: e.i0 + e.mx] = a[:, 2:-2, 2:-2]
    return g


def global_run(p, q, nsteps):
    op = oracle_problem(p)
    a = np.zeros(op.shape)
    a[:, 2:-2, 2:-2] = q
    dt = 0.8 / oracle.max_cell_speed(op, a)
    out, t, dt, nrej, flags = oracle.advance(op, a, nsteps, 0.8, 1.0, 0.0, dt)
    assert flags == 0
    return out[:, 2:-2, 2:-2], t


def test_split_and_neighbours():
    assert split(10, 3) == ([4, 3, 3], [0, 4, 7])
    assert split(7, 1) == ([7], [0])
    p = global_problem(mc.SWE_ROE, 10, 9, (P, P, W, X))
    d = Decomposition(p, 3, 2)
    # x periodic over three blocks wraps; y keeps its physical kinds
    assert d.neighbour(0, 0) == 2 and d.neighbour(2, 1) == 0 and d.neighbour(1, 0) == 0
    assert d.neighbour(0, 2) is None and d.neighbour(0, 3) == 3 and d.neighbour(4, 3) is None
    lp = d.local_problem(4)
    assert (lp.mx, lp.my) == (3, 4) and list(lp.bc) == [G, G, G, X]
    # a periodic direction held by one block keeps its own kind
    d1 = Decomposition(p, 1, 2)
    assert list(d1.local_problem(0).bc) == [P, P, W, G]
    with pytest.raises(ValueError):
        Decomposition(p, 6, 1)


@pytest.mark.parametrize("px,py,bc", [(2, 2, (P, P, P, P)), (3, 2, (W, X, P, P)), (2, 3, (P, P, W, W)),
                                      (1, 2, (X, W, P, P))])
def test_messages_pair_up_in_order(px, py, bc):
    """Every send meets the receive of its ghosts, and between each ordered
    pair of ranks the tags of the sends come in the order of the receives."""
    d = Decomposition(global_problem(mc.SWE_ROE, 12, 12, bc), px, py)
    for direction in (0, 1):
        sent, wanted = {}, {}
        for r in range(d.nblocks):
            sends, recvs = d.messages(r, direction)
            for side, dst in sends:
                sent.setdefault((r, dst), []).append(side ^ 1)
            for side, src in recvs:
                wanted.setdefault((src, r), []).append(side)
        assert sent == wanted


@pytest.mark.parametrize("solver,bc,px,py,trans", [
    (mc.SWE_ROE, (W, W, W, W), 2, 2, 1),
    (mc.SWE_ROE, (P, P, W, X), 3, 2, 1),
    (mc.EULER_ROE, (X, X, X, X), 2, 3, 2),
    (mc.ACOUSTICS, (P, P, P, P), 2, 2, 1),
    (mc.ADVECTION, (P, P, P, P), 3, 3, 1),
    (mc.ADVECTION, (X, W, P, P), 1, 2, 0),
])
def test_local_blocks_equal_single_grid(solver, bc, px, py, trans):
    mx, my = 13, 11
    p = global_problem(solver, mx, my, bc, transverse=trans)
    q = initial(solver, mx, my)
    want, t_want = global_run(p, q, 3)
    d = Decomposition(p, px, py)
    blocks = [Block(d, r, OracleOps(d.local_problem(r))) for r in range(d.nblocks)]
    qa = scatter(d, q)
    qb = [np.zeros_like(a) for a in qa]
    t, dt, in_b, nrej = Stepper(blocks).advance(qa, qb, 3, 0.8, 1.0)
    got = gather(d, qb if in_b else qa, q.shape[0])
    assert t == t_want
    np.testing.assert_array_equal(got, want)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, args, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    solver, bc, px, py, mx, my, nsteps = args
    p = global_problem(solver, mx, my, bc)
    d = Decomposition(p, px, py)
    q = initial(solver, mx, my)
    block = Block(d, rank, OracleOps(d.local_problem(rank)))
    qa = scatter(d, q)[rank]
    qb = np.zeros_like(qa)
    t, dt, in_b, nrej = Stepper([block], DistTransport()).advance([qa], [qb], nsteps, 0.8, 1.0)
    out[rank] = ((qb if in_b else qa).copy(), t)
    dist.destroy_process_group()


@pytest.mark.parametrize("solver,bc,px,py", [
    (mc.SWE_ROE, (P, P, W, W), 2, 1),          # both x sides of each rank face the other rank
    (mc.EULER_ROE, (X, W, P, P), 2, 2),
])
def test_gloo_ranks_equal_single_grid(solver, bc, px, py):
    import torch.multiprocessing as mp
    mx, my, nsteps = 12, 10, 3
    world = px * py
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(world, _free_port(), (solver, bc, px, py, mx, my, nsteps), out),
             nprocs=world, join=True)
    p = global_problem(solver, mx, my, bc)
    q = initial(solver, mx, my)
    want, t_want = global_run(p, q, nsteps)
    d = Decomposition(p, px, py)
    got = gather(d, [out[r][0] for r in range(world)], q.shape[0])
    assert all(out[r][1] == t_want for r in range(world))
    np.testing.assert_array_equal(got, want)


def test_lpt_shards():
    """Greedy longest-processing-time sharing of independent units: every
    unit in exactly one shard, shards sorted, the list-scheduling bound
    (heaviest part <= total / parts + (1 - 1/parts) largest unit), one part =
    everything, and the textbook instance where LPT misses the optimum."""
    from paper_1308_1464_gb300.blocks import lpt_shards
    rng = np.random.default_rng(5)
    for parts in (1, 2, 3, 8):
        w = [int(x) for x in rng.integers(1, 5000, 997)]
        shards = lpt_shards(w, parts)
        assert len(shards) == parts
        flat = sorted(k for s in shards for k in s)
        assert flat == list(range(len(w)))
        assert all(s == sorted(s) for s in shards)
        loads = [sum(w[k] for k in s) for s in shards]
        assert max(loads) <= sum(w) / parts + (1 - 1 / parts) * max(w)
    assert lpt_shards([3, 1, 2], 1) == [[0, 1, 2]]
    # textbook case: 3, 3, 2, 2, 2 on two machines, LPT gives 7 against the optimum 6
    loads = sorted(sum([3, 3, 2, 2, 2][k] for k in s) for s in lpt_shards([3, 3, 2, 2, 2], 2))
    assert loads == [5, 7]


def test_patch_subset_matches_whole_set():
    """A rank's share of the seeded patch set equals those patches of the
    whole set."""
    from paper_1308_1464_gb300 import workloads
    whole = workloads.swe_patches(40)
    some = workloads.swe_patches(40, only=[3, 17, 39])
    for k, p in zip([3, 17, 39], some):
        assert (p.nx, p.ny) == (whole[k].nx, whole[k].ny)
        np.testing.assert_array_equal(p.grid.q, whole[k].grid.q)


@pytest.mark.parametrize("name", ["swe_dambreak", "euler_quadrants", "advection_pulse",
                                  "acoustics_layered", "acoustics_pulse"])
def test_grid_window_matches_whole_grid(name):
    """A block's window of a seeded grid equals that slice of the whole grid
    (same counter-based draws, same cell centres), and its x_lo, y_lo locate
    the window's first cell."""
    from paper_1308_1464_gb300 import workloads
    f = getattr(workloads, name)
    whole = f(37, 29)
    for i0, j0, nx, ny in ((0, 0, 37, 29), (5, 3, 17, 11), (36, 28, 1, 1), (0, 20, 37, 9)):
        part = f(37, 29, window=(i0, j0, nx, ny))
        np.testing.assert_array_equal(part.q, whole.q[:, j0:j0 + ny, i0:i0 + nx])
        assert (part.dx, part.dy) == (whole.dx, whole.dy)
        assert part.x_lo == pytest.approx(whole.x_lo + i0 * whole.dx)
        assert part.y_lo == pytest.approx(whole.y_lo + j0 * whole.dy)
    with pytest.raises(ValueError):
        f(37, 29, window=(30, 0, 8, 4))
