"""Blocks of a decomposed grid on the GPU: halo strips, directional ghost
fills, and decomposed runs against the single grid.

* mc_halo_pack / mc_halo_unpack move exactly the cells the strip layout
  names (compared with slices of the downloaded array, bit for bit);
* mc_bc_fill_dir(0) then (1) equals mc_bc_fill, and with MC_BC_GIVEN sides
  the fill equals the oracle's, which leaves those sides alone;
* a run over 2 x 2 and 3 x 2 blocks exchanging halos in one process equals
  the single-grid run of the same kernels bit for bit (every cell reads the
  same values; the global smax is the maximum of the same edge speeds), and
  the oracle within the parity tolerance;
* two gloo ranks on this one GPU, exchanging host-staged strips through
  torch.distributed, give the same bits.  Their kernels never wait on each
  other: every exchange is a host-side send and receive between launches.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import paper_1308_1464_gb300 as mc
from gpu_util import TOL, embed, initial_state, problems, scaled_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1308_1464_gb300.blocks import (Block, Decomposition, DeviceBlockOps,  # noqa: E402
                                          DistTransport, Stepper)
from paper_1308_1464_gb300.state import DeviceState  # noqa: E402

P, X, W, G = mc.BC_PERIODIC, mc.BC_EXTRAP, mc.BC_WALL, mc.BC_GIVEN


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1308_1464_gb300 import _build
    _build.build()
    oracle.build()


def random_state(ctx, seed):
    """A state whose every element (ghosts and padding too) is random."""
    s = DeviceState(ctx)
    g = torch.Generator(device="cpu").manual_seed(seed)
    vals = torch.rand(s.buf.numel() // (8 if s.t_dtype == torch.float64 else 4), generator=g,
                      dtype=torch.float64) + 0.5
    s.buf.view(s.t_dtype).copy_(vals.to(s.t_dtype).cuda())
    return s


@pytest.mark.parametrize("dtype", [mc.F32, mc.F64])
def test_halo_strips(dtype):
    mx, my = 37, 9
    p, _ = problems("euler", mx, my, 0.1, 0.1, dtype, (G, G, G, G))
    with mc.Context(p) as ctx:
        s = random_state(ctx, 1)
        full = s.with_ghosts()                                  # (meqn, my + 4, mx + 4)
        for side in range(4):
            n = ctx.halo_elems(side)
            buf = torch.empty(n, dtype=s.t_dtype, device="cuda")
            ctx.halo_pack(s.ptr, side, buf.data_ptr())
            if side < 2:
                cols = slice(2, 4) if side == 0 else slice(mx, mx + 2)
                want = full[:, 2:2 + my, cols]
            else:
                rows = slice(2, 4) if side == 2 else slice(my, my + 2)
                want = full[:, rows, :]
            assert n == want.size
            torch.cuda.synchronize()
            np.testing.assert_array_equal(buf.cpu().numpy().reshape(want.shape), want)
        # unpack fresh strips into the ghosts, nothing else changes
        t = random_state(ctx, 2)
        before = t.with_ghosts()
        expect = before.copy()
        for side in range(4):
            n = ctx.halo_elems(side)
            strip = (torch.arange(n, dtype=torch.float64) * 0.25 + side).to(s.t_dtype)
            ctx.halo_unpack(strip.cuda().data_ptr(), side, t.ptr)
            torch.cuda.synchronize()
            if side < 2:
                cols = slice(0, 2) if side == 0 else slice(mx + 2, mx + 4)
                expect[:, 2:2 + my, cols] = strip.numpy().reshape(expect[:, 2:2 + my, cols].shape)
            else:
                rows = slice(0, 2) if side == 2 else slice(my + 2, my + 4)
                expect[:, rows, :] = strip.numpy().reshape(expect[:, rows, :].shape)
        np.testing.assert_array_equal(t.with_ghosts(), expect)


@pytest.mark.parametrize("bc", [(P, P, P, P), (W, X, P, P), (X, W, W, X), (W, W, W, W)])
@pytest.mark.parametrize("dtype", [mc.F32, mc.F64])
def test_directional_fill_equals_fill(bc, dtype):
    p, _ = problems("swe", 23, 14, 0.1, 0.1, dtype, bc)
    with mc.Context(p) as ctx:
        a, b = random_state(ctx, 3), random_state(ctx, 3)
        ctx.bc_fill(a.ptr)
        ctx.bc_fill_dir(b.ptr, 0)
        ctx.bc_fill_dir(b.ptr, 1)
        np.testing.assert_array_equal(a.with_ghosts(), b.with_ghosts())


@pytest.mark.parametrize("bc", [(G, W, X, G), (G, G, P, P), (P, P, G, W), (G, G, G, G)])
def test_fill_leaves_given_sides(bc):
    p, op = problems("swe", 19, 12, 0.1, 0.1, mc.F64, bc)
    with mc.Context(p) as ctx:
        a = random_state(ctx, 4)
        before = a.with_ghosts()
        ctx.bc_fill(a.ptr)
        want = oracle.bc_fill(op, before)                      # GIVEN sides untouched
        np.testing.assert_array_equal(a.with_ghosts(), want)


def test_given_sides_rejected_where_unsupported():
    p, _ = problems("swe", 16, 16, 0.1, 0.1, mc.F32, (G, W, W, W))
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        with pytest.raises(mc.McError):
            ctx.advance(a.ptr, b.ptr, 1, 0.9, 1.0, 0.0, 1e-3)
    narrow, _ = problems("swe", 1, 8, 0.1, 0.1, mc.F32, (G, W, W, W))
    with pytest.raises(mc.McError):
        mc.Context(narrow)                                     # a strip needs two columns


def single_grid(p, q, nsteps, cfl=0.8):
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(q)
        dt = cfl / ctx.max_cell_speed(a.ptr)
        t, dt, in_b, nrej = ctx.advance(a.ptr, b.ptr, nsteps, cfl, 1.0, 0.0, dt)
        return (b if in_b else a).download(), t


def decomposed(p, q, px, py, nsteps, cfl=0.8):
    d = Decomposition(p, px, py)
    ctxs = [mc.Context(d.local_problem(r)) for r in range(d.nblocks)]
    blocks = [Block(d, r, DeviceBlockOps(c)) for r, c in enumerate(ctxs)]
    qa, qb = [], []
    for r, c in enumerate(ctxs):
        e = d.extent(r)
        a, b = DeviceState(c).zero_(), DeviceState(c).zero_()
        a.upload(q[:, e.j0: e.j0 + e.my, e.i0: e.i0 + e.mx])
        qa.append(a)
        qb.append(b)
    t, dt, in_b, nrej = Stepper(blocks).advance([s.ptr for s in qa], [s.ptr for s in qb],
                                                nsteps, cfl, 1.0)
    out = np.zeros(q.shape, dtype=qa[0].np_dtype)
    for r in range(d.nblocks):
        e = d.extent(r)
        out[:, e.j0: e.j0 + e.my, e.i0: e.i0 + e.mx] = (qb[r] if in_b else qa[r]).download()
    for c in ctxs:
        c.close()
    return out, t


CASES = [
    ("swe", mc.F32, (W, W, W, W), 2, 2, 1),
    ("swe", mc.F32, (P, P, W, X), 3, 2, 1),
    ("euler", mc.F32, (X, X, X, X), 2, 3, 2),
    ("euler", mc.F64, (P, P, P, P), 2, 2, 1),
    ("acoustics", mc.F64, (P, P, P, P), 3, 3, 1),
    ("advection", mc.F32, (P, P, X, W), 2, 2, 0),
]


@pytest.mark.parametrize("solver,dtype,bc,px,py,trans", CASES)
def test_blocks_equal_single_grid(solver, dtype, bc, px, py, trans):
    mx, my, nsteps = 75, 61, 4
    q, dx, dy = initial_state(solver, mx, my, seed=9)
    p, op = problems(solver, mx, my, dx, dy, dtype, bc, transverse=trans)
    qin = q.astype(np.float64 if dtype == mc.F64 else np.float32)
    want, t_want = single_grid(p, qin, nsteps)
    got, t = decomposed(p, qin, px, py, nsteps)
    assert t == t_want
    np.testing.assert_array_equal(got, want)
    ref, _, _, _, flags = oracle.advance(op, embed(op, qin.astype(np.float64)), nsteps, 0.8, 1.0, 0.0,
                                         0.8 / oracle.max_cell_speed(op, embed(op, qin.astype(np.float64))))
    assert scaled_error(solver, got.astype(np.float64), ref[:, 2:-2, 2:-2]) <= TOL[dtype] * nsteps


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
    torch.cuda.set_device(0)
    solver, dtype, bc, px, py, mx, my, nsteps = args
    q, dx, dy = initial_state(solver, mx, my, seed=9)
    p, _ = problems(solver, mx, my, dx, dy, dtype, bc)
    qin = q.astype(np.float64 if dtype == mc.F64 else np.float32)
    d = Decomposition(p, px, py)
    e = d.extent(rank)
    with mc.Context(d.local_problem(rank)) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(qin[:, e.j0: e.j0 + e.my, e.i0: e.i0 + e.mx])
        st = Stepper([Block(d, rank, DeviceBlockOps(ctx))], DistTransport())
        t, dt, in_b, nrej = st.advance([a.ptr], [b.ptr], nsteps, 0.8, 1.0)
        out[rank] = ((b if in_b else a).download(), t)
    dist.destroy_process_group()


def test_gloo_ranks_on_one_gpu_equal_single_grid():
    import torch.multiprocessing as mp
    solver, dtype, bc, px, py, mx, my, nsteps = "swe", mc.F32, (P, P, W, W), 2, 1, 64, 40, 3
    mgr = mp.get_context("spawn").Manager()   # no fork of a process that holds a CUDA context
    out = mgr.dict()
    mp.spawn(_rank, args=(2, _free_port(), (solver, dtype, bc, px, py, mx, my, nsteps), out),
             nprocs=2, join=True)
    q, dx, dy = initial_state(solver, mx, my, seed=9)
    p, _ = problems(solver, mx, my, dx, dy, dtype, bc)
    want, t_want = single_grid(p, q.astype(np.float32), nsteps)
    d = Decomposition(p, px, py)
    got = np.zeros_like(want)
    for r in range(2):
        e = d.extent(r)
        got[:, e.j0: e.j0 + e.my, e.i0: e.i0 + e.mx] = out[r][0]
        assert out[r][1] == t_want
    np.testing.assert_array_equal(got, want)


def decomposed_device(p, q, px, py, nsteps, cfl=0.8, dt0=None, stream=None, graph=True):
    """The decomposed run with the time-step state on the device
    (DeviceStepper over mc_block_*), all blocks in this process, on the
    given torch stream (default: the default stream)."""
    from paper_1308_1464_gb300.blocks import DeviceStepper
    d = Decomposition(p, px, py)
    ctxs = [mc.Context(d.local_problem(r)) for r in range(d.nblocks)]
    sh = stream.cuda_stream if stream is not None else 0
    blocks = [Block(d, r, DeviceBlockOps(c, sh)) for r, c in enumerate(ctxs)]
    qa, qb = [], []
    for r, c in enumerate(ctxs):
        e = d.extent(r)
        a, b = DeviceState(c).zero_(), DeviceState(c).zero_()
        a.upload(q[:, e.j0: e.j0 + e.my, e.i0: e.i0 + e.mx])
        qa.append(a)
        qb.append(b)
    torch.cuda.synchronize()
    t, dt, in_b, nrej = DeviceStepper(blocks, graph=graph).advance(
        [s.ptr for s in qa], [s.ptr for s in qb], nsteps, cfl, 1.0, dt=dt0)
    torch.cuda.synchronize()
    out = np.zeros(q.shape, dtype=qa[0].np_dtype)
    for r in range(d.nblocks):
        e = d.extent(r)
        out[:, e.j0: e.j0 + e.my, e.i0: e.i0 + e.mx] = (qb[r] if in_b else qa[r]).download()
    for c in ctxs:
        c.close()
    return out, t, dt, nrej


@pytest.mark.parametrize("solver,dtype,bc,px,py", [("swe", mc.F32, (W, W, W, W), 2, 2),
                                                   ("euler", mc.F64, (P, P, X, X), 3, 2)])
def test_device_stepper_equals_single_grid(solver, dtype, bc, px, py):
    """The device-side loop (halo exchange of the current buffer, step with
    the device dt, max-reduction, accept/reject on the device) equals the
    single-grid mc_advance bit for bit, a rejected first attempt included."""
    mx, my, nsteps = 75, 61, 5
    q, dx, dy = initial_state(solver, mx, my, seed=9)
    p, _ = problems(solver, mx, my, dx, dy, dtype, bc)
    qin = q.astype(np.float64 if dtype == mc.F64 else np.float32)
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(qin)
        dt0 = 3.0 * 0.8 / ctx.max_cell_speed(a.ptr)          # rejected, then retaken
        t_w, dt_w, inb_w, nrej_w = ctx.advance(a.ptr, b.ptr, nsteps, 0.8, 1.0, 0.0, dt0)
        want = (b if inb_w else a).download()
    got, t, dt, nrej = decomposed_device(p, qin, px, py, nsteps, dt0=dt0)
    assert nrej == nrej_w >= 1
    assert t == t_w and dt == dt_w
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("graph", [True, False])
def test_device_stepper_on_a_side_stream(graph):
    """Blocks whose operations run on a stream other than torch's current
    one: the halo copies, the max-reduction and the graph replays queue on
    that stream too, so the run equals the default-stream run bit for bit."""
    mx, my, nsteps = 75, 61, 6
    q, dx, dy = initial_state("swe", mx, my, seed=4)
    p, _ = problems("swe", mx, my, dx, dy, mc.F32, (W, W, W, W))
    qin = q.astype(np.float32)
    want, t_w, dt_w, nrej_w = decomposed_device(p, qin, 2, 2, nsteps, graph=graph)
    got, t, dt, nrej = decomposed_device(p, qin, 2, 2, nsteps, stream=torch.cuda.Stream(),
                                         graph=graph)
    assert (t, dt, nrej) == (t_w, dt_w, nrej_w)
    np.testing.assert_array_equal(got, want)


def _rank_device(rank, world, port, args, out):
    import torch.distributed as dist
    from paper_1308_1464_gb300.blocks import DeviceStepper
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    solver, dtype, bc, px, py, mx, my, nsteps = args
    q, dx, dy = initial_state(solver, mx, my, seed=9)
    p, _ = problems(solver, mx, my, dx, dy, dtype, bc)
    qin = q.astype(np.float64 if dtype == mc.F64 else np.float32)
    d = Decomposition(p, px, py)
    e = d.extent(rank)
    with mc.Context(d.local_problem(rank)) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(qin[:, e.j0: e.j0 + e.my, e.i0: e.i0 + e.mx])
        st = DeviceStepper([Block(d, rank, DeviceBlockOps(ctx))], DistTransport())
        t, dt, in_b, nrej = st.advance([a.ptr], [b.ptr], nsteps, 0.8, 1.0)
        out[rank] = ((b if in_b else a).download(), t)
    dist.destroy_process_group()


def test_gloo_ranks_device_stepper_equal_single_grid():
    """Two gloo ranks on this one GPU run the device-side loop; strips and the
    speed maximum go through host memory (gloo), decisions stay on the
    device.  No kernel waits on another rank's: every exchange happens
    between launches."""
    import torch.multiprocessing as mp
    solver, dtype, bc, px, py, mx, my, nsteps = "swe", mc.F32, (P, P, W, W), 2, 1, 64, 40, 3
    mgr = mp.get_context("spawn").Manager()   # no fork of a process that holds a CUDA context
    out = mgr.dict()
    mp.spawn(_rank_device, args=(2, _free_port(), (solver, dtype, bc, px, py, mx, my, nsteps), out),
             nprocs=2, join=True)
    q, dx, dy = initial_state(solver, mx, my, seed=9)
    p, _ = problems(solver, mx, my, dx, dy, dtype, bc)
    want, t_want = single_grid(p, q.astype(np.float32), nsteps)
    d = Decomposition(p, px, py)
    got = np.zeros_like(want)
    for r in range(2):
        e = d.extent(r)
        got[:, e.j0: e.j0 + e.my, e.i0: e.i0 + e.mx] = out[r][0]
        assert out[r][1] == t_want
    np.testing.assert_array_equal(got, want)


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench_line(cmd, timeout=900):
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable] + cmd, cwd=ROOT, capture_output=True, text=True,
                       timeout=timeout)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert lines, r.stdout[-2000:]
    return json.loads(lines[-1])


def test_bench_blocks_in_one_process():
    """bench.py's decomposed-grid path with every block on this GPU: 2 x 2
    blocks of 256^2 cells, K accepted steps, launches counted per attempt."""
    line = _bench_line(["bench.py", "--blocks", "2x2", "--size", "256", "--steps", "6",
                        "--warmup", "3", "--no-e2e"])
    assert line["config"]["blocks"] == [2, 2] and line["config"]["mx"] == 512
    assert line["value"] > 0 and line["steps"] == 6
    # per attempt and block: 2 directions x (1 pack + 1 unpack + 1 fill), the
    # step kernel and the guard kernel of FP32 shallow water, the dt rule
    assert line["gpu_launches"] == 4 * (2 * 3 + 2 + 1) * (6 + line["config"]["rejected_steps"])


def test_bench_blocks_two_gloo_ranks():
    """The multi-rank path of bench.py (torchrun, one block per rank) with
    two gloo ranks sharing this GPU: strips and the speed maximum are staged
    through host memory between launches, so no kernel waits on the other
    rank.  Rank 0 prints one line for the whole job."""
    port = _free_port()
    line = _bench_line(["-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
                        "--dist-backend", "gloo", "--size", "192", "--steps", "4", "--warmup", "3"])
    assert line["n_gpus"] == 2 and line["config"]["blocks"] == [2, 1]
    assert line["config"]["parallelism"] == "blocks"
    assert line["value"] > 0 and line["e2e"]["value"] > 0
