"""Multi-step runs at the full benchmark sizes against the oracle, every cell.

The bench times mc_advance on 4096 x 4096 grids (ghost fill, fused step and
the device-side time-step rule in captured graphs).  Here the same call runs
10 steps of the shallow-water dam break (FP64 and FP32) and of the
four-quadrant Euler problem (FP32) from the bench's initial states, and the
oracle's driver runs the same 10 steps on all host cores; every interior
cell is compared.  FP64 must agree to rounding; FP32 within the per-step
tolerance times the number of steps (the FP32 run also takes its own dt
sequence, from FP32 speeds).
"""
import os

import numpy as np
import pytest

import oracle
import paper_1308_1464_gb300 as mc
from paper_1308_1464_gb300 import workloads
from gpu_util import TOL, embed, problems, scaled_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1308_1464_gb300.state import DeviceState  # noqa: E402

W, X = mc.BC_WALL, mc.BC_EXTRAP
NSTEPS = 10


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1308_1464_gb300 import _build
    _build.build()
    oracle.build()


CASES = [
    ("swe", mc.F64, (W, W, W, W), 0.9),
    ("swe", mc.F32, (W, W, W, W), 0.9),
    ("euler", mc.F32, (X, X, X, X), 0.8),
]


@pytest.mark.parametrize("solver,dtype,bc,cfl", CASES)
def test_ten_steps_full_size(solver, dtype, bc, cfl):
    n = 4096
    g = workloads.swe_dambreak(n, n) if solver == "swe" else workloads.euler_quadrants(n, n)
    p, op = problems(solver, n, n, g.dx, g.dy, dtype, bc)
    npdt = np.float64 if dtype == mc.F64 else np.float32
    qin = np.ascontiguousarray(g.q.astype(npdt))
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(qin)
        dt0 = cfl / ctx.max_cell_speed(a.ptr)
        t, dt, inb, nrej = ctx.advance(a.ptr, b.ptr, NSTEPS, cfl, 1.0, 0.0, dt0)
        got = (b if inb else a).download().astype(np.float64)
    qo = embed(op, qin.astype(np.float64))
    odt0 = cfl / oracle.max_cell_speed(op, oracle.bc_fill(op, qo))
    want, t_ref, _, nrej_ref, flags = oracle.advance(op, qo, NSTEPS, cfl, 1.0, 0.0, odt0,
                                                     nthreads=len(os.sched_getaffinity(0)))
    assert flags == 0 and nrej == nrej_ref == 0
    if dtype == mc.F64:
        assert t == pytest.approx(t_ref, rel=1e-13)
        tol = 1e-11
    else:
        assert t == pytest.approx(t_ref, rel=1e-5)
        tol = TOL[mc.F32] * NSTEPS
    err = scaled_error(solver, got, want[:, 2:-2, 2:-2])
    assert err <= tol, err


@pytest.mark.parametrize("solver,bc", [("swe", (W, W, W, W)), ("euler", (X, X, X, X))])
def test_default_layout_equals_uniform_tiles(solver, bc):
    """On a 4096^2 grid the default layout cuts most rows in 128-row tasks,
    launched first, and the last wave's worth in 64-row tasks; one step with
    it gives the bits of uniform 64-row tasks (and of uniform 32-row ones),
    speed maximum included."""
    n = 4096
    g = workloads.swe_dambreak(n, n) if solver == "swe" else workloads.euler_quadrants(n, n)
    p, _ = problems(solver, n, n, g.dx, g.dy, mc.F32, bc)
    qin = np.ascontiguousarray(g.q.astype(np.float32))
    outs = []
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(qin)
        dt = 0.8 / ctx.max_cell_speed(a.ptr)
        for rows in (0, 64, 32):
            ctx.set_tile_rows(rows)
            smax = ctx.step(a.ptr, b.ptr, dt)
            outs.append((b.download(), smax))
    for q, smax in outs[1:]:
        assert smax == outs[0][1]
        np.testing.assert_array_equal(q, outs[0][0])
