"""GPU parity of the fused step (K1) and ghost fill (K2) against the oracle.

Every case calls the CUDA library through its C ABI (mc_step) and compares
with the FP64 oracle run on the same (precision-rounded) input with the same
dt.  The tolerance is the field-scaled max error of one step: 1e-12 for FP64,
2e-5 for FP32.
"""
import numpy as np
import pytest

import oracle
import paper_1308_1464_gb300 as mc
from paper_1308_1464_gb300 import workloads
from gpu_util import (TOL, embed, field_scales, initial_state, problems, scaled_error,
                      window_step)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1308_1464_gb300.state import DeviceState  # noqa: E402

W, X, P = mc.BC_WALL, mc.BC_EXTRAP, mc.BC_PERIODIC


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1308_1464_gb300 import _build
    _build.build()
    oracle.build()


def run_step(p, op, q_interior, cfl=0.9, tile_rows=None):
    """One GPU step and the oracle's step on the same rounded input."""
    npdt = np.float64 if p.dtype == mc.F64 else np.float32
    qin = q_interior.astype(npdt)
    qo = embed(op, qin.astype(np.float64))
    dt = cfl / oracle.max_cell_speed(op, oracle.bc_fill(op, qo))
    with mc.Context(p) as ctx:
        if tile_rows:
            ctx.set_tile_rows(tile_rows)
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(qin)
        smax = ctx.step(a.ptr, b.ptr, dt)
        got = b.download().astype(np.float64)
        ghosts = a.with_ghosts().astype(np.float64)
    want, smax_ref, _ = oracle.step(op, qo, dt)
    return got, want[:, 2:-2, 2:-2], smax, smax_ref, ghosts, oracle.bc_fill(op, qo)


CASES = [
    ("acoustics", mc.F64, (P, P, P, P), 4, 1),
    ("acoustics", mc.F32, (W, X, P, P), 1, 1),
    ("swe", mc.F32, (W, W, W, W), 4, 1),
    ("swe", mc.F64, (W, W, W, W), 4, 1),
    ("swe", mc.F32, (X, X, P, P), 1, 1),
    ("swe", mc.F64, (P, P, X, W), 0, 1),
    ("swe", mc.F32, (W, X, X, W), 4, 0),
    ("euler", mc.F32, (X, X, X, X), 4, 1),
    ("euler", mc.F64, (X, X, X, X), 4, 1),
    ("euler", mc.F32, (W, W, P, P), 1, 1),
    ("euler", mc.F64, (P, P, W, X), 4, 0),
    # advection, the superbee and van Leer limiters, transverse option 2
    ("advection", mc.F32, (P, P, P, P), 4, 1),
    ("advection", mc.F64, (W, X, P, P), 2, 2),
    ("advection", mc.F32, (X, X, W, W), 3, 2),
    ("advection", mc.F64, (P, P, X, X), 0, 0),
    ("acoustics", mc.F64, (P, P, W, W), 3, 2),
    ("acoustics", mc.F32, (W, W, P, P), 2, 2),
    ("swe", mc.F32, (W, W, W, W), 2, 2),
    ("swe", mc.F64, (X, W, P, P), 3, 2),
    ("swe", mc.F32, (W, X, X, W), 4, 2),
    ("euler", mc.F32, (X, X, X, X), 3, 2),
    ("euler", mc.F64, (W, W, X, X), 4, 2),
    ("euler", mc.F32, (P, P, W, W), 2, 1),
    # variable-coefficient acoustics (material planes carried with the state)
    ("acoustics_var", mc.F64, (P, P, P, P), 4, 1),
    ("acoustics_var", mc.F32, (W, X, P, P), 3, 2),
    ("acoustics_var", mc.F64, (X, X, W, W), 1, 0),
    ("acoustics_var", mc.F32, (W, W, W, W), 2, 1),
    # Euler with the exact-solution normal solve
    ("euler_godunov", mc.F32, (X, X, X, X), 4, 1),
    ("euler_godunov", mc.F64, (W, W, P, P), 3, 2),
    ("euler_godunov", mc.F32, (P, P, X, X), 1, 0),
    ("euler_godunov", mc.F64, (X, X, X, X), 4, 1),
]


@pytest.mark.parametrize("solver,dtype,bc,lim,trans", CASES)
def test_step_parity(solver, dtype, bc, lim, trans):
    mx, my = 70, 45   # 3 bands (29 + 29 + 12 columns), several row tiles, ragged tails
    q, dx, dy = initial_state(solver, mx, my, seed=3)
    p, op = problems(solver, mx, my, dx, dy, dtype, bc, limiter=lim, transverse=trans)
    got, want, smax, smax_ref, ghosts, ghosts_ref = run_step(p, op, q, tile_rows=8)
    err = scaled_error(solver, got, want)
    assert err <= TOL[dtype], f"field-scaled error {err:.3e}"
    assert smax == pytest.approx(smax_ref, rel=1e-13 if dtype == mc.F64 else 2e-6)
    # ghost layers of the input filled like the oracle's
    np.testing.assert_array_equal(ghosts, ghosts_ref.astype(np.float32 if dtype == mc.F32 else np.float64)
                                  .astype(np.float64))


def test_first_order_and_no_limiter():
    for order, lim in ((1, 4), (2, 0)):
        q, dx, dy = initial_state("swe", 40, 33, seed=5)
        p, op = problems("swe", 40, 33, dx, dy, mc.F64, (W, X, X, W), limiter=lim, order=order)
        got, want, *_ = run_step(p, op, q, tile_rows=16)
        assert scaled_error("swe", got, want) <= 1e-12


@pytest.mark.parametrize("mx,my", [(1, 1), (1, 7), (7, 1), (2, 3), (29, 2), (30, 31), (59, 5),
                                   (58, 9), (87, 3)])
@pytest.mark.parametrize("solver,dtype,bc,trans", [("swe", mc.F64, (W, W, W, W), 1),
                                                   ("euler", mc.F32, (X, X, P, P), 1),
                                                   ("acoustics", mc.F64, (P, P, W, W), 1),
                                                   ("swe", mc.F32, (W, X, X, W), 2),
                                                   ("advection", mc.F64, (P, P, X, W), 2),
                                                   ("acoustics_var", mc.F32, (X, W, P, P), 2),
                                                   ("euler_godunov", mc.F32, (W, X, X, W), 1)])
def test_tiny_and_odd_grids(mx, my, solver, dtype, bc, trans):
    q, _, _ = initial_state(solver, max(mx, 4), max(my, 4), seed=mx * 100 + my)
    q = np.ascontiguousarray(q[:, :my, :mx])
    p, op = problems(solver, mx, my, 0.01, 0.013, dtype, bc, transverse=trans)
    got, want, smax, smax_ref, ghosts, ghosts_ref = run_step(p, op, q, cfl=0.5)
    assert scaled_error(solver, got, want) <= TOL[dtype]
    assert smax == pytest.approx(smax_ref, rel=1e-12 if dtype == mc.F64 else 2e-6)


@pytest.mark.parametrize("solver,dtype,trans", [("swe", mc.F32, 1), ("euler", mc.F64, 1),
                                                ("swe", mc.F32, 2), ("euler", mc.F32, 2),
                                                ("acoustics", mc.F64, 1), ("swe", mc.F64, 1)])
def test_tile_shape_invariance(solver, dtype, trans):
    """Results do not depend on the tile height, down to one row per warp
    task (the small grids' tiles): bitwise equal outputs."""
    mx, my = 100, 130
    q, dx, dy = initial_state(solver, mx, my, seed=9)
    p, op = problems(solver, mx, my, dx, dy, dtype, (W, X, X, W), transverse=trans)
    outs = [run_step(p, op, q, tile_rows=t)[0] for t in (8, 1, 2, 3, 5, 17, 64, 256)]
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


FULL = [
    ("swe", mc.F32, 4096, 4096, (W, W, W, W), {}),     # shallow-water dam break, bench configuration
    ("swe", mc.F64, 4096, 4096, (W, W, W, W), {}),
    ("euler", mc.F32, 4096, 4096, (X, X, X, X), {}),   # four-quadrant Euler
    ("advection", mc.F32, 4096, 4096, (P, P, P, P), {}),
    ("acoustics_var", mc.F32, 4096, 4096, (X, X, X, X), {}),
    ("swe", mc.F32, 4096, 4096, (W, W, W, W), dict(limiter=3, transverse=2)),
    ("euler_godunov", mc.F32, 4096, 4096, (X, X, X, X), {}),
]


@pytest.mark.parametrize("solver,dtype,mx,my,bc,opts", FULL)
def test_full_size_windows(solver, dtype, mx, my, bc, opts):
    """Full-size grid, default launch configuration: 40 windows of 8 x 8 cells
    (corners, edges, random interior) recomputed by the oracle from the GPU
    step's filled input, plus conservation of mass across the walls/extrapolation."""
    if solver == "swe":
        g = workloads.swe_dambreak(mx, my)
    elif solver == "advection":
        g = workloads.advection_pulse(mx, my)
    elif solver == "acoustics_var":
        g = workloads.acoustics_layered(mx, my)
    else:   # Euler, either normal solve
        g = workloads.euler_quadrants(mx, my)
    p, op = problems(solver, mx, my, g.dx, g.dy, dtype, bc, **opts)
    if solver == "advection":
        p.param[0], p.param[1] = 1.0, 0.6
        op.param = (1.0, 0.6, 0, 0)
    npdt = np.float64 if dtype == mc.F64 else np.float32
    qin = g.q.astype(npdt)
    # dt from the oracle's cell-speed rule on the same rounded input
    dt = 0.9 / oracle.max_cell_speed(op, embed(op, qin.astype(np.float64)))
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(qin)
        ctx.step(a.ptr, b.ptr, dt)
        full_in = a.with_ghosts().astype(np.float64)
        out = b.download().astype(np.float64)
    S = field_scales(solver, full_in[:, 2:-2, 2:-2])
    rng = np.random.default_rng(17)
    w = h = 8
    spots = [(0, 0), (mx - w, 0), (0, my - h), (mx - w, my - h), (mx // 2 - 4, 0), (0, my // 2)]
    spots += [(int(rng.integers(0, mx - w)), int(rng.integers(0, my - h))) for _ in range(34)]
    for (i0, j0) in spots:
        want = window_step(op, full_in, dt, i0, j0, w, h)
        got = out[:, j0: j0 + h, i0: i0 + w]
        err = max(np.abs(got[m] - want[m]).max() / S[m] for m in range(want.shape[0]))
        assert err <= TOL[dtype], (i0, j0, err)
    # mass is conserved by walls exactly; with extrapolation it changes only by boundary fluxes
    if solver == "swe":
        m0, m1 = qin[0].astype(np.float64).sum(), out[0].sum()
        rel = abs(m1 - m0) / m0
        assert rel <= (1e-13 if dtype == mc.F64 else 1e-6), rel


def _transonic_state(solver, mx, my, axis, seed):
    """A Riemann problem across the middle of the grid along `axis` whose
    left-going rarefaction is transonic (shallow water: h = 3, u_n = 1 against
    h = 1, u_n = 4; Euler: Toro's first test, rho, u_n, p = 1, 0.75, 1 against
    0.125, 0, 0.1), with 1% noise and a small tangential velocity."""
    rng = np.random.default_rng(seed)
    left = (np.arange(mx)[None, :] < mx // 2) if axis == 0 else (np.arange(my)[:, None] < my // 2)
    left = np.broadcast_to(left, (my, mx))
    noise = 1 + 0.01 * rng.uniform(-1, 1, (my, mx))
    vt = 0.1 * rng.uniform(-1, 1, (my, mx))
    if solver == "swe":
        q = np.zeros((3, my, mx))
        q[0] = np.where(left, 3.0, 1.0) * noise
        q[1 + axis] = q[0] * np.where(left, 1.0, 4.0)
        q[2 - axis] = q[0] * vt
        return q
    q = np.zeros((4, my, mx))
    rho = np.where(left, 1.0, 0.125) * noise
    un = np.where(left, 0.75, 0.0)
    p = np.where(left, 1.0, 0.1)
    q[0] = rho
    q[1 + axis] = rho * un
    q[2 - axis] = rho * vt
    q[3] = p / (1.4 - 1) + 0.5 * rho * (un * un + vt * vt)
    return q


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("solver,dtype", [("swe", mc.F32), ("swe", mc.F64),
                                          ("euler", mc.F32), ("euler", mc.F64)])
def test_entropy_fix_transonic(solver, dtype, axis):
    """Harten-Hyman fix at a transonic rarefaction normal to x and to y (the
    FP32 step solves an x-edge and a y-edge side by side, so both halves of
    that path are exercised).  The fix must matter here: the oracle without it
    differs by far more than the parity tolerance."""
    mx, my = 40, 36
    q = _transonic_state(solver, mx, my, axis, seed=11 + axis)
    bc = (X, X, X, X)
    p, op = problems(solver, mx, my, 0.01, 0.01, dtype, bc, efix=1)
    got, want, smax, smax_ref, *_ = run_step(p, op, q)
    assert scaled_error(solver, got, want) <= TOL[dtype]
    _, op0 = problems(solver, mx, my, 0.01, 0.01, dtype, bc, efix=0)
    qo = embed(op0, q.astype(np.float32 if dtype == mc.F32 else np.float64).astype(np.float64))
    dt = 0.9 / oracle.max_cell_speed(op0, oracle.bc_fill(op0, qo))
    unfixed, _, _ = oracle.step(op0, qo, dt)
    assert scaled_error(solver, unfixed[:, 2:-2, 2:-2], want) > 50 * TOL[mc.F32]


@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("dtype", [mc.F32, mc.F64])
def test_godunov_transonic(dtype, axis):
    """The exact-solution normal solve at a transonic rarefaction (no entropy
    fix involved), along x and along y."""
    mx, my = 40, 36
    q = _transonic_state("euler", mx, my, axis, seed=21 + axis)
    p, op = problems("euler_godunov", mx, my, 0.01, 0.01, dtype, (X, X, X, X))
    got, want, smax, smax_ref, *_ = run_step(p, op, q)
    assert scaled_error("euler_godunov", got, want) <= TOL[dtype]
    assert smax == pytest.approx(smax_ref, rel=1e-12 if dtype == mc.F64 else 1e-5)
