"""The FP64 guard of FP32 steps (paper §1.2, "local precision"): FP32 runs of
the shallow-water and Euler Roe solvers recompute in FP64 the normal solve
and transverse splits of edges across a near-dry or near-vacuum front (the
smaller depth or density below tau times the larger, tau = 1e-3 by default),
and the speeds and split of a near-sonic transonic entropy fix (a
characteristic speed within tau times the Roe sound speed of zero).

Each case runs one step through the C ABI with the guard on and off and
compares both with the FP64 oracle on the same FP32-rounded input at the
per-step tolerance 2e-5 (field-scaled).  The number of edges the guard
recomputed (mc_guard_stats) is predicted exactly on the CPU from the same
FP32 comparison the kernel makes."""
import numpy as np
import pytest

import oracle
import paper_1308_1464_gb300 as mc
from gpu_util import GAMMA, G, TOL, embed, scaled_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1308_1464_gb300.state import DeviceState  # noqa: E402

W, X = mc.BC_WALL, mc.BC_EXTRAP
TAU = np.float32(1e-3)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1308_1464_gb300 import _build
    _build.build()
    oracle.build()


def step(solver, q, bc, tau, dx=1.0 / 64):
    """One FP32 step with guard parameter tau and the oracle's FP64 step on
    the same rounded input -> (gpu, oracle, guarded edges, ghosted input)."""
    my, mx = q.shape[1], q.shape[2]
    sid, oid, g0 = ((mc.SWE_ROE, oracle.SWE, G) if solver == "swe"
                    else (mc.EULER_ROE, oracle.EULER, GAMMA))
    p = mc.Problem.make(sid, mx, my, dx, dx, dtype=mc.F32, bc=bc, param=(g0, 0, 0, tau))
    op = oracle.Problem(oid, mx, my, dx, dx, bc=tuple(bc), param=(g0, 0, 0, 0))
    q32 = q.astype(np.float32)
    qo = embed(op, q32.astype(np.float64))
    filled = oracle.bc_fill(op, qo)
    dt = 0.9 / oracle.max_cell_speed(op, filled)
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(q32)
        ctx.guard_stats(reset=True)
        ctx.step(a.ptr, b.ptr, dt)
        got = b.download().astype(np.float64)
        nguard = ctx.guard_stats(reset=True)
    want, _, _ = oracle.step(op, qo, dt)
    return got, want[:, 2:-2, 2:-2], nguard, filled


def predicted_guard_edges(filled, mx, my):
    """Interior x- and y-edges whose smaller first component (depth or
    density) is below tau times the larger, with the kernel's FP32 products."""
    h = filled[0].astype(np.float32)
    xl, xr = h[2:2 + my, 1:2 + mx], h[2:2 + my, 2:3 + mx]        # x-edges i - 1/2, i = 0..mx
    yl, yr = h[1:2 + my, 2:2 + mx], h[2:3 + my, 2:2 + mx]        # y-edges j - 1/2, j = 0..my
    nx = np.count_nonzero((xl < TAU * xr) | (xr < TAU * xl))
    ny = np.count_nonzero((yl < TAU * yr) | (yr < TAU * yl))
    return nx + ny


def transpose_state(q):
    """The same state with x and y exchanged (momenta swapped)."""
    t = np.transpose(q, (0, 2, 1)).copy()
    t[[1, 2]] = t[[2, 1]]
    return t


def near_dry_dambreak(mx, my, seed):
    """h = 1 on the left 40%, 1e-5 (a near-dry bed) elsewhere, both with
    relative noise of 1e-3; velocities 0.5 on the wet side, 0 on the bed."""
    rng = np.random.default_rng(seed)
    x = (np.arange(mx) + 0.5) / mx
    h = np.where(x[None, :] < 0.4, 1.0, 1e-5) * np.ones((my, 1))
    h *= 1 + 1e-3 * rng.uniform(-1, 1, size=h.shape)
    hu = np.where(x[None, :] < 0.4, 0.5, 0.0) * h
    hv = 0.1 * rng.uniform(-1, 1, size=h.shape) * np.where(x[None, :] < 0.4, h, 0.0)
    return np.stack([h, hu, hv])


@pytest.mark.parametrize("direction", ["x", "y"])
def test_near_dry_dambreak(direction):
    mx, my = 70, 45
    q = near_dry_dambreak(mx, my, seed=7)
    if direction == "y":
        q = transpose_state(near_dry_dambreak(my, mx, seed=7))
    errs = {}
    for tau in (0.0, -1.0):
        got, want, nguard, filled = step("swe", q, (W, W, W, W), tau)
        errs[tau] = scaled_error("swe", got, want)
        if tau == 0.0:
            npred = predicted_guard_edges(filled, mx, my)
            assert npred > 0 and nguard == npred, (nguard, npred)
        else:
            assert nguard == 0
    print(f"near-dry {direction}: guarded {errs[0.0]:.3e}, unguarded {errs[-1.0]:.3e}")
    assert errs[0.0] <= TOL[mc.F32], errs


def transonic_state(mx, my, seed):
    """Left half subsonic (u - c < 0), right half supersonic (u - c > 0),
    flow along x: the 1-wave is a transonic rarefaction."""
    rng = np.random.default_rng(seed)
    x = (np.arange(mx) + 0.5) / mx
    left = (x[None, :] < 0.5) * np.ones((my, 1)) > 0
    h = np.where(left, 1.0, 0.6) * (1 + 1e-4 * rng.uniform(-1, 1, size=(my, mx)))
    u = np.where(left, 2.5, 5.0)
    return np.stack([h, h * u, 0.05 * h])


@pytest.mark.parametrize("direction", ["x", "y"])
def test_transonic_rarefaction(direction):
    mx, my = 64, 33
    q = transonic_state(mx, my, 3) if direction == "x" else transpose_state(transonic_state(my, mx, 3))
    c = np.sqrt(G * q[0])
    un = (q[1] if direction == "x" else q[2]) / q[0]
    assert (un - c).min() < 0 < (un - c).max()
    for tau in (0.0, -1.0):
        got, want, nguard, _ = step("swe", q, (X, X, X, X), tau)
        err = scaled_error("swe", got, want)
        assert nguard == 0
        assert err <= TOL[mc.F32], (tau, err)


def euler_cons(rho, u, v, p):
    return np.stack([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])


def near_vacuum_state(mx, my, seed):
    """A gas (rho = p = 1) on the left half next to a near-vacuum region
    (rho = p = 1e-5, the same temperature), noise 1e-3, small velocities."""
    rng = np.random.default_rng(seed)
    x = (np.arange(mx) + 0.5) / mx
    dense = (x[None, :] < 0.5) * np.ones((my, 1)) > 0
    rho = np.where(dense, 1.0, 1e-5) * (1 + 1e-3 * rng.uniform(-1, 1, size=(my, mx)))
    p = np.where(dense, 1.0, 1e-5) * (1 + 1e-3 * rng.uniform(-1, 1, size=(my, mx)))
    u = 0.2 * rng.uniform(-1, 1, size=(my, mx))
    v = 0.2 * rng.uniform(-1, 1, size=(my, mx))
    return euler_cons(rho, u, v, p)


@pytest.mark.parametrize("direction", ["x", "y"])
def test_near_vacuum_euler(direction):
    mx, my = 70, 45
    q = near_vacuum_state(mx, my, 11) if direction == "x" else transpose_state(near_vacuum_state(my, mx, 11))
    for tau in (0.0, -1.0):
        got, want, nguard, filled = step("euler", q, (X, X, X, X), tau)
        err = scaled_error("euler", got, want)
        if tau == 0.0:
            npred = predicted_guard_edges(filled, mx, my)
            assert npred > 0 and nguard == npred, (nguard, npred)
        print(f"near-vacuum {direction} tau {tau}: error {err:.3e}")
        assert err <= TOL[mc.F32], (tau, err)


def test_cold_high_mach_euler():
    """Cold flow (p = 1e-4 rho, Mach numbers up to about 80): c^2 is a small
    difference of the enthalpy and the kinetic energy, yet FP32 meets the
    tolerance without FP64 (the waves' errors cancel in the fluctuations,
    all speeds being about u).  The momentum scale of the tolerance is
    rho_max max(|u| + c), the size of the momenta (with rho_max c_max alone
    the FP32 rounding of the stored momenta would exceed it)."""
    mx, my = 64, 40
    rng = np.random.default_rng(5)
    xx, yy = np.meshgrid((np.arange(mx) + 0.5) / mx, (np.arange(my) + 0.5) / my)
    rho = 1 + 0.5 * np.sin(2 * np.pi * xx) * np.cos(2 * np.pi * yy)
    u = np.cos(2 * np.pi * yy) + 0.01 * rng.uniform(-1, 1, size=xx.shape)
    v = 0.5 * np.sin(2 * np.pi * xx)
    p = 1e-4 * rho
    q = euler_cons(rho, u, v, p)
    for tau in (0.0, -1.0):
        got, want, nguard, _ = step("euler", q, (X, X, X, X), tau)
        cmax = np.sqrt(GAMMA * 1e-4)
        mom = np.abs(want[0]).max() * (np.sqrt(u * u + v * v).max() + cmax)
        S = np.array([np.abs(want[0]).max(), mom, mom, np.abs(want[3]).max()])
        err = max(np.abs(got[m] - want[m]).max() / S[m] for m in range(4))
        assert nguard == 0
        print(f"cold Euler tau {tau}: error {err:.3e}")
        assert err <= TOL[mc.F32], (tau, err)


def test_guard_quiet_on_the_bench_dambreak():
    """The 4096^2 bench problem's cousin at 256^2 (h >= 0.999, subsonic) has
    no guarded edge, so it pays only for the predicate."""
    from paper_1308_1464_gb300 import workloads
    g = workloads.swe_dambreak(256, 256)
    got, want, nguard, _ = step("swe", g.q, (W, W, W, W), 0.0, dx=g.dx)
    assert nguard == 0
    assert scaled_error("swe", got, want) <= TOL[mc.F32]


def test_advance_with_queued_tasks():
    """mc_advance of an FP32 run whose steps queue tasks for the FP64 guard:
    the guard kernel then recomputes them and, in the graph-captured loop,
    applies the time-step rule once the speed maximum is complete (its last
    block).  An initial dt three times too large is rejected and retaken;
    times, step sizes, the rejection count and the state follow the oracle's
    driver as for an unguarded run."""
    mx, my, nsteps = 70, 45, 6
    q32 = near_dry_dambreak(mx, my, seed=7).astype(np.float32)
    dx = 1.0 / 64
    p = mc.Problem.make(mc.SWE_ROE, mx, my, dx, dx, dtype=mc.F32, bc=(W, W, W, W),
                        param=(G, 0, 0, 0))
    op = oracle.Problem(oracle.SWE, mx, my, dx, dx, bc=(W, W, W, W), param=(G, 0, 0, 0))
    qo = embed(op, q32.astype(np.float64))
    dt0 = 3.0 * 0.9 / oracle.max_cell_speed(op, oracle.bc_fill(op, qo))
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(q32)
        ctx.guard_stats(reset=True)
        t, dt, inb, nrej = ctx.advance(a.ptr, b.ptr, nsteps, 0.9, 1.0, 0.0, dt0)
        got = (b if inb else a).download().astype(np.float64)
        nguard = ctx.guard_stats(reset=True)
    want, t_ref, dt_ref, nrej_ref, _ = oracle.advance(op, qo, nsteps, 0.9, 1.0, 0.0, dt0)
    assert nguard > 0
    assert nrej == nrej_ref >= 1
    assert t == pytest.approx(t_ref, rel=1e-5) and dt == pytest.approx(dt_ref, rel=1e-5)
    assert scaled_error("swe", got, want[:, 2:-2, 2:-2]) <= 1e-4
