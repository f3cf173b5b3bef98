"""Helpers shared by the GPU tests: problem construction for both sides, the
field scales of the parity tolerance, and windowed oracle evaluation."""
import numpy as np

import oracle
import paper_1308_1464_gb300 as mc
from paper_1308_1464_gb300 import workloads

G = 9.81
GAMMA = 1.4
SOLVER_IDS = {"acoustics": (mc.ACOUSTICS, oracle.ACOUSTICS, (1.0, 4.0, 0, 0)),
              "swe": (mc.SWE_ROE, oracle.SWE, (G, 0, 0, 0)),
              "euler": (mc.EULER_ROE, oracle.EULER, (GAMMA, 0, 0, 0)),
              "advection": (mc.ADVECTION, oracle.ADVECTION, (1.0, -0.6, 0, 0)),
              "acoustics_var": (mc.ACOUSTICS_VAR, oracle.ACOUSTICS_VAR, (0, 0, 0, 0)),
              "euler_godunov": (mc.EULER_GODUNOV, oracle.EULER_GODUNOV, (GAMMA, 0, 0, 0))}
TOL = {mc.F64: 1e-12, mc.F32: 2e-5}


def problems(solver, mx, my, dx, dy, dtype, bc, limiter=4, order=2, transverse=1, efix=1):
    sid, oid, param = SOLVER_IDS[solver]
    p = mc.Problem.make(sid, mx, my, dx, dy, dtype=dtype, limiter=limiter, order=order,
                        transverse=transverse, efix=efix, bc=bc, param=param)
    op = oracle.Problem(oid, mx, my, dx, dy, limiter=limiter, order=order, transverse=transverse,
                        efix=efix, bc=tuple(bc), param=param)
    return p, op


def field_scales(solver, q):
    """Per-field scales S_m of the parity norm max|gpu - oracle| / S_m."""
    if solver in ("acoustics", "advection", "acoustics_var"):
        return np.ones(q.shape[0])
    if solver == "swe":
        h = np.abs(q[0]).max()
        mom = h * np.sqrt(G * h)
        return np.array([h, mom, mom])
    rho = np.abs(q[0]).max()
    u = q[1] / q[0]
    v = q[2] / q[0]
    p = (GAMMA - 1) * (q[3] - 0.5 * q[0] * (u * u + v * v))
    c = np.sqrt(GAMMA * np.abs(p) / q[0]).max()
    return np.array([rho, rho * c, rho * c, np.abs(q[3]).max()])


def scaled_error(solver, got, want):
    S = field_scales(solver, want)
    return max(np.abs(got[m] - want[m]).max() / S[m] for m in range(want.shape[0]))


def embed(op, interior):
    q = np.zeros(op.shape)
    q[:, 2:-2, 2:-2] = interior
    return q


def initial_state(solver, mx, my, seed=0):
    """Seeded test data with every term of the step active."""
    rng = np.random.default_rng(seed)
    if solver == "acoustics_var":
        # a pulse over a layered medium: density jump at mid-height, sound
        # speed growing along x, small noise in the material too
        g = workloads.acoustics_pulse(mx, my)
        x = (np.arange(mx) + 0.5) / mx
        y = (np.arange(my) + 0.5) / my
        X, Y = np.meshgrid(x, y)
        rho = np.where(Y < 0.5, 1.0, 3.0) * (1 + 0.05 * rng.uniform(-1, 1, size=X.shape))
        c = (1.0 + X) * (1 + 0.05 * rng.uniform(-1, 1, size=X.shape))
        p0 = g.q[0]
        return np.stack([p0, 0.3 * np.roll(p0, 3, axis=1), -0.2 * np.roll(p0, 2, axis=0), rho, c]), g.dx, g.dy
    if solver == "advection":
        g = workloads.acoustics_pulse(mx, my)
        q = g.q[:1].copy() + 0.3 * np.sin(2 * np.pi * np.arange(mx) / mx)[None, None, :]
        q += 0.01 * rng.uniform(-1, 1, size=q.shape)
        return q, g.dx, g.dy
    if solver == "acoustics":
        g = workloads.acoustics_pulse(mx, my)
        q = g.q.copy()
        q[1] = 0.3 * np.roll(q[0], 3, axis=1)
        q[2] = -0.2 * np.roll(q[0], 2, axis=0)
        q += 0.01 * rng.uniform(-1, 1, size=q.shape)
        return q, g.dx, g.dy
    if solver == "swe":
        g = workloads.swe_dambreak(mx, my, seed=seed + 1)
        q = g.q.copy()
        q[1] = 0.2 * q[0] * rng.uniform(-1, 1, size=q[0].shape)
        q[2] = 0.2 * q[0] * rng.uniform(-1, 1, size=q[0].shape)
        return q, g.dx, g.dy
    g = workloads.euler_quadrants(mx, my, seed=seed + 1)
    return g.q.copy(), g.dx, g.dy


def window_step(op_full, q_full_ghosted, dt, i0, j0, w, h):
    """Oracle step of the window of cells [i0, i0+w) x [j0, j0+h) using the
    given (already filled) neighbours as ghosts.  Returns the window interior."""
    win = oracle.Problem(op_full.solver, w, h, op_full.dx, op_full.dy, limiter=op_full.limiter,
                         order=op_full.order, transverse=op_full.transverse, efix=op_full.efix,
                         bc=(oracle.BC_GIVEN,) * 4, param=op_full.param)
    qw = np.ascontiguousarray(q_full_ghosted[:, j0: j0 + h + 4, i0: i0 + w + 4], dtype=np.float64)
    out, _, _ = oracle.step(win, qw, dt)
    return out[:, 2:-2, 2:-2]
