"""Pins of the oracle's coupling of refined patches to a coarse grid (CPU).

The paper's "dynamic time stepping" kernel (§1.2, Table 1): refined grids
take their own time steps and get boundary values from the adjacent grid by
spatial and temporal interpolation.  Pinned independently of amr.c:

* the coarse reconstruction reproduces linear data exactly, and the fine
  cells of one coarse cell average to the coarse value (conservation);
* the time interpolation is linear between the coarse states;
* ghost cells covered by another patch are that patch's values;
* ratio 1 with one patch over the whole grid is exactly the single-grid step;
* a uniform state stays uniform;
* refining the region an advected pulse crosses brings the result closer to
  a uniformly fine run than the coarse grid alone;
* the pointwise edge flux reproduces the step (minus its differences is each
  cell's update), and refluxing with it conserves the coarse sum on a
  periodic grid to rounding.
"""
import numpy as np
import pytest

BCP, BCX = 0, 1


def problem(oracle, mx, my, solver="advection", bc=(BCX,) * 4, limiter=4, transverse=1):
    sid = {"advection": oracle.ADVECTION, "swe": oracle.SWE, "euler": oracle.EULER}[solver]
    param = {"advection": (1.0, 0.6, 0, 0), "swe": (9.81, 0, 0, 0), "euler": (1.4, 0, 0, 0)}[solver]
    return oracle.Problem(sid, mx, my, 1.0 / mx, 1.0 / my, limiter=limiter, transverse=transverse,
                          bc=bc, param=param)


def centres(n, lo=0.0, hi=1.0):
    h = (hi - lo) / n
    return lo + (np.arange(-2, n + 2) + 0.5) * h


def test_reconstruction_linear_exact_and_conservative(oracle_mod):
    mx, my, r = 12, 10, 2
    pc = problem(oracle_mod, mx, my)
    xc, yc = centres(mx), centres(my)
    X, Y = np.meshgrid(xc, yc)
    lin = (0.3 + 1.7 * X - 0.8 * Y)[None]                  # linear data, ghosts included
    patches = [(3, 2, 5, 4)]
    pf = oracle_mod.fine_problem(pc, r, patches[0])
    qf = [np.zeros(pf.shape)]
    oracle_mod.amr_fill_ghosts(pc, r, lin, lin, 0.0, patches, qf)
    ci0, cj0, cw, ch = patches[0]
    xf = (ci0 + (np.arange(-2, r * cw + 2) + 0.5) / r) / mx
    yf = (cj0 + (np.arange(-2, r * ch + 2) + 0.5) / r) / my
    XF, YF = np.meshgrid(xf, yf)
    want = 0.3 + 1.7 * XF - 0.8 * YF
    ring = np.ones(want.shape, bool)
    ring[2:-2, 2:-2] = False
    np.testing.assert_allclose(qf[0][0][ring], want[ring], atol=1e-13)
    # random data: each coarse cell of the ghost ring is the mean of its 2 x 2 fine ghosts
    rng = np.random.default_rng(1)
    qc = rng.uniform(-1, 1, (1, my + 4, mx + 4))
    qf = [np.zeros(pf.shape)]
    oracle_mod.amr_fill_ghosts(pc, r, qc, qc, 0.0, patches, qf)
    g = qf[0][0]
    for cj in range(cj0 - 1, cj0 + ch + 1):
        for ci in range(ci0 - 1, ci0 + cw + 1):
            if ci0 <= ci < ci0 + cw and cj0 <= cj < cj0 + ch:
                continue
            fi, fj = r * (ci - ci0) + 2, r * (cj - cj0) + 2
            assert g[fj: fj + r, fi: fi + r].mean() == pytest.approx(qc[0, cj + 2, ci + 2], abs=1e-14)


def test_time_interpolation_is_linear(oracle_mod):
    mx, my, r = 10, 10, 4
    pc = problem(oracle_mod, mx, my)
    rng = np.random.default_rng(2)
    q0 = rng.uniform(0, 1, (1, my + 4, mx + 4))
    q1 = q0 + 0.25                                          # a uniform shift in time
    patches = [(2, 3, 4, 3)]
    pf = oracle_mod.fine_problem(pc, r, patches[0])
    base = [np.zeros(pf.shape)]
    oracle_mod.amr_fill_ghosts(pc, r, q0, q0, 0.0, patches, base)
    for alpha in (0.0, 0.25, 0.5, 0.75):
        qf = [np.zeros(pf.shape)]
        oracle_mod.amr_fill_ghosts(pc, r, q0, q1, alpha, patches, qf)
        ring = np.ones(pf.shape[1:], bool)
        ring[2:-2, 2:-2] = False
        np.testing.assert_allclose(qf[0][0][ring], base[0][0][ring] + 0.25 * alpha, atol=1e-14)


def test_ghosts_from_a_neighbouring_patch(oracle_mod):
    mx, my, r = 12, 8, 2
    pc = problem(oracle_mod, mx, my)
    patches = [(2, 2, 4, 4), (6, 2, 3, 4)]                 # side by side at coarse column 6
    pfs = [oracle_mod.fine_problem(pc, r, pt) for pt in patches]
    rng = np.random.default_rng(3)
    qf = [rng.uniform(0, 1, pf.shape) for pf in pfs]
    qc = rng.uniform(0, 1, (1, my + 4, mx + 4))
    oracle_mod.amr_fill_ghosts(pc, r, qc, qc, 0.0, patches, qf)
    # patch 0's right ghost columns are patch 1's first interior columns (same rows)
    np.testing.assert_array_equal(qf[0][0, 2:-2, -2:], qf[1][0, 2:-2, 2:4])
    np.testing.assert_array_equal(qf[1][0, 2:-2, 0:2], qf[0][0, 2:-2, -4:-2])


@pytest.mark.parametrize("solver", ["advection", "swe", "euler"])
def test_ratio_one_whole_grid_is_the_single_grid_step(oracle_mod, solver):
    mx, my = 9, 7
    pc = problem(oracle_mod, mx, my, solver=solver, bc=(BCX, BCX, 2, BCX))
    rng = np.random.default_rng(4)
    if solver == "advection":
        inner = rng.uniform(0, 1, (1, my, mx))
    elif solver == "swe":
        inner = np.stack([1 + 0.2 * rng.uniform(0, 1, (my, mx)), 0.1 * rng.uniform(-1, 1, (my, mx)),
                          0.1 * rng.uniform(-1, 1, (my, mx))])
    else:
        rho = 1 + 0.2 * rng.uniform(0, 1, (my, mx))
        inner = np.stack([rho, 0.1 * rho, -0.1 * rho, 2.5 + 0.2 * rng.uniform(0, 1, (my, mx))])
    qc = np.zeros(pc.shape)
    qc[:, 2:-2, 2:-2] = inner
    dt = 0.5 / oracle_mod.max_cell_speed(pc, oracle_mod.bc_fill(pc, qc))
    single, _, _ = oracle_mod.step(pc, qc, dt)
    patches = [(0, 0, mx, my)]
    qf = [qc.copy()]
    amr, flags = oracle_mod.amr_step(pc, 1, patches, qc, qf, dt)
    assert flags == 0
    np.testing.assert_allclose(amr, single, atol=1e-14)


def test_uniform_state_stays_uniform(oracle_mod):
    mx, my, r = 10, 8, 2
    pc = problem(oracle_mod, mx, my, solver="swe", bc=(2, 2, 2, 2))
    patches = [(2, 2, 3, 3), (5, 2, 3, 4)]
    qc = np.zeros(pc.shape)
    qc[0], qc[1], qc[2] = 1.3, 0.0, 0.0
    qf = []
    for pt in patches:
        a = np.zeros(oracle_mod.fine_problem(pc, r, pt).shape)
        a[0] = 1.3
        qf.append(a)
    out, _ = oracle_mod.amr_step(pc, r, patches, qc, qf, 0.02)
    np.testing.assert_allclose(out[:, 2:-2, 2:-2], qc[:, 2:-2, 2:-2], atol=1e-14)
    for a in qf:
        np.testing.assert_allclose(a[:, 2:-2, 2:-2], np.stack([np.full(a.shape[1:], 1.3), 0 * a[0], 0 * a[0]])[:, 2:-2, 2:-2], atol=1e-14)


def test_refinement_improves_an_advected_pulse(oracle_mod):
    """A Gaussian advected by (1, 0.6) on a periodic coarse grid; a patch of
    ratio 4 covers the region it crosses.  Compared on that region with a
    uniformly fine run, the coupled solution is much closer than the coarse
    grid alone (interpolated to the fine cells)."""
    n, r = 24, 4
    pc = problem(oracle_mod, n, n, bc=(BCP,) * 4)
    pfull = problem(oracle_mod, r * n, r * n, bc=(BCP,) * 4)
    gauss = lambda X, Y: np.exp(-((X - 0.35) ** 2 + (Y - 0.4) ** 2) / 0.006)
    xc = (np.arange(n) + 0.5) / n
    Xc, Yc = np.meshgrid(xc, xc)
    xf = (np.arange(r * n) + 0.5) / (r * n)
    Xf, Yf = np.meshgrid(xf, xf)
    qc = np.zeros(pc.shape)
    qfull = np.zeros(pfull.shape)
    qfull[0, 2:-2, 2:-2] = gauss(Xf, Yf)
    qc[0, 2:-2, 2:-2] = qfull[0, 2:-2, 2:-2].reshape(n, r, n, r).mean(axis=(1, 3))
    patch = (5, 5, 14, 12)                               # coarse cells 5..18 x 5..16
    ci0, cj0, cw, ch = patch
    qf = np.zeros(oracle_mod.fine_problem(pc, r, patch).shape)
    qf[0, 2:-2, 2:-2] = qfull[0, 2 + r * cj0: 2 + r * (cj0 + ch), 2 + r * ci0: 2 + r * (ci0 + cw)]
    dt = 0.5 / n                                         # Courant 0.5 in x on both levels
    qco = qc.copy()
    qcoarse = qc.copy()
    qfs = [qf]
    for _ in range(8):
        qco, _ = oracle_mod.amr_step(pc, r, [patch], qco, qfs, dt)
        qcoarse, _, _ = oracle_mod.step(pc, qcoarse, dt)
        for _ in range(r):
            qfull, _, _ = oracle_mod.step(pfull, qfull, dt / r)
    ref = qfull[0, 2 + r * cj0: 2 + r * (cj0 + ch), 2 + r * ci0: 2 + r * (ci0 + cw)]
    err_amr = np.abs(qfs[0][0, 2:-2, 2:-2] - ref).max()
    coarse_on_fine = np.repeat(np.repeat(qcoarse[0, 2 + cj0: 2 + cj0 + ch, 2 + ci0: 2 + ci0 + cw], r, 0), r, 1)
    err_coarse = np.abs(coarse_on_fine - ref).max()
    assert err_amr < 0.25 * err_coarse, (err_amr, err_coarse)
    # the covered coarse cells are the averages of the patch
    np.testing.assert_allclose(qco[0, 2 + cj0: 2 + cj0 + ch, 2 + ci0: 2 + ci0 + cw],
                               qfs[0][0, 2:-2, 2:-2].reshape(ch, r, cw, r).mean(axis=(1, 3)), atol=1e-14)


# ---- the edge flux and refluxing --------------------------------------------

def _random_state(oracle_mod, solver, mx, my, seed):
    rng = np.random.default_rng(seed)
    if solver == "advection":
        return rng.uniform(0, 1, (1, my, mx))
    if solver == "acoustics":
        return rng.uniform(-1, 1, (3, my, mx))
    if solver == "swe":
        return np.stack([1 + 0.5 * rng.uniform(0, 1, (my, mx)), 0.3 * rng.uniform(-1, 1, (my, mx)),
                         0.3 * rng.uniform(-1, 1, (my, mx))])
    rho = 1 + 0.5 * rng.uniform(0, 1, (my, mx))
    return np.stack([rho, 0.4 * rho * rng.uniform(-1, 1, (my, mx)), 0.4 * rho * rng.uniform(-1, 1, (my, mx)),
                     2.5 + rng.uniform(0, 1, (my, mx))])


def _prob(oracle_mod, solver, mx, my, bc, limiter=4, order=2, transverse=1):
    sid = {"advection": oracle_mod.ADVECTION, "acoustics": oracle_mod.ACOUSTICS, "swe": oracle_mod.SWE,
           "euler": oracle_mod.EULER}[solver]
    param = {"advection": (1.0, -0.6, 0, 0), "acoustics": (1.0, 4.0, 0, 0), "swe": (9.81, 0, 0, 0),
             "euler": (1.4, 0, 0, 0)}[solver]
    return oracle_mod.Problem(sid, mx, my, 1.0 / mx, 1.0 / my, limiter=limiter, order=order,
                              transverse=transverse, bc=bc, param=param)


@pytest.mark.parametrize("solver,limiter,order,transverse", [
    ("advection", 4, 2, 1), ("acoustics", 1, 2, 2), ("swe", 4, 2, 1), ("swe", 3, 2, 2),
    ("euler", 4, 2, 1), ("euler", 2, 1, 0), ("euler", 4, 2, 2)])
def test_edge_fluxes_reproduce_the_step(oracle_mod, solver, limiter, order, transverse):
    """Minus the difference of the edge fluxes, computed edge by edge from
    the stencil, is the step's update of every cell (step.c builds it from
    whole-grid work arrays instead)."""
    mx, my = 9, 7
    p = _prob(oracle_mod, solver, mx, my, (BCX, 2, BCP, BCP), limiter, order, transverse)
    q = np.zeros(p.shape)
    q[:, 2:-2, 2:-2] = _random_state(oracle_mod, solver, mx, my, 11)
    q = oracle_mod.bc_fill(p, q)
    dt = 0.6 / oracle_mod.max_cell_speed(p, q)
    want, _, flags = oracle_mod.step(p, q, dt)
    assert flags == 0
    Fx = np.array([[oracle_mod.edge_flux(p, q, dt, 0, i, j) for i in range(mx + 1)] for j in range(my)])
    Fy = np.array([[oracle_mod.edge_flux(p, q, dt, 1, i, j) for i in range(mx)] for j in range(my + 1)])
    got = q[:p.meqn, 2:-2, 2:-2] - dt / p.dx * np.moveaxis(Fx[:, 1:] - Fx[:, :-1], 2, 0) \
        - dt / p.dy * np.moveaxis(Fy[1:] - Fy[:-1], 2, 0)
    scale = np.abs(q[:p.meqn]).max()
    np.testing.assert_allclose(got, want[:p.meqn, 2:-2, 2:-2], atol=1e-12 * scale)


@pytest.mark.parametrize("solver", ["advection", "swe", "euler"])
def test_refluxing_conserves(oracle_mod, solver):
    """On a periodic coarse grid the sum over all coarse cells is conserved
    to rounding with the flux correction, and not without it."""
    mx, my, r = 16, 14, 2
    p = _prob(oracle_mod, solver, mx, my, (BCP,) * 4)
    q0 = np.zeros(p.shape)
    q0[:, 2:-2, 2:-2] = _random_state(oracle_mod, solver, mx, my, 5)
    patches = [(3, 2, 4, 5), (9, 6, 4, 4), (2, 9, 5, 3)]
    dt = 0.4 / oracle_mod.max_cell_speed(p, oracle_mod.bc_fill(p, q0))
    drift = {}
    for reflux in (False, True):
        qc = q0.copy()
        qf = []
        for (ci0, cj0, cw, ch) in patches:
            a = np.zeros(oracle_mod.fine_problem(p, r, (ci0, cj0, cw, ch)).shape)
            a[:, 2:-2, 2:-2] = np.repeat(np.repeat(q0[:, 2 + cj0: 2 + cj0 + ch, 2 + ci0: 2 + ci0 + cw], r, 1), r, 2)
            qf.append(a)
        s0 = q0[:, 2:-2, 2:-2].sum(axis=(1, 2))
        for _ in range(3):
            qc, flags = oracle_mod.amr_step(p, r, patches, qc, qf, dt, reflux=reflux)
            assert flags == 0
        drift[reflux] = np.abs(qc[:, 2:-2, 2:-2].sum(axis=(1, 2)) - s0).max() / np.abs(s0).max()
    assert drift[True] < 1e-13, drift
    assert drift[False] > 1e3 * max(drift[True], 1e-16), drift


def test_refluxing_keeps_uniform_state_and_single_grid(oracle_mod):
    """A uniform state stays uniform; ratio 1 with one patch over the whole
    grid has no corrected edge and is the single-grid step."""
    mx, my = 10, 8
    p = _prob(oracle_mod, "swe", mx, my, (2, 2, 2, 2))
    qc = np.zeros(p.shape)
    qc[0] = 1.3
    qf = [np.zeros(oracle_mod.fine_problem(p, 2, pt).shape) for pt in [(2, 2, 3, 3), (6, 2, 3, 4)]]
    for a in qf:
        a[0] = 1.3
    out, _ = oracle_mod.amr_step(p, 2, [(2, 2, 3, 3), (6, 2, 3, 4)], qc, qf, 0.02, reflux=True)
    np.testing.assert_allclose(out[:, 2:-2, 2:-2], qc[:, 2:-2, 2:-2], atol=1e-14)
    q = np.zeros(p.shape)
    q[:, 2:-2, 2:-2] = _random_state(oracle_mod, "swe", mx, my, 2)
    dt = 0.5 / oracle_mod.max_cell_speed(p, oracle_mod.bc_fill(p, q))
    single, _, _ = oracle_mod.step(p, q, dt)
    amr, _ = oracle_mod.amr_step(p, 1, [(0, 0, mx, my)], q, [q.copy()], dt, reflux=True)
    np.testing.assert_allclose(amr, single, atol=1e-14)
