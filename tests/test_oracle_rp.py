"""Pins of the oracle's pointwise Riemann solvers and limiter (CPU only).

The paper (§1.1, §1.2/Table 1, §2) defines the Riemann kernel as the map
from two adjacent cell states to edge waves and fluctuations but gives no
formulas.  These tests pin the oracle against facts fixed by the mathematics,
computed here independently of the oracle's code:

* waves are the eigen-decomposition of the jump qr - ql in the eigenvectors of
  the Roe matrix, obtained here from numpy eigenvalues and Sylvester's
  spectral projectors of the flux Jacobian,
  itself taken by complex-step differentiation of the physical flux at the
  Roe-averaged state (LeVeque 2002, §15.3);
* the Roe matrix reproduces the flux difference exactly (Roe property), so
  the fluctuations sum to f(qr) - f(ql), with or without the entropy fix;
* transverse splits B-(x), B+(x) are the negative/positive-speed parts of the
  transverse Jacobian applied to x;
* limiter values match the closed forms tabulated in tests/golden.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

GAMMA = 1.4
G = 9.81


def flux_swe(q, d):
    h, m, n = q
    un = (m if d == 0 else n) / h
    f = np.array([h * un, m * un, n * un], dtype=q.dtype)
    f[1 + d] += 0.5 * G * h * h
    return f


def flux_euler(q, d):
    rho, m, n, E = q
    p = (GAMMA - 1.0) * (E - 0.5 * (m * m + n * n) / rho)
    un = (m if d == 0 else n) / rho
    f = np.array([rho * un, m * un, n * un, (E + p) * un], dtype=q.dtype)
    f[1 + d] += p
    return f


def flux_acoustics(q, d, rho=1.0, K=4.0):
    p, u, v = q
    if d == 0:
        return np.array([K * u, p / rho, 0.0 * p], dtype=q.dtype)
    return np.array([K * v, 0.0 * p, p / rho], dtype=q.dtype)


def jacobian(flux, q, d):
    """Complex-step derivative of the flux: exact to round-off."""
    n = len(q)
    J = np.zeros((n, n))
    hstep = 1e-30
    for k in range(n):
        qc = q.astype(complex)
        qc[k] += 1j * hstep
        J[:, k] = np.imag(flux(qc, d)) / hstep
    return J


def roe_state_swe(ql, qr):
    sl, sr = np.sqrt(ql[0]), np.sqrt(qr[0])
    u = (ql[1] / sl + qr[1] / sr) / (sl + sr)
    v = (ql[2] / sl + qr[2] / sr) / (sl + sr)
    h = 0.5 * (ql[0] + qr[0])
    return np.array([h, h * u, h * v])


def roe_state_euler(ql, qr):
    def prim(q):
        rho, m, n, E = q
        p = (GAMMA - 1.0) * (E - 0.5 * (m * m + n * n) / rho)
        return rho, m / rho, n / rho, (E + p) / rho
    rl, ul, vl, Hl = prim(ql)
    rr, ur, vr, Hr = prim(qr)
    sl, sr = np.sqrt(rl), np.sqrt(rr)
    u = (sl * ul + sr * ur) / (sl + sr)
    v = (sl * vl + sr * vr) / (sl + sr)
    H = (sl * Hl + sr * Hr) / (sl + sr)
    rho = sl * sr
    # conserved state with velocity (u, v) and enthalpy H: E + p = rho H
    E = (rho * H + (GAMMA - 1.0) * 0.5 * rho * (u * u + v * v)) / GAMMA
    return np.array([rho, rho * u, rho * v, E])


def random_states(solver, rng, n):
    out = []
    for _ in range(n):
        if solver == "acoustics":
            out.append((rng.normal(size=3), rng.normal(size=3)))
        elif solver == "swe":
            def st():
                h = rng.uniform(0.1, 3.0)
                return np.array([h, h * rng.uniform(-2, 2), h * rng.uniform(-2, 2)])
            out.append((st(), st()))
        else:
            def st():
                rho, p = rng.uniform(0.1, 3.0), rng.uniform(0.1, 3.0)
                u, v = rng.uniform(-2, 2), rng.uniform(-2, 2)
                return np.array([rho, rho * u, rho * v, p / (GAMMA - 1) + 0.5 * rho * (u * u + v * v)])
            out.append((st(), st()))
    return out


def make_problem(oracle, solver, efix=1):
    sid = {"acoustics": oracle.ACOUSTICS, "swe": oracle.SWE, "euler": oracle.EULER}[solver]
    param = {"acoustics": (1.0, 4.0, 0, 0), "swe": (G, 0, 0, 0), "euler": (GAMMA, 0, 0, 0)}[solver]
    return oracle.Problem(sid, 4, 4, 0.1, 0.1, efix=efix, param=param)


def roe_matrix(solver, ql, qr, d):
    if solver == "acoustics":
        return jacobian(flux_acoustics, ql, d)
    if solver == "swe":
        return jacobian(flux_swe, roe_state_swe(ql, qr), d)
    return jacobian(flux_euler, roe_state_euler(ql, qr), d)


def spectral_pieces(A, x):
    """Split x by the spectral projectors of a diagonalisable A (Sylvester's
    formula over its distinct eigenvalues): returns (eigenvalues, pieces)."""
    ev = np.sort(np.linalg.eigvals(A).real)
    distinct = []
    for e in ev:
        if not distinct or abs(e - distinct[-1]) > 1e-8 * (1.0 + abs(e)):
            distinct.append(e)
    n = A.shape[0]
    pieces = []
    for k, lk in enumerate(distinct):
        P = np.eye(n)
        for m, mu in enumerate(distinct):
            if m != k:
                P = P @ (A - mu * np.eye(n)) / (lk - mu)
        pieces.append(P @ x)
    return distinct, pieces


def phys_flux(solver, q, d):
    return {"acoustics": flux_acoustics, "swe": flux_swe, "euler": flux_euler}[solver](q, d)


SOLVERS = ["acoustics", "swe", "euler"]


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("d", [0, 1])
def test_roe_matrix_is_roe(solver, d):
    """The test's own Roe average satisfies A(qr - ql) = f(qr) - f(ql)."""
    rng = np.random.default_rng(11)
    for ql, qr in random_states(solver, rng, 50):
        A = roe_matrix(solver, ql, qr, d)
        df = phys_flux(solver, qr, d) - phys_flux(solver, ql, d)
        np.testing.assert_allclose(A @ (qr - ql), df, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("d", [0, 1])
def test_waves_are_eigen_decomposition(oracle_mod, solver, d):
    """Oracle waves/speeds equal the eigen-decomposition of the jump (numpy eig)."""
    prob = make_problem(oracle_mod, solver, efix=0)
    rng = np.random.default_rng(12 + d)
    for ql, qr in random_states(solver, rng, 200):
        wave, s, amdq, apdq, flags = oracle_mod.rpn2(prob, d, ql, qr)
        assert flags == 0
        A = roe_matrix(solver, ql, qr, d)
        lam, pieces = spectral_pieces(A, qr - ql)
        scale = np.abs(qr - ql).max() + 1e-300
        if solver == "acoustics":
            # speeds -c, 0, +c: the zero-speed piece (tangential velocity) is not carried
            exp_s = [lam[0], lam[2]]
            exp_w = [pieces[0], pieces[2]]
            assert abs(lam[1]) < 1e-12
        elif solver == "swe":
            exp_s, exp_w = list(lam), pieces
        else:
            # entropy and shear share the middle speed: one combined wave,
            # which is the projection on that eigenvalue's 2D eigenspace
            assert len(lam) == 3
            exp_s, exp_w = list(lam), pieces
        np.testing.assert_allclose(s, exp_s, rtol=1e-11, atol=1e-11)
        for w in range(len(exp_s)):
            np.testing.assert_allclose(wave[w], exp_w[w], rtol=1e-9, atol=1e-11 * scale)


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("d", [0, 1])
@pytest.mark.parametrize("efix", [0, 1])
def test_waves_sum_to_jump_and_fluctuations_to_flux_difference(oracle_mod, solver, d, efix):
    prob = make_problem(oracle_mod, solver, efix=efix)
    rng = np.random.default_rng(100 + 2 * d + efix)
    for ql, qr in random_states(solver, rng, 300):
        wave, s, amdq, apdq, flags = oracle_mod.rpn2(prob, d, ql, qr)
        jump = qr - ql
        tot = wave.sum(axis=0)
        if solver == "acoustics":
            # the tangential-velocity jump rides on the dropped zero-speed wave
            jump = jump.copy()
            jump[2 - d] = 0.0
        scale = np.abs(qr - ql).max()
        np.testing.assert_allclose(tot, jump, rtol=0, atol=1e-13 * max(scale, 1.0))
        df = phys_flux(solver, qr, d) - phys_flux(solver, ql, d)
        fscale = max(np.abs(df).max(), np.abs(phys_flux(solver, ql, d)).max(), 1.0)
        np.testing.assert_allclose(amdq + apdq, df, rtol=0, atol=1e-12 * fscale)
        if not efix:
            np.testing.assert_allclose(amdq, sum(min(s[w], 0) * wave[w] for w in range(len(s))),
                                       atol=1e-13 * fscale)


def test_acoustics_closed_form_eigenvectors(oracle_mod):
    """rho = 1, K = 4: c = 2, Z = 2; waves are multiples of (-Z, 1, 0), (Z, 1, 0)."""
    prob = make_problem(oracle_mod, "acoustics")
    ql, qr = np.array([0.3, -0.2, 0.7]), np.array([1.1, 0.4, -0.5])
    wave, s, amdq, apdq, _ = oracle_mod.rpn2(prob, 0, ql, qr)
    np.testing.assert_allclose(s, [-2.0, 2.0])
    dp, du = 0.8, 0.6
    a1 = (-dp + 2 * du) / 4.0
    a2 = (dp + 2 * du) / 4.0
    np.testing.assert_allclose(wave[0], [-2 * a1, a1, 0.0], atol=1e-15)
    np.testing.assert_allclose(wave[1], [2 * a2, a2, 0.0], atol=1e-15)
    np.testing.assert_allclose(amdq, -2.0 * wave[0], atol=1e-15)
    np.testing.assert_allclose(apdq, 2.0 * wave[1], atol=1e-15)


@pytest.mark.parametrize("solver", SOLVERS)
@pytest.mark.parametrize("d", [0, 1])
def test_transverse_split(oracle_mod, solver, d):
    """B-(x) + B+(x) = B x and each part is the signed-speed part of B (numpy eig)."""
    prob = make_problem(oracle_mod, solver)
    rng = np.random.default_rng(200 + d)
    for ql, qr in random_states(solver, rng, 150):
        x = rng.normal(size=len(ql))
        bm, bp = oracle_mod.rpt2(prob, d, ql, qr, x)
        B = roe_matrix(solver, ql, qr, 1 - d)
        lam, pieces = spectral_pieces(B, x)
        exp_m = sum(min(l, 0.0) * pc for l, pc in zip(lam, pieces))
        exp_p = sum(max(l, 0.0) * pc for l, pc in zip(lam, pieces))
        sc = max(1.0, np.abs(B).max()) * np.abs(x).max()
        np.testing.assert_allclose(bm + bp, B @ x, atol=1e-12 * sc)
        np.testing.assert_allclose(bm, exp_m, atol=1e-10 * sc)
        np.testing.assert_allclose(bp, exp_p, atol=1e-10 * sc)


def test_entropy_fix_transonic_split(oracle_mod):
    """In a transonic 1-rarefaction the left-going fluctuation is the part of the
    wave between the left characteristic speed and zero (Harten-Hyman):
    amdq = beta lam_l W1 with lam_l beta + lam_r (1 - beta) = s1."""
    prob = make_problem(oracle_mod, "swe", efix=1)
    ql = np.array([3.0, 3.0 * 1.5, 0.0])       # u - c < 0
    qr = np.array([0.5, 0.5 * 3.0, 0.0])
    wave, s, amdq, apdq, _ = oracle_mod.rpn2(prob, 0, ql, qr)
    lam_l = ql[1] / ql[0] - np.sqrt(G * ql[0])
    qm = ql + wave[0]
    lam_r = qm[1] / qm[0] - np.sqrt(G * qm[0])
    assert lam_l < 0 < lam_r, "case must be transonic"
    beta = (lam_r - s[0]) / (lam_r - lam_l)
    assert 0 < beta < 1
    expected = beta * lam_l * wave[0] + sum(min(s[w], 0) * wave[w] for w in (1, 2))
    np.testing.assert_allclose(amdq, expected, rtol=1e-13, atol=1e-14)
    # without the fix the 1-wave counts entirely to one side
    prob0 = make_problem(oracle_mod, "swe", efix=0)
    _, _, amdq0, _, _ = oracle_mod.rpn2(prob0, 0, ql, qr)
    assert np.abs(amdq0 - amdq).max() > 1e-3


def _golden_limiter():
    path = os.path.join(os.path.dirname(__file__), "golden", "limiter_phi.txt")
    rows = []
    with open(path) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append([float(Fraction(tok)) for tok in line.split()])
    return rows


def test_limiter_table(oracle_mod):
    for theta, phi_mm, phi_mc, phi_sb, phi_vl in _golden_limiter():
        assert oracle_mod.philim(oracle_mod.LIM_MINMOD, theta) == pytest.approx(phi_mm, abs=1e-15)
        assert oracle_mod.philim(oracle_mod.LIM_MC, theta) == pytest.approx(phi_mc, abs=1e-15)
        assert oracle_mod.philim(oracle_mod.LIM_SUPERBEE, theta) == pytest.approx(phi_sb, abs=1e-15)
        assert oracle_mod.philim(oracle_mod.LIM_VANLEER, theta) == pytest.approx(phi_vl, abs=1e-15)
        assert oracle_mod.philim(oracle_mod.LIM_NONE, theta) == 1.0


def test_limiter_tvd_region(oracle_mod):
    """Sweby's TVD region: 0 <= phi <= min(2, 2 theta) for theta > 0, phi = 0 below, phi(1) = 1;
    minmod and superbee are its lower and upper boundaries, so every limiter lies between them."""
    lims = (oracle_mod.LIM_MINMOD, oracle_mod.LIM_SUPERBEE, oracle_mod.LIM_VANLEER, oracle_mod.LIM_MC)
    for theta in np.linspace(-5, 10, 301):
        lo = oracle_mod.philim(oracle_mod.LIM_MINMOD, theta)
        hi = oracle_mod.philim(oracle_mod.LIM_SUPERBEE, theta)
        assert hi == pytest.approx(max(0.0, min(1.0, 2 * theta), min(2.0, theta)) if theta > 0 else 0.0)
        for lim in lims:
            assert lo - 1e-15 <= oracle_mod.philim(lim, theta) <= hi + 1e-15
    for lim in lims:
        for theta in np.linspace(-5, 10, 301):
            phi = oracle_mod.philim(lim, theta)
            if theta <= 0:
                assert phi == 0.0
            else:
                assert 0.0 <= phi <= min(2.0, 2.0 * theta) + 1e-15
        assert oracle_mod.philim(lim, 1.0) == 1.0
