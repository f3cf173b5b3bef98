"""Pins of the oracle's variable-coefficient acoustics (CPU only).

The paper lists variable-coefficient acoustics among its four Riemann kernels
(§3, Table 2) without formulas; the mathematics is LeVeque (2002) §9.6
(Riemann problem at a material interface) and the transverse splitting for
heterogeneous media.  These tests pin the oracle against facts that do not
come from its code:

* the waves of an interface Riemann problem lie along the eigenvectors of
  their own media and connect through the state fixed by continuity of
  pressure and normal velocity; each fluctuation is the flux jump across its
  wave in its own medium;
* the transverse split is the projection on the neighbouring media's
  eigenvectors, solved here as a linear system with numpy;
* uniform material reproduces constant-coefficient acoustics;
* a pulse crossing an interface transmits and reflects pressure with the
  textbook coefficients 2 Z2 / (Z1 + Z2) and (Z2 - Z1) / (Z1 + Z2).
"""
import numpy as np
import pytest

BCP, BCX = 0, 1


def var_problem(oracle, mx, my, dx, dy, bc=(BCP,) * 4, limiter=4, transverse=1, order=2):
    return oracle.Problem(oracle.ACOUSTICS_VAR, mx, my, dx, dy, limiter=limiter, order=order,
                          transverse=transverse, efix=0, bc=bc, param=(0, 0, 0, 0))


def cell(p, u, v, rho, c):
    return np.array([p, u, v, rho, c], dtype=float)


def test_interface_riemann_problem(oracle_mod):
    rng = np.random.default_rng(3)
    prob = var_problem(oracle_mod, 4, 4, 0.1, 0.1)
    for _ in range(20):
        rl, cl, rr, cr = rng.uniform(0.3, 3.0, 4)
        for d in (0, 1):
            un, ut = 1 + d, 2 - d
            ql = cell(*rng.uniform(-1, 1, 3), rl, cl)
            qr = cell(*rng.uniform(-1, 1, 3), rr, cr)
            W, s, amdq, apdq, flags = oracle_mod.rpn2(prob, d, ql, qr)
            assert flags == 0
            zl, zr = rl * cl, rr * cr
            # middle state: continuity of p and u_n, with p - Z u constant
            # across the left-going wave and p + Z u across the right-going one
            ustar = (ql[0] - qr[0] + zl * ql[un] + zr * qr[un]) / (zl + zr)
            pstar = ql[0] - zl * (ustar - ql[un])
            assert pstar == pytest.approx(qr[0] - zr * (qr[un] - ustar), abs=1e-13)
            w1 = np.zeros(3); w1[0] = pstar - ql[0]; w1[un] = ustar - ql[un]
            w2 = np.zeros(3); w2[0] = qr[0] - pstar; w2[un] = qr[un] - ustar
            np.testing.assert_allclose(W[0], w1, atol=1e-13)
            np.testing.assert_allclose(W[1], w2, atol=1e-13)
            assert s[0] == pytest.approx(-cl) and s[1] == pytest.approx(cr)
            # fluctuation = flux jump across the wave in its own medium
            qs_l = cell(pstar, 0, 0, rl, cl); qs_l[un] = ustar; qs_l[ut] = ql[ut]
            qs_r = cell(pstar, 0, 0, rr, cr); qs_r[un] = ustar; qs_r[ut] = qr[ut]
            f = lambda q: oracle_mod.flux(prob, d, q)
            np.testing.assert_allclose(amdq, f(qs_l) - f(ql), atol=1e-12)
            np.testing.assert_allclose(apdq, f(qr) - f(qs_r), atol=1e-12)


def test_transverse_split_is_a_projection(oracle_mod):
    rng = np.random.default_rng(4)
    prob = var_problem(oracle_mod, 4, 4, 0.1, 0.1)
    for _ in range(20):
        mats = rng.uniform(0.3, 3.0, (3, 2))          # (rho, c) below, centre, above
        qlo, qc, qhi = (cell(0, 0, 0, r, c) for r, c in mats)
        z = mats[:, 0] * mats[:, 1]
        for d in (0, 1):
            vn, vt = 2 - d, 1 + d                     # velocity along / across the split direction
            a = rng.uniform(-1, 1, 3)
            bm, bp = oracle_mod.rpt2_var(prob, d, qlo, qc, qhi, a)

            def basis(zminus, zplus):
                rm = np.zeros(3); rm[0] = -zminus; rm[vn] = 1.0
                rp = np.zeros(3); rp[0] = zplus; rp[vn] = 1.0
                r0 = np.zeros(3); r0[vt] = 1.0
                return rm, rp, r0

            rm, rp, r0 = basis(z[0], z[1])           # interface between the cell below and the cell
            coef = np.linalg.solve(np.stack([rm, rp, r0], axis=1), a)
            np.testing.assert_allclose(bm, -mats[0, 1] * coef[0] * rm, atol=1e-13)
            rm, rp, r0 = basis(z[1], z[2])           # interface between the cell and the cell above
            coef = np.linalg.solve(np.stack([rm, rp, r0], axis=1), a)
            np.testing.assert_allclose(bp, mats[2, 1] * coef[1] * rp, atol=1e-13)


@pytest.mark.parametrize("transverse,limiter", [(1, 4), (2, 3), (0, 1), (2, 0)])
def test_uniform_material_is_constant_coefficient_acoustics(oracle_mod, transverse, limiter):
    mx, my = 11, 9
    rng = np.random.default_rng(7)
    base = rng.uniform(-1, 1, (3, my, mx))
    rho, c = 1.0, 2.0                                 # K = rho c^2 = 4
    pc = oracle_mod.Problem(oracle_mod.ACOUSTICS, mx, my, 0.1, 0.12, limiter=limiter,
                            transverse=transverse, bc=(BCP, BCP, 2, 1), param=(rho, c * c * rho, 0, 0))
    pv = var_problem(oracle_mod, mx, my, 0.1, 0.12, bc=(BCP, BCP, 2, 1), limiter=limiter,
                     transverse=transverse)
    qc = np.zeros(pc.shape); qc[:, 2:-2, 2:-2] = base
    qv = np.zeros(pv.shape); qv[:3, 2:-2, 2:-2] = base; qv[3, 2:-2, 2:-2] = rho; qv[4, 2:-2, 2:-2] = c
    dt = 0.8 * 0.1 / c
    oc, sc, _ = oracle_mod.step(pc, qc, dt)
    ov, sv, _ = oracle_mod.step(pv, qv, dt)
    np.testing.assert_allclose(ov[:3], oc, atol=1e-13)
    assert sv == pytest.approx(sc, rel=1e-14)
    np.testing.assert_array_equal(ov[3:, 2:-2, 2:-2], qv[3:, 2:-2, 2:-2])   # material carried unchanged


def test_pulse_transmission_and_reflection(oracle_mod):
    """A right-going pulse (p = Z1 u) in medium 1 meets medium 2 at x = 1/2.
    Afterwards the reflected pressure integrates to R I0 and the transmitted
    one to T (c2/c1) I0 (the pulse is compressed by c2/c1), with
    R = (Z2 - Z1)/(Z1 + Z2), T = 2 Z2/(Z1 + Z2) (LeVeque 2002, §9.7)."""
    mx, my = 400, 2
    dx = 1.0 / mx
    x = (np.arange(mx) + 0.5) * dx
    r1, c1, r2, c2 = 1.0, 1.0, 4.0, 0.5
    z1, z2 = r1 * c1, r2 * c2
    prob = var_problem(oracle_mod, mx, my, dx, dx, bc=(BCX, BCX, BCP, BCP), limiter=4)
    p0 = np.exp(-((x - 0.25) / 0.04) ** 2)
    q = np.zeros(prob.shape)
    q[0, 2:-2, 2:-2] = p0
    q[1, 2:-2, 2:-2] = p0 / z1
    q[3, 2:-2, 2:-2] = np.where(x < 0.5, r1, r2)
    q[4, 2:-2, 2:-2] = np.where(x < 0.5, c1, c2)
    dt = 0.8 * dx / max(c1, c2)
    nsteps = int(round(0.5 / dt))
    for _ in range(nsteps):
        q, _, _ = oracle_mod.step(prob, q, dt)
    p = q[0, 2, 2:-2]
    I0 = p0.sum() * dx
    refl = p[x < 0.5].sum() * dx
    trans = p[x > 0.5].sum() * dx
    R, T = (z2 - z1) / (z1 + z2), 2 * z2 / (z1 + z2)
    assert refl == pytest.approx(R * I0, rel=0.02)
    assert trans == pytest.approx(T * (c2 / c1) * I0, rel=0.02)
