"""Pins of the oracle's exact Euler Riemann solver and its pressure guesses (CPU only).

The solver (Toro, ch. 4) is pinned by facts it must satisfy, computed here
without its code:

* Newton's root equals the root found by bisection on the monotone pressure
  function;
* across a shock the Rankine-Hugoniot conditions (mass, momentum, energy)
  hold between the outer and star states; across a rarefaction the entropy
  p / rho^gamma and the Riemann invariant u +- 2c/(gamma-1) are unchanged;
* the two-rarefaction guess is exact when both waves are rarefactions, the
  primitive-variable guess is second-order accurate for weak jumps;
* the vacuum criterion matches the absence of a positive root.
"""
import math

import numpy as np
import pytest

from paper_1308_1464_gb300 import workloads

GAMMA = 1.4


def states(n, seed=5):
    return list(zip(*workloads.riemann_states(n, seed=seed)))


def star_densities_and_checks(rl, ul, pl, rr, ur, pr, ps, us):
    g = GAMMA
    for side, (r, u, p) in (("L", (rl, ul, pl)), ("R", (rr, ur, pr))):
        E = p / (g - 1) + 0.5 * r * u * u
        if ps > p:
            # shock: density from the Hugoniot curve, then all three jump conditions
            m = (g - 1) / (g + 1)
            rs = r * (ps / p + m) / (m * ps / p + 1)
            S = (rs * us - r * u) / (rs - r)
            Es = ps / (g - 1) + 0.5 * rs * us * us
            mom = (rs * us * us + ps) - (r * u * u + p) - S * (rs * us - r * u)
            ene = (us * (Es + ps)) - (u * (E + p)) - S * (Es - E)
            sc = max(abs(r * u * u + p), abs(u * (E + p)), 1.0) * (1 + abs(S))
            assert abs(mom) < 1e-9 * sc, (side, mom)
            assert abs(ene) < 1e-9 * sc, (side, ene)
        else:
            # rarefaction: isentropic, Riemann invariant carried through the fan
            rs = r * (ps / p) ** (1.0 / g)
            c, cs = math.sqrt(g * p / r), math.sqrt(g * ps / rs)
            assert abs(ps / rs ** g - p / r ** g) <= 1e-10 * p / r ** g
            if side == "L":
                inv, invs = u + 2 * c / (g - 1), us + 2 * cs / (g - 1)
            else:
                inv, invs = u - 2 * c / (g - 1), us - 2 * cs / (g - 1)
            assert abs(inv - invs) < 1e-9 * (1 + abs(inv)), (side, inv, invs)


def test_newton_matches_bisection_and_wave_relations(oracle_mod):
    n_ok = 0
    for rl, ul, pl, rr, ur, pr in states(400):
        ps, us, it, flag = oracle_mod.exact_riemann(GAMMA, rl, ul, pl, rr, ur, pr, tol=1e-12)
        pb, ub, fb = oracle_mod.exact_bisect(GAMMA, rl, ul, pl, rr, ur, pr)
        if flag & oracle_mod.RS_VACUUM:
            assert fb == oracle_mod.RS_VACUUM and ps == 0.0
            continue
        assert flag == 0
        n_ok += 1
        assert ps == pytest.approx(pb, rel=1e-10)
        assert us == pytest.approx(ub, rel=1e-9, abs=1e-9)
        star_densities_and_checks(rl, ul, pl, rr, ur, pr, ps, us)
    assert n_ok > 100


def test_vacuum_criterion(oracle_mod):
    g = GAMMA
    rl, pl, rr, pr = 1.0, 0.1, 1.0, 0.1
    c = math.sqrt(g * pl / rl)
    crit = 2.0 / (g - 1) * 2 * c
    _, _, _, flag = oracle_mod.exact_riemann(g, rl, -0.5 * crit * 1.01, pl, rr, 0.5 * crit * 1.01, pr)
    assert flag == oracle_mod.RS_VACUUM
    ps, _, _, flag = oracle_mod.exact_riemann(g, rl, -0.5 * crit * 0.99, pl, rr, 0.5 * crit * 0.99, pr)
    assert flag == 0 and 0 < ps < 1e-6
    # no positive root: f(0+) >= 0 exactly when vacuum is generated
    f0, _ = oracle_mod.pressure_function(g, rl, -0.5 * crit * 1.01, pl, rr, 0.5 * crit * 1.01, pr, 1e-300)
    assert f0 > 0


def test_two_rarefaction_guess_is_exact_for_two_rarefactions(oracle_mod):
    count = 0
    for rl, ul, pl, rr, ur, pr in states(400, seed=9):
        ps, us, it, flag = oracle_mod.exact_riemann(GAMMA, rl, ul, pl, rr, ur, pr, tol=1e-13)
        if flag != 0 or ps >= min(pl, pr):
            continue
        count += 1
        ptr = oracle_mod.seed(oracle_mod.SEED_TR, GAMMA, rl, ul, pl, rr, ur, pr)
        assert ptr == pytest.approx(ps, rel=1e-10)
    assert count > 20


def test_pv_guess_second_order_for_weak_jumps(oracle_mod):
    base = (1.0, 0.1, 1.0)
    errs = []
    for eps in (1e-2, 5e-3, 2.5e-3):
        rl, ul, pl = base
        rr, ur, pr = 1.0 + eps, 0.1 - 0.7 * eps, 1.0 + 1.3 * eps
        ps, _, _, _ = oracle_mod.exact_riemann(GAMMA, rl, ul, pl, rr, ur, pr, tol=1e-14)
        ppv = oracle_mod.seed(oracle_mod.SEED_PV, GAMMA, rl, ul, pl, rr, ur, pr)
        errs.append(abs(ppv - ps))
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5, errs


def test_adaptive_seed_choice(oracle_mod):
    g = GAMMA
    # small pressure ratio, PV inside [pmin, pmax] -> PV
    a = (1.0, 0.0, 1.0, 1.0, 0.0, 1.5)
    assert oracle_mod.seed(oracle_mod.SEED_ADAPTIVE, g, *a) == oracle_mod.seed(oracle_mod.SEED_PV, g, *a)
    # strong expansion: PV below pmin -> TR
    b = (1.0, -2.0, 1.0, 1.0, 2.0, 1.2)
    assert oracle_mod.seed(oracle_mod.SEED_ADAPTIVE, g, *b) == oracle_mod.seed(oracle_mod.SEED_TR, g, *b)
    # strong compression: PV above pmax -> TS
    c = (1.0, 3.0, 1.0, 1.0, -3.0, 1.1)
    assert oracle_mod.seed(oracle_mod.SEED_ADAPTIVE, g, *c) == oracle_mod.seed(oracle_mod.SEED_TS, g, *c)


def test_given_seed_and_fallback(oracle_mod):
    s = (1.0, 0.2, 2.0, 0.3, -0.4, 0.5)
    ps, us, it, flag = oracle_mod.exact_riemann(GAMMA, *s, tol=1e-12)
    # a perfect proposal converges in one update
    p1, u1, it1, f1 = oracle_mod.exact_riemann(GAMMA, *s, seed_mode=oracle_mod.SEED_GIVEN,
                                               p_given=ps, tol=1e-12)
    assert f1 == 0 and it1 == 1 and p1 == pytest.approx(ps, rel=1e-14)
    # a non-physical proposal falls back to the plain seed and still converges
    for bad in (float("nan"), -1.0, 1e30):
        p2, u2, it2, f2 = oracle_mod.exact_riemann(GAMMA, *s, seed_mode=oracle_mod.SEED_GIVEN,
                                                   p_given=bad, tol=1e-12)
        assert f2 == oracle_mod.RS_FALLBACK and p2 == pytest.approx(ps, rel=1e-12)
        assert it2 == it


def test_batch_matches_scalar(oracle_mod):
    st = workloads.riemann_states(64, seed=3)
    ps, us, it, fl = oracle_mod.exact_batch(GAMMA, *st, nthreads=2)
    for k in range(64):
        p1, u1, i1, f1 = oracle_mod.exact_riemann(GAMMA, *[a[k] for a in st])
        assert fl[k] == f1 and it[k] == i1
        if f1 == 0:
            assert ps[k] == p1 and us[k] == u1
