"""GPU parity of the exact Euler Riemann solver (mc_riemann_exact) against the
oracle's solver, for every plain seed, the learned seed with an untrained
network (exercising the fallback), and a sampled full-size batch of 2^24
interfaces in the benchmark's launch configuration."""
import numpy as np
import pytest

import oracle
import paper_1308_1464_gb300 as mc
from paper_1308_1464_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

GAMMA = 1.4
ORACLE_SEED = {mc.SEED_ADAPTIVE: oracle.SEED_ADAPTIVE, mc.SEED_PV: oracle.SEED_PV,
               mc.SEED_TR: oracle.SEED_TR, mc.SEED_TS: oracle.SEED_TS,
               mc.SEED_PVTR: oracle.SEED_PVTR}


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1308_1464_gb300 import _build
    _build.build()
    oracle.build()


def gpu_solve(states32, seed_mode=mc.SEED_ADAPTIVE, net=None, tol=1e-8, max_iter=30, gamma=GAMMA):
    n = states32[0].size
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in states32]
    ps = torch.empty(n, dtype=torch.float32, device="cuda")
    us = torch.empty_like(ps)
    it = torch.empty(n, dtype=torch.uint8, device="cuda")
    fl = torch.empty_like(it)
    stats = torch.zeros(8, dtype=torch.int64, device="cuda")
    mc.riemann_exact(n, gamma, [d.data_ptr() for d in dev], ps.data_ptr(), us.data_ptr(),
                     it.data_ptr(), fl.data_ptr(), seed_mode, net, tol, max_iter, stats.data_ptr())
    torch.cuda.synchronize()
    return (ps.cpu().numpy(), us.cpu().numpy(), it.cpu().numpy().astype(np.int32),
            fl.cpu().numpy().astype(np.int32), stats.cpu().numpy())


def f32_states(n, seed, offset=0):
    return [a.astype(np.float32) for a in workloads.riemann_states(n, seed=seed, offset=offset)]


def compare(states32, ps, us, it, fl, ref):
    ps_r, us_r, it_r, fl_r = ref
    np.testing.assert_array_equal(fl & mc.RS_VACUUM, fl_r & oracle.RS_VACUUM)
    ok = (fl_r & oracle.RS_VACUUM) == 0
    assert ok.sum() > 0
    # FP64 iterates on both sides; outputs are rounded to FP32
    np.testing.assert_allclose(ps[ok], ps_r[ok].astype(np.float32), rtol=3e-7, atol=0)
    scale = 1.0 + np.abs(us_r[ok])
    assert np.all(np.abs(us[ok] - us_r[ok]) <= 1e-6 * scale)
    assert np.all(ps[~ok] == 0.0) and np.all(np.isnan(us[~ok]))
    d = np.abs(it[ok] - it_r[ok])
    assert d.max() <= 1 and (d == 0).mean() >= 0.99, (d.max(), (d == 0).mean())


@pytest.mark.parametrize("mode", [mc.SEED_ADAPTIVE, mc.SEED_PV, mc.SEED_TR, mc.SEED_TS,
                                  mc.SEED_PVTR])
def test_plain_seeds_match_oracle(mode):
    st = f32_states(20011, seed=21)
    ps, us, it, fl, stats = gpu_solve(st, mode)
    ref = oracle.exact_batch(GAMMA, *[a.astype(np.float64) for a in st], seed_mode=ORACLE_SEED[mode])
    compare(st, ps, us, it, fl, ref)
    n = st[0].size
    assert stats[0] == n
    assert stats[1] == int(((fl & mc.RS_VACUUM) != 0).sum())
    assert stats[3] == int(((fl & mc.RS_NOCONV) != 0).sum())
    assert stats[4] == int(it.sum()) and stats[5] == int(it.max())


@pytest.mark.parametrize("gamma", [5.0 / 3.0, 1.3, 2.0])
def test_other_gammas_match_oracle(gamma):
    """2 gamma / (gamma - 1) = 5 and 4 (integer: the powers come from roots
    and products) and 8.67 (not an integer: FP64 pow); the same parity as at
    gamma = 1.4."""
    st = f32_states(20011, seed=22)
    ps, us, it, fl, stats = gpu_solve(st, mc.SEED_ADAPTIVE, gamma=gamma)
    r = [a.astype(np.float64) for a in st]
    ref = oracle.exact_batch(gamma, *r, seed_mode=oracle.SEED_ADAPTIVE)
    cl, cr = np.sqrt(gamma * r[2] / r[0]), np.sqrt(gamma * r[5] / r[3])
    vac = 2.0 / (gamma - 1.0) * (cl + cr) <= r[4] - r[1]
    np.testing.assert_array_equal((fl & mc.RS_VACUUM) != 0, vac)
    compare(st, ps, us, it, fl, ref)
    assert stats[3] == 0


def test_vacuum_criterion_and_edge_cases():
    # vacuum by construction, tiny and ragged sizes
    for n in (1, 31, 33, 100):
        st = f32_states(n, seed=n)
        ps, us, it, fl, _ = gpu_solve(st)
        r = [a.astype(np.float64) for a in st]
        cl, cr = np.sqrt(GAMMA * r[2] / r[0]), np.sqrt(GAMMA * r[5] / r[3])
        vac = 2.0 / (GAMMA - 1.0) * (cl + cr) <= r[4] - r[1]
        np.testing.assert_array_equal((fl & mc.RS_VACUUM) != 0, vac)
        assert np.all(it[vac] == 0)


def test_learned_seed_with_untrained_network_falls_back():
    """Random weights: bad proposals fall back to the plain seed; p* agrees."""
    rng = np.random.default_rng(3)
    params = np.zeros(mc.MLP_NPARAM, dtype=np.float32)
    params[: mc.MLP_NWEIGHT] = rng.normal(scale=0.5, size=mc.MLP_NWEIGHT)
    params[:16 * 64].reshape(16, 64)[10:] = 0.0
    params[mc.MLP_NWEIGHT + 10:] = 1.0    # sigma
    net = mc.SeedNet()
    net.set_params(params.ctypes.data)
    st = f32_states(8000, seed=4)
    ps_m, us_m, it_m, fl_m, stats = gpu_solve(st, mc.SEED_MLP, net)
    ps_p, us_p, it_p, fl_p, _ = gpu_solve(st, mc.SEED_ADAPTIVE)
    ok = (fl_p & mc.RS_VACUUM) == 0
    np.testing.assert_array_equal(fl_m & mc.RS_VACUUM, fl_p & mc.RS_VACUUM)
    # the same root to within the convergence tolerance: equal or one FP32 ulp
    np.testing.assert_allclose(ps_m[ok], ps_p[ok], rtol=1.2e-7, atol=0)
    assert stats[2] == int(((fl_m & mc.RS_FALLBACK) != 0).sum())
    # fallback rows count the wasted updates too
    fb = ok & ((fl_m & mc.RS_FALLBACK) != 0)
    assert np.all(it_m[fb] >= it_p[fb])


def test_full_size_sampled():
    """2^24 interfaces (the benchmark's batch), adaptive seed; 20000 sampled
    interfaces recomputed by the oracle, flags checked everywhere."""
    n = 1 << 24
    st = f32_states(n, seed=1308)
    ps, us, it, fl, stats = gpu_solve(st)
    r = [a.astype(np.float64) for a in st]
    cl, cr = np.sqrt(GAMMA * r[2] / r[0]), np.sqrt(GAMMA * r[5] / r[3])
    vac = 2.0 / (GAMMA - 1.0) * (cl + cr) <= r[4] - r[1]
    np.testing.assert_array_equal((fl & mc.RS_VACUUM) != 0, vac)
    idx = np.random.default_rng(0).choice(n, 20000, replace=False)
    sub = [a[idx] for a in st]
    ref = oracle.exact_batch(GAMMA, *[a.astype(np.float64) for a in sub])
    compare(sub, ps[idx], us[idx], it[idx], fl[idx], ref)
    assert stats[0] == n and stats[3] == 0


@pytest.mark.parametrize("mode", [mc.SEED_ADAPTIVE, mc.SEED_TR, mc.SEED_PVTR])
def test_mixed_precision_newton_matches_oracle(mode):
    """FP32 Newton stage then FP64 updates to the same |dp|/p < 1e-8 test:
    p* and u* as the oracle's; the update counts are reported per stage (the
    FP64 stage takes about two updates per interface)."""
    st = f32_states(20011, seed=23)
    ps, us, it, fl, stats = gpu_solve(st, mode | mc.NEWTON_MIXED)
    ps_r, us_r, it_r, fl_r = oracle.exact_batch(GAMMA, *[a.astype(np.float64) for a in st],
                                                seed_mode=ORACLE_SEED[mode])
    np.testing.assert_array_equal(fl & mc.RS_VACUUM, fl_r & oracle.RS_VACUUM)
    ok = (fl_r & oracle.RS_VACUUM) == 0
    np.testing.assert_allclose(ps[ok], ps_r[ok].astype(np.float32), rtol=3e-7, atol=0)
    assert np.all(np.abs(us[ok] - us_r[ok]) <= 1e-6 * (1.0 + np.abs(us_r[ok])))
    assert (fl & mc.RS_NOCONV).sum() == 0
    nonvac = stats[0] - stats[1]
    assert stats[6] + stats[7] == stats[4] == int(it.sum())
    f64_per = stats[7] / nonvac
    print(f"mode {mode}: FP32 updates {stats[6] / nonvac:.3f}, FP64 updates {f64_per:.3f} per solve "
          f"(all-FP64 oracle {it_r[ok].mean():.3f})")
    assert 1.0 <= f64_per <= 2.5


def test_mixed_precision_learned_seed():
    """The learned seed with the FP32 stage: an untrained (zero) network
    proposes p_TR, the stage and the FP64 finish still reach the oracle's p*."""
    net = mc.SeedNet()
    params = np.zeros(mc.MLP_NPARAM, dtype=np.float32)
    params[mc.MLP_NWEIGHT + 10:] = 1.0
    net.set_params(params.ctypes.data)
    st = f32_states(8191, seed=29)
    ps, us, it, fl, stats = gpu_solve(st, mc.SEED_MLP | mc.NEWTON_MIXED, net)
    ps_r, us_r, it_r, fl_r = oracle.exact_batch(GAMMA, *[a.astype(np.float64) for a in st])
    ok = (fl_r & oracle.RS_VACUUM) == 0
    np.testing.assert_allclose(ps[ok], ps_r[ok].astype(np.float32), rtol=3e-7, atol=0)
    assert stats[6] + stats[7] == stats[4]
    net.close()
