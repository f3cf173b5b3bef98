"""GPU checks of the batched persistent step (mc_batch_advance): bitwise equal
to the per-patch launch loop and to one launch per step over all patches
(mc_batch_advance_steps), and per patch equal to the oracle advancing the
same patch with its own dt sequence (dt_k = cfl / smax_{k-1})."""
import numpy as np
import pytest

import oracle
import paper_1308_1464_gb300 as mc
from paper_1308_1464_gb300 import workloads
from gpu_util import G, field_scales

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1308_1464_gb300.state import PatchSet  # noqa: E402

W = mc.BC_WALL


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1308_1464_gb300 import _build
    _build.build()
    oracle.build()


def proto(dtype):
    return mc.Problem.make(mc.SWE_ROE, 16, 16, 1 / 128, 1 / 128, dtype=dtype, bc=(W,) * 4,
                           param=(G, 0, 0, 0))


def oracle_patch(q, dx, dy, nsteps, cfl):
    """The oracle's step applied nsteps times with the batched dt rule."""
    my, mx = q.shape[1:]
    op = oracle.Problem(oracle.SWE, mx, my, dx, dy, bc=(oracle.BC_WALL,) * 4, param=(G, 0, 0, 0))
    qq = np.zeros(op.shape)
    qq[:, 2:-2, 2:-2] = q
    smax = oracle.max_cell_speed(op, oracle.bc_fill(op, qq))
    t = 0.0
    for _ in range(nsteps):
        dt = cfl / smax
        qq, smax, _ = oracle.step(op, qq, dt)
        t += dt
    return qq[:, 2:-2, 2:-2], t


def small_patches(n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        mx, my = int(rng.integers(4, 70)), int(rng.integers(4, 70))
        x = (np.arange(mx) + 0.5) / 128
        y = (np.arange(my) + 0.5) / 128
        xc, yc = rng.uniform(0, mx / 128), rng.uniform(0, my / 128)
        q = np.zeros((3, my, mx))
        q[0] = 1.0 + 0.5 * np.exp(-50 * ((x[None, :] - xc) ** 2 + (y[:, None] - yc) ** 2))
        q[1] = 0.1 * rng.uniform(-1, 1, size=(my, mx))
        out.append((mx, my, 1 / 128, 1 / 128, q))
    return out


@pytest.mark.parametrize("dtype", [mc.F64, mc.F32])
def test_batched_equals_plain_and_oracle(dtype):
    pats = small_patches(23, seed=5)
    nsteps, cfl = 7, 0.9
    res = {}
    for form in ("batched", "plain", "steps"):
        ps = PatchSet(proto(dtype), pats)
        b = mc.Batch(proto(dtype), ps.pointers())
        b.set_tile_rows([8 + 8 * (k % 3) for k in range(len(pats))])   # uneven splits
        run = {"batched": b.advance, "plain": b.advance_plain, "steps": b.advance_steps}[form]
        t, inb = run(nsteps, cfl, want_t=True)
        res[form] = (ps.interiors(inb), t)
        b.close()
    for form in ("plain", "steps"):
        for qa, qb in zip(res["batched"][0], res[form][0]):
            np.testing.assert_array_equal(qa, qb)
        assert res["batched"][1] == res[form][1]
    tol = 1e-11 if dtype == mc.F64 else 2e-5 * nsteps
    for k, (mx, my, dx, dy, q) in enumerate(pats):
        qin = q.astype(np.float32).astype(np.float64) if dtype == mc.F32 else q
        want, t_ref = oracle_patch(qin, dx, dy, nsteps, cfl)
        S = field_scales("swe", want)
        got = res["batched"][0][k].astype(np.float64)
        err = max(np.abs(got[m] - want[m]).max() / S[m] for m in range(3))
        assert err <= tol, (k, mx, my, err)
        assert res["batched"][1][k] == pytest.approx(t_ref, rel=1e-12 if dtype == mc.F64 else 1e-5)


def test_full_configuration_sampled():
    """2000 patches (log-uniform sizes 16..256), FP32, 20 steps in one
    persistent launch: equal to the per-patch launch loop bitwise; 12 sampled
    patches recomputed by the oracle; mass conserved by the walls."""
    pats_w = workloads.swe_patches(2000)
    pats = [(p.nx, p.ny, p.grid.dx, p.grid.dy, p.grid.q) for p in pats_w]
    nsteps, cfl = 20, 0.9
    ps = PatchSet(proto(mc.F32), pats)
    b = mc.Batch(proto(mc.F32), ps.pointers())
    t, inb = b.advance(nsteps, cfl, want_t=True)
    got = ps.interiors(inb)
    b.close()
    ps2 = PatchSet(proto(mc.F32), pats)
    b2 = mc.Batch(proto(mc.F32), ps2.pointers())
    t2, inb2 = b2.advance_plain(nsteps, cfl, want_t=True)
    ref = ps2.interiors(inb2)
    b2.close()
    assert t == t2
    for a, c in zip(got, ref):
        np.testing.assert_array_equal(a, c)
    rng = np.random.default_rng(1)
    for k in rng.choice(len(pats), 12, replace=False):
        mx, my, dx, dy, q = pats[k]
        want, t_ref = oracle_patch(q.astype(np.float32).astype(np.float64), dx, dy, nsteps, cfl)
        S = field_scales("swe", want)
        err = max(np.abs(got[k][m].astype(np.float64) - want[m]).max() / S[m] for m in range(3))
        assert err <= 2e-5 * nsteps, (k, err)
        assert t[k] == pytest.approx(t_ref, rel=1e-5)
    for k in range(len(pats)):
        m0 = pats[k][4][0].astype(np.float32).astype(np.float64).sum()
        assert abs(got[k][0].astype(np.float64).sum() - m0) <= 1e-5 * m0


def test_bounded_wait_reports_timeout_and_batch_recovers():
    """Fault injection on the host: one patch's tasks wait for a completion
    that never comes.  The device waits are bounded (about a second), the call
    returns MC_ETIMEOUT instead of hanging, and the next advance is correct."""
    import time
    pats = small_patches(4, seed=9)
    ps = PatchSet(proto(mc.F32), pats)
    b = mc.Batch(proto(mc.F32), ps.pointers())
    b.inject_stall(2)
    t0 = time.time()
    with pytest.raises(mc.McError) as ei:
        b.advance(4, 0.9)
    assert ei.value.status == mc.MC_ETIMEOUT
    assert time.time() - t0 < 60
    # recovery: a clean run from the initial state equals the per-patch loop
    ps.reset()
    _, inb = b.advance(4, 0.9)
    got = ps.interiors(inb)
    ps.reset()
    _, inb2 = b.advance_plain(4, 0.9)
    ref = ps.interiors(inb2)
    for a, c in zip(got, ref):
        np.testing.assert_array_equal(a, c)
    b.close()


def test_tuned_split_is_bitwise_equal_to_untuned():
    """The autotuner changes only the work split: the tuned batch gives the
    same interiors and times, bit for bit, as the batch as created."""
    from paper_1308_1464_gb300 import autotune
    pats = small_patches(31, seed=9)
    sizes = [(p[0], p[1]) for p in pats]
    ps = PatchSet(proto(mc.F32), pats)
    b = mc.Batch(proto(mc.F32), ps.pointers())
    nsteps = 6
    t0, inb0 = b.advance(nsteps, 0.9, want_t=True)
    q0 = ps.interiors(inb0)
    desc, timings = autotune.tune_batch(b, sizes, ps.reset, nsteps=2, repeats=1)
    assert len(timings) > len(autotune.POLICIES)
    ps.reset()
    t1, inb1 = b.advance(nsteps, 0.9, want_t=True)
    for qa, qb in zip(q0, ps.interiors(inb1)):
        np.testing.assert_array_equal(qa, qb)
    assert t0 == t1 and inb0 == inb1
    b.close()
