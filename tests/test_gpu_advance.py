"""GPU parity of the time-step loop (mc_advance: ghost fill, fused step and
the device-side dt rule inside one CUDA graph) against the oracle's driver."""
import numpy as np
import pytest

import oracle
import paper_1308_1464_gb300 as mc
from paper_1308_1464_gb300 import workloads
from gpu_util import TOL, embed, initial_state, problems, scaled_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1308_1464_gb300.state import DeviceState  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1308_1464_gb300 import _build
    _build.build()
    oracle.build()


def test_acoustics_pulse_ten_steps():
    """Acoustics, 128 x 128, FP64, periodic, MC, CFL 0.9, 10 steps."""
    g = workloads.acoustics_pulse(128, 128)
    P = mc.BC_PERIODIC
    p, op = problems("acoustics", 128, 128, g.dx, g.dy, mc.F64, (P, P, P, P))
    dt0 = 0.9 * g.dx / 2.0
    assert dt0 == 0.003515625
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(g.q)
        t, dt, inb, nrej = ctx.advance(a.ptr, b.ptr, 10, 0.9, 1.0, 0.0, dt0)
        got = (b if inb else a).download()
    want, t_ref, dt_ref, nrej_ref, _ = oracle.advance(op, embed(op, g.q), 10, 0.9, 1.0, 0.0, dt0)
    assert nrej == nrej_ref == 0
    assert t == pytest.approx(t_ref, rel=1e-14) and t == pytest.approx(10 * dt0, rel=1e-14)
    assert dt == pytest.approx(dt_ref, rel=1e-14)
    assert scaled_error("acoustics", got, want[:, 2:-2, 2:-2]) <= 1e-12


@pytest.mark.parametrize("dtype", [mc.F64, mc.F32])
def test_rejection_and_retake(dtype):
    """An initial dt three times too large is rejected and retaken; the
    accepted sequence matches the oracle's driver."""
    mx, my = 64, 48
    q, dx, dy = initial_state("swe", mx, my, seed=2)
    W = mc.BC_WALL
    p, op = problems("swe", mx, my, dx, dy, dtype, (W, W, W, W))
    npdt = np.float64 if dtype == mc.F64 else np.float32
    qin = q.astype(npdt)
    qo = embed(op, qin.astype(np.float64))
    dt0 = 3.0 * 0.9 / oracle.max_cell_speed(op, oracle.bc_fill(op, qo))
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(qin)
        t, dt, inb, nrej = ctx.advance(a.ptr, b.ptr, 6, 0.9, 1.0, 0.0, dt0)
        got = (b if inb else a).download().astype(np.float64)
    want, t_ref, dt_ref, nrej_ref, _ = oracle.advance(op, qo, 6, 0.9, 1.0, 0.0, dt0)
    assert nrej == nrej_ref >= 1
    rel = 1e-12 if dtype == mc.F64 else 1e-5
    assert t == pytest.approx(t_ref, rel=rel)
    # FP32: dt follows the FP32 speeds, so states differ by more than one step's rounding
    assert scaled_error("swe", got, want[:, 2:-2, 2:-2]) <= (1e-11 if dtype == mc.F64 else 1e-4)


@pytest.mark.parametrize("mx,my,dtype", [(96, 80, mc.F32), (37, 23, mc.F32), (64, 50, mc.F64),
                                         (37, 23, mc.F64), (5, 3, mc.F32)])
def test_advance_host_matches_device_path(mx, my, dtype):
    """The host-buffer form (one contiguous transfer each way, repacked on the
    device: 16-byte words where rows allow, elements otherwise) gives the
    device path's bits; its buffers start with garbage, so every interior
    cell must come from the upload."""
    g = workloads.swe_dambreak(mx, my)
    W = mc.BC_WALL
    p, _ = problems("swe", mx, my, g.dx, g.dy, dtype, (W, W, W, W))
    qin = g.q.astype(np.float64 if dtype == mc.F64 else np.float32)
    dt0 = 0.9 * g.dx / (2.0 + np.sqrt(9.81 * 2.0))
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(qin)
        t1, dt1, inb, _ = ctx.advance(a.ptr, b.ptr, 7, 0.9, 1.0, 0.0, dt0)
        dev = (b if inb else a).download()
        a2, b2 = DeviceState(ctx), DeviceState(ctx)
        a2.buf.fill_(0x7F)
        b2.buf.fill_(0x3C)
        host = np.zeros_like(qin)
        t2, dt2, _ = ctx.advance_host(qin.ctypes.data, host.ctypes.data, a2.ptr, b2.ptr, 7, 0.9,
                                      1.0, 0.0, dt0)
    assert t1 == t2 and dt1 == dt2
    np.testing.assert_array_equal(dev, host)


def test_nonphysical_state_is_reported():
    """A negative depth in the input is flagged by the device status word."""
    q, dx, dy = initial_state("swe", 40, 30, seed=1)
    q[0, 10, 10] = -1.0
    W = mc.BC_WALL
    p, _ = problems("swe", 40, 30, dx, dy, mc.F32, (W, W, W, W))
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(q)
        with pytest.raises(mc.McError) as ei:
            ctx.step(a.ptr, b.ptr, 1e-4)
        assert ei.value.status == mc.MC_ENONPHYS
        # the status word was cleared: a good state steps cleanly afterwards
        q2, _, _ = initial_state("swe", 40, 30, seed=1)
        a.upload(q2)
        ctx.step(a.ptr, b.ptr, 1e-4)


def test_usage_example_runs():
    """The usage example of the package documentation: a lake at rest stays
    at rest over 100 steps of the time-step loop."""
    p = mc.Problem.make(mc.SWE_ROE, 512, 512, 1 / 256, 1 / 256, dtype=mc.F32,
                        bc=(mc.BC_WALL,) * 4, param=(9.81, 0, 0, 0))
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        q0 = np.zeros((3, 512, 512), np.float32)
        q0[0] = 1.0
        a.upload(q0)
        dt = 0.9 / ctx.max_cell_speed(a.ptr)
        t, dt, in_b, nrej = ctx.advance(a.ptr, b.ptr, 100, 0.9, 1.0, 0.0, dt)
        q = (b if in_b else a).download()
    assert nrej == 0 and t > 0
    np.testing.assert_array_equal(q[0], 1.0)
    np.testing.assert_array_equal(q[1:], 0.0)


@pytest.mark.parametrize("dtype", [mc.F64, mc.F32])
def test_degenerate_waves(dtype):
    """Zero and vanishing waves.  A lake at rest (every jump zero, so every
    wave and every limiter ratio's denominator is zero) stays exactly at
    rest.  FP64: momenta of 1e-60 give squared wave norms near 1e-120, whose
    product over a cell's six waves leaves the normal range; the step stays
    finite and equal to the oracle's."""
    n = 96
    W = mc.BC_WALL
    p, op = problems("swe", n, n, 1 / 64, 1 / 64, dtype, (W, W, W, W))
    npdt = np.float64 if dtype == mc.F64 else np.float32
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        q0 = np.zeros((3, n, n), npdt)
        q0[0] = 1.0
        a.upload(q0)
        ctx.step(a.ptr, b.ptr, 0.002)
        q = b.download()
        np.testing.assert_array_equal(q[0], 1.0)
        np.testing.assert_array_equal(q[1:], 0.0)
        if dtype == mc.F64:
            rng = np.random.default_rng(60)
            q1 = q0.copy()
            q1[1] = 1e-60 * rng.uniform(-1, 1, (n, n))
            a.upload(q1)
            ctx.step(a.ptr, b.ptr, 0.002)
            got = b.download()
            assert np.isfinite(got).all()
            want, _, _ = oracle.step(op, embed(op, q1), 0.002)
            want = want[:, 2:-2, 2:-2]
            np.testing.assert_array_equal(got[0], want[0])
            assert np.abs(got[1:] - want[1:]).max() <= 1e-12 * 1e-60
            assert np.abs(got[1]).max() > 1e-61


@pytest.mark.parametrize("mx,my,dtype", [(64, 20, mc.F32), (37, 23, mc.F32), (37, 23, mc.F64),
                                         (1, 1, mc.F64)])
def test_repack_moves_exactly_the_interior(mx, my, dtype):
    """mc_repack: dense -> layout writes the interior cells and nothing else
    (ghosts and padding keep their bytes), and layout -> dense reads back the
    same array that mc_download gives."""
    W = mc.BC_WALL
    p, _ = problems("swe", mx, my, 1.0 / mx, 1.0 / my, dtype, (W, W, W, W))
    npdt = np.float64 if dtype == mc.F64 else np.float32
    rng = np.random.default_rng(mx * 100 + my)
    q = (1.0 + rng.uniform(size=(3, my, mx))).astype(npdt)
    with mc.Context(p) as ctx:
        s = DeviceState(ctx)
        s.buf.fill_(0x5A)
        before = s.buf.cpu().numpy().copy()
        dense = torch.from_numpy(q.ravel().copy()).cuda()
        ctx.repack(dense.data_ptr(), s.ptr, True)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(s.download(), q)
        after = s.buf.cpu().numpy()
        # every byte outside the interior is untouched
        ref = DeviceState(ctx)
        ref.buf.copy_(torch.from_numpy(before).cuda())
        ref.upload(q)
        np.testing.assert_array_equal(after, ref.buf.cpu().numpy())
        back = torch.zeros_like(dense)
        ctx.repack(s.ptr, back.data_ptr(), False)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(back.cpu().numpy().reshape(q.shape), q)
        with pytest.raises(mc.McError):
            ctx.repack(s.ptr, s.ptr, False)
