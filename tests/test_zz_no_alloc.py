"""mc_step_noalloc: the unsplit step for callers that cannot allocate device
memory (stream capture in progress, fixed plug-in memory budgets, loops that
must not risk the synchronisation of cudaMalloc/cudaFree).  It keeps its
16 bytes of scratch in a static device array; two calls in a row must each
match the context-based mc_step, so the second call also shows that the
array's previous contents were cleared.  Named to be collected last."""
import ctypes

import numpy as np
import pytest

import paper_1308_1464_gb300 as mc

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from gpu_util import TOL, initial_state, problems, scaled_error  # noqa: E402
from paper_1308_1464_gb300.state import DeviceState  # noqa: E402


@pytest.fixture(scope="module")
def L():
    from paper_1308_1464_gb300 import _build
    _build.build()
    lib = mc.lib()
    lib.mc_step_noalloc.argtypes = [ctypes.POINTER(mc.Problem), ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                    ctypes.c_void_p]
    return lib


def step_both(L, solver, dtype, bc, q, scale_momentum):
    mx, my = q.shape[2], q.shape[1]
    p, _ = problems(solver, mx, my, 2.0 / mx, 2.0 / my, dtype, bc)
    q = q.copy()
    if solver == "swe":
        q[1:] *= scale_momentum
    npdt = np.float64 if dtype == mc.F64 else np.float32
    qin = q.astype(npdt)
    dt = 1e-4
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(qin)
        smax_ctx = ctx.step(a.ptr, b.ptr, dt)
        want = b.download()
        a2, b2 = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a2.upload(qin)
        smax = ctypes.c_double(-1.0)
        st = L.mc_step_noalloc(ctypes.byref(p), a2.ptr, b2.ptr, dt, ctypes.byref(smax), None)
        assert st == mc.MC_OK, mc.last_error()
        got = b2.download()
    return got.astype(np.float64), want.astype(np.float64), smax.value, smax_ctx


def test_noalloc_step_matches_context_step_twice(L):
    W = mc.BC_WALL
    q, _, _ = initial_state("swe", 90, 70, seed=12)
    # first call: fast flow (large smax); second: slow flow, so a maximum left
    # over from the first call would show
    got1, want1, s1, r1 = step_both(L, "swe", mc.F32, (W, W, W, W), q, 4.0)
    got2, want2, s2, r2 = step_both(L, "swe", mc.F32, (W, W, W, W), q, 0.25)
    assert scaled_error("swe", got1, want1) <= TOL[mc.F32]
    assert scaled_error("swe", got2, want2) <= TOL[mc.F32]
    assert s1 == r1 and s2 == r2 and s2 < s1


def test_noalloc_rejects_invalid_arguments(L):
    p, _ = problems("swe", 8, 8, 0.1, 0.1, mc.F32, (mc.BC_WALL,) * 4)
    p.mbc = 3
    st = L.mc_step_noalloc(ctypes.byref(p), 16, 32, 0.1, None, None)
    assert st == mc.MC_EINVAL and "mbc" in mc.last_error()
