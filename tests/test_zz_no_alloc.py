"""mc_step_noalloc: the unsplit step for callers that cannot allocate device
memory -- plug-ins whose host hands them a fixed device-memory budget and owns
every allocation, and loops that must not risk the device synchronisation of
cudaMalloc/cudaFree.  The call keeps its scratch (192 bytes: speed maximum,
status word, tensor map) in a 256-byte static device array shared by every
call, so each call must clear what the previous one left there.

The main test runs the calls in a fresh child process that never creates a
context (so nothing else has prepared the kernels' shared-memory limits),
for all six solvers in FP32 and FP64, two calls in a row per case; the
parent compares each result with the oracle at the per-step tolerance and
with the context-based mc_step.  A second test repeats two calls inside this
process, after whatever tests ran before.  The file is named to be collected
last, so that a run that stops at the first failure has run every other test
before it."""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)

import paper_1308_1464_gb300 as mc  # noqa: E402

W, X, P = mc.BC_WALL, mc.BC_EXTRAP, mc.BC_PERIODIC
# (solver, boundary kinds): every solver, each with a boundary mix it supports
SOLVERS = [("acoustics", (P, P, W, W)), ("swe", (W, W, W, W)), ("euler", (X, X, X, X)),
           ("advection", (P, P, X, W)), ("acoustics_var", (W, X, P, P)),
           ("euler_godunov", (X, X, P, P))]
MX, MY = 90, 70   # 4 bands of 29 columns (the last ragged), two row tiles of 64 with a tail


def _cases():
    """(solver, dtype, bc, call index, dx scale): the second call of each case
    uses cells twice as large, so its speed maximum (per unit length) is about
    half the first's and a maximum left over from the first call would show."""
    for solver, bc in SOLVERS:
        for dtype in (mc.F32, mc.F64):
            yield solver, dtype, bc


def _problem(solver, dtype, bc, call):
    from gpu_util import problems
    d = (1.0 if call == 0 else 2.0) / MX
    return problems(solver, MX, MY, d, d, dtype, bc)


def _input(solver, call):
    from gpu_util import initial_state
    q, _, _ = initial_state(solver, MX, MY, seed=20 + call)
    return q


def _padded(p, interior, torch):
    """A device state array in the library layout holding `interior`."""
    lay = mc.layout_of(p)
    tdt = torch.float64 if lay.elem_bytes == 8 else torch.float32
    buf = torch.zeros(int(lay.meqn * lay.ld_field), dtype=tdt, device="cuda")
    v = buf.view(int(lay.meqn), p.my + 4, int(lay.ld_x))
    x0 = int(lay.x_offset)
    v[:, 2:-2, x0: x0 + p.mx] = torch.from_numpy(np.ascontiguousarray(interior)).to(tdt).cuda()
    return buf, v


def _interior(p, v):
    lay = mc.layout_of(p)
    x0 = int(lay.x_offset)
    return v[:, 2:-2, x0: x0 + p.mx].double().cpu().numpy()


def _child(out_path):
    """Runs in a fresh process: mc_step_noalloc only, no context."""
    import torch
    torch.cuda.set_device(0)
    L = mc.lib()
    res = {}
    for solver, dtype, bc in _cases():
        for call in (0, 1):
            p, _ = _problem(solver, dtype, bc, call)
            npdt = np.float64 if dtype == mc.F64 else np.float32
            q = _input(solver, call).astype(npdt)
            dt = np.load(out_path + ".in.npz")[f"dt_{solver}_{dtype}_{call}"]
            a, _ = _padded(p, q, torch)
            b, vb = _padded(p, np.zeros_like(q), torch)
            smax = ctypes.c_double(-1.0)
            st = L.mc_step_noalloc(ctypes.byref(p), a.data_ptr(), b.data_ptr(), float(dt),
                                   ctypes.byref(smax), None)
            if st != mc.MC_OK:
                raise RuntimeError(f"{solver} dtype {dtype} call {call}: {mc.last_error()}")
            torch.cuda.synchronize()
            res[f"q_{solver}_{dtype}_{call}"] = _interior(p, vb)
            res[f"s_{solver}_{dtype}_{call}"] = smax.value
    np.savez(out_path, **res)


def _oracle_step(solver, dtype, bc, call):
    import oracle
    from gpu_util import embed
    p, op = _problem(solver, dtype, bc, call)
    npdt = np.float64 if dtype == mc.F64 else np.float32
    q = _input(solver, call).astype(npdt).astype(np.float64)
    qo = embed(op, q)
    dt = 0.9 / oracle.max_cell_speed(op, oracle.bc_fill(op, qo))
    want, smax_ref, _ = oracle.step(op, qo, dt)
    return p, dt, want[:, 2:-2, 2:-2], smax_ref


if __name__ == "__main__" and len(sys.argv) == 3 and sys.argv[1] == "--child":
    _child(sys.argv[2])
    sys.exit(0)


pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def built():
    import oracle
    from paper_1308_1464_gb300 import _build
    _build.build()
    oracle.build()


def _context_step(p, q, dt):
    from paper_1308_1464_gb300.state import DeviceState
    with mc.Context(p) as ctx:
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(q)
        s = ctx.step(a.ptr, b.ptr, dt)
        return b.download().astype(np.float64), s


def test_noalloc_fresh_process_all_solvers(built, tmp_path):
    from gpu_util import TOL, scaled_error
    ref = {}
    dts = {}
    for solver, dtype, bc in _cases():
        for call in (0, 1):
            p, dt, want, smax_ref = _oracle_step(solver, dtype, bc, call)
            ref[(solver, dtype, call)] = (p, dt, want, smax_ref)
            dts[f"dt_{solver}_{dtype}_{call}"] = dt
    out = str(tmp_path / "noalloc")
    np.savez(out + ".in.npz", **dts)
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + HERE)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--child", out],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    got = np.load(out + ".npz")
    for solver, dtype, bc in _cases():
        npdt = np.float64 if dtype == mc.F64 else np.float32
        for call in (0, 1):
            p, dt, want, smax_ref = ref[(solver, dtype, call)]
            q = got[f"q_{solver}_{dtype}_{call}"]
            s = float(got[f"s_{solver}_{dtype}_{call}"])
            err = scaled_error(solver, q, want)
            assert err <= TOL[dtype], f"{solver} dtype {dtype} call {call}: oracle error {err:.3e}"
            assert s == pytest.approx(smax_ref, rel=1e-13 if dtype == mc.F64 else 2e-6), \
                (solver, dtype, call, s, smax_ref)
            # the context-based step of the same input and dt
            want_ctx, s_ctx = _context_step(p, _input(solver, call).astype(npdt), dt)
            err = scaled_error(solver, q, want_ctx)
            assert err <= TOL[dtype], f"{solver} dtype {dtype} call {call}: mc_step error {err:.3e}"
            assert s == s_ctx
        # the second call's cells are twice as large: no maximum left over
        assert got[f"s_{solver}_{dtype}_1"] < got[f"s_{solver}_{dtype}_0"]


def test_noalloc_two_calls_in_this_process(built):
    """Two calls in a row in the test process itself, after the other tests."""
    from gpu_util import TOL, scaled_error
    L = mc.lib()
    for solver, dtype, bc in (("swe", mc.F32, (W, W, W, W)), ("euler_godunov", mc.F64, (X, X, P, P))):
        smaxes = []
        for call in (0, 1):
            p, dt, want, _ = _oracle_step(solver, dtype, bc, call)
            npdt = np.float64 if dtype == mc.F64 else np.float32
            q = _input(solver, call).astype(npdt)
            a, _ = _padded(p, q, torch)
            b, vb = _padded(p, np.zeros_like(q), torch)
            smax = ctypes.c_double(-1.0)
            st = L.mc_step_noalloc(ctypes.byref(p), a.data_ptr(), b.data_ptr(), dt,
                                   ctypes.byref(smax), None)
            assert st == mc.MC_OK, mc.last_error()
            got = _interior(p, vb)
            want_ctx, s_ctx = _context_step(p, q, dt)
            assert scaled_error(solver, got, want_ctx) <= TOL[dtype]
            assert scaled_error(solver, got, want) <= TOL[dtype]
            assert smax.value == s_ctx
            smaxes.append(smax.value)
        assert smaxes[1] < smaxes[0]


def test_noalloc_rejects_invalid_arguments(built):
    from gpu_util import problems
    L = mc.lib()
    p, _ = problems("swe", 8, 8, 0.1, 0.1, mc.F32, (W,) * 4)
    p.mbc = 3
    st = L.mc_step_noalloc(ctypes.byref(p), 16, 32, 0.1, None, None)
    assert st == mc.MC_EINVAL and "mbc" in mc.last_error()
    p.mbc = 2
    st = L.mc_step_noalloc(ctypes.byref(p), 16, 16, 0.1, None, None)
    assert st == mc.MC_EINVAL and "differ" in mc.last_error()
