"""GPU parity of refined patches with their own time steps (mc_amr_*).

The coarse grid and every patch after each coarse step (ratio fine steps of
every patch, ghost layers from neighbouring patches or the interpolated
coarse state, covered coarse cells averaged down) are compared with the
oracle's two-level step on the same rounded input.  One coarse step chains
ratio + 1 fused steps, so the FP32 bound is the per-step tolerance times
(ratio + 1).  With refluxing the coarse cells outside the patches also get
the flux correction, and on a periodic FP64 grid the coarse sum is conserved
to rounding.
"""
import numpy as np
import pytest

import oracle
import paper_1308_1464_gb300 as mc
from gpu_util import TOL, embed, initial_state, problems, scaled_error

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1308_1464_gb300.state import DeviceState  # noqa: E402

W, X, P = mc.BC_WALL, mc.BC_EXTRAP, mc.BC_PERIODIC


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1308_1464_gb300 import _build
    _build.build()
    oracle.build()


def dev_array(prob):
    lay = mc.layout_of(prob)
    return torch.zeros(int(lay.bytes), dtype=torch.uint8, device="cuda"), lay


def upload_interior(buf, lay, prob, q):
    """Write the interior (nplane, my, mx) of a state array in the library layout."""
    t = torch.float64 if lay.elem_bytes == 8 else torch.float32
    v = buf.view(t)[: lay.meqn * lay.ld_field].view(int(lay.meqn), prob.my + 4, int(lay.ld_x))
    x0 = int(lay.x_offset)
    v[:, 2:-2, x0: x0 + prob.mx] = torch.from_numpy(q).to(v.dtype).cuda()


def interior(buf, lay, prob):
    t = torch.float64 if lay.elem_bytes == 8 else torch.float32
    v = buf.view(t)[: lay.meqn * lay.ld_field].view(int(lay.meqn), prob.my + 4, int(lay.ld_x))
    x0 = int(lay.x_offset)
    torch.cuda.synchronize()
    return v[:, 2:-2, x0: x0 + prob.mx].double().cpu().numpy()


CASES = [
    ("advection", mc.F64, (P, P, P, P), 2, [(4, 3, 6, 5), (10, 3, 4, 5)]),
    ("swe", mc.F32, (W, W, W, W), 2, [(0, 0, 5, 4), (5, 0, 4, 4), (3, 7, 8, 5)]),
    ("euler", mc.F64, (X, X, X, X), 4, [(2, 2, 5, 4), (9, 6, 6, 5)]),
    ("euler_godunov", mc.F32, (X, X, W, W), 2, [(6, 4, 7, 6)]),
    ("swe", mc.F64, (W, X, P, P), 4, [(0, 2, 4, 4), (4, 2, 4, 4)]),
]


@pytest.mark.parametrize("reflux", [False, True])
@pytest.mark.parametrize("solver,dtype,bc,ratio,patches", CASES)
def test_amr_parity(solver, dtype, bc, ratio, patches, reflux):
    mx, my = 18, 14
    q, dx, dy = initial_state(solver, mx, my, seed=6)
    p, op = problems(solver, mx, my, dx, dy, dtype, bc)
    if solver == "advection":
        p.param[0], p.param[1] = 1.0, -0.6
    npdt = np.float64 if dtype == mc.F64 else np.float32
    qin = q.astype(npdt)
    qo = embed(op, qin.astype(np.float64))
    dt = 0.45 / oracle.max_cell_speed(op, oracle.bc_fill(op, qo))
    # fine initial data: each coarse value repeated on its fine cells
    fine_q = [np.repeat(np.repeat(qin[:, cj0: cj0 + ch, ci0: ci0 + cw], ratio, 1), ratio, 2)
              for (ci0, cj0, cw, ch) in patches]
    ca, lay = dev_array(p)
    cb, _ = dev_array(p)
    upload_interior(ca, lay, p, qin)
    fbufs, fprobs, flays = [], [], []
    for (ci0, cj0, cw, ch), fq in zip(patches, fine_q):
        fp = mc.amr_fine_problem(p, ratio, ci0, cj0, cw, ch)
        a, fl = dev_array(fp)
        b, _ = dev_array(fp)
        upload_interior(a, fl, fp, fq)
        fbufs.append((a, b))
        fprobs.append(fp)
        flays.append(fl)
    amr = mc.Amr(p, ratio, [(ci0, cj0, cw, ch, a.data_ptr(), b.data_ptr())
                            for (ci0, cj0, cw, ch), (a, b) in zip(patches, fbufs)], reflux=reflux)
    # oracle state
    oqc = qo.copy()
    oqf = []
    for (ci0, cj0, cw, ch), fq in zip(patches, fine_q):
        pf = oracle.fine_problem(op, ratio, (ci0, cj0, cw, ch))
        a = np.zeros(pf.shape)
        a[:, 2:-2, 2:-2] = fq.astype(np.float64)
        oqf.append(a)
    opatches = [tuple(pt) for pt in patches]
    tol = TOL[dtype] * (ratio + 1)
    cur_a = True
    for step in range(2):
        c_in_b, f_in_b = amr.advance(ca.data_ptr() if cur_a else cb.data_ptr(),
                                     cb.data_ptr() if cur_a else ca.data_ptr(), 1, dt)
        cur_a = not cur_a
        oqc, flags = oracle.amr_step(op, ratio, opatches, oqc, oqf, dt, reflux=reflux)
        assert flags == 0
        got_c = interior(ca if cur_a else cb, lay, p)
        assert scaled_error(solver, got_c, oqc[:, 2:-2, 2:-2]) <= tol * (step + 1), step
        for k, ((a, b), fp, fl) in enumerate(zip(fbufs, fprobs, flays)):
            got_f = interior(b if f_in_b else a, fl, fp)
            err = scaled_error(solver, got_f, oqf[k][:, 2:-2, 2:-2])
            assert err <= tol * (step + 1), (step, k, err)
    amr.close()


def test_amr_rejects_bad_patches():
    p, _ = problems("swe", 10, 10, 0.1, 0.1, mc.F32, (W, W, W, W))
    fake = 256
    with pytest.raises(mc.McError):
        mc.Amr(p, 2, [(8, 0, 4, 4, fake, fake * 2)])          # leaves the interior
    with pytest.raises(mc.McError):
        mc.Amr(p, 2, [(0, 0, 4, 4, fake, fake * 2), (3, 3, 4, 4, fake * 3, fake * 4)])   # overlap


@pytest.mark.parametrize("solver,trans", [("swe", 1), ("euler", 2), ("advection", 0)])
def test_reflux_conserves_on_the_gpu(solver, trans):
    """Periodic FP64 coarse grid, three separated patches: the sum over the
    coarse cells stays at its initial value to rounding with refluxing."""
    mx, my, ratio = 24, 20, 2
    q, dx, dy = initial_state(solver, mx, my, seed=3)
    p, op = problems(solver, mx, my, dx, dy, mc.F64, (P, P, P, P), transverse=trans)
    patches = [(3, 2, 5, 6), (12, 9, 6, 5), (4, 13, 7, 4)]
    dt = 0.4 / oracle.max_cell_speed(op, oracle.bc_fill(op, embed(op, q)))
    ca, lay = dev_array(p)
    cb, _ = dev_array(p)
    upload_interior(ca, lay, p, q)
    bufs = []
    for (ci0, cj0, cw, ch) in patches:
        fp = mc.amr_fine_problem(p, ratio, ci0, cj0, cw, ch)
        a, fl = dev_array(fp)
        b, _ = dev_array(fp)
        upload_interior(a, fl, fp, np.repeat(np.repeat(q[:, cj0: cj0 + ch, ci0: ci0 + cw], ratio, 1), ratio, 2))
        bufs.append((a, b))
    amr = mc.Amr(p, ratio, [(ci0, cj0, cw, ch, a.data_ptr(), b.data_ptr())
                            for (ci0, cj0, cw, ch), (a, b) in zip(patches, bufs)], reflux=True)
    c_in_b, _ = amr.advance(ca.data_ptr(), cb.data_ptr(), 4, dt)
    got = interior(cb if c_in_b else ca, lay, p)
    meqn = op.meqn
    s0, s1 = q[:meqn].sum(axis=(1, 2)), got[:meqn].sum(axis=(1, 2))
    assert np.abs(s1 - s0).max() <= 1e-12 * np.abs(q[:meqn]).sum(axis=(1, 2)).max(), (s0, s1)
    amr.close()
