"""The exact-solution Euler step with the learned pressure seed (GPU).

A seed changes only where Newton starts, so the step must still match the
oracle (which solves from Toro's guess to 1e-14) within the parity
tolerance, whatever the network: a trained one, and an untrained one whose
poor proposals exercise the restart from the plain guess.  The context's
Newton counters report the work.
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

from paper_1308_1464_gb300.seednet import initial_params, train_seed_net  # noqa: E402
from paper_1308_1464_gb300.state import DeviceState  # noqa: E402

X = mc.BC_EXTRAP


@pytest.fixture(scope="module")
def nets():
    from paper_1308_1464_gb300 import _build
    _build.build()
    oracle.build()
    # training quality is covered by test_gpu_mlp.py; a seed only changes
    # where Newton starts, so the parity below holds for any network
    trained, losses, _ = train_seed_net(ntrain=1 << 16, epochs=4)
    assert np.isfinite(losses).all() and losses[-1] < losses[0], losses
    untrained = mc.SeedNet()
    untrained.set_params(initial_params(mc, seed=5))
    return {"trained": trained, "untrained": untrained}


@pytest.mark.parametrize("which", [None, "trained", "untrained"])
@pytest.mark.parametrize("dtype", [mc.F32, mc.F64])
def test_seeded_step_parity(nets, which, dtype):
    mx, my = 70, 45
    q, dx, dy = initial_state("euler_godunov", mx, my, seed=4)
    p, op = problems("euler_godunov", mx, my, dx, dy, dtype, (X, X, X, X))
    npdt = np.float64 if dtype == mc.F64 else np.float32
    qin = q.astype(npdt)
    qo = embed(op, qin.astype(np.float64))
    dt = 0.8 / oracle.max_cell_speed(op, oracle.bc_fill(op, qo))
    with mc.Context(p) as ctx:
        ctx.set_seed_net(nets[which] if which else None)
        ctx.newton_stats(reset=True)
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        a.upload(qin)
        ctx.step(a.ptr, b.ptr, dt)
        got = b.download().astype(np.float64)
        updates, solves = ctx.newton_stats(reset=True)
    want, _, _ = oracle.step(op, qo, dt)
    assert scaled_error("euler_godunov", got, want[:, 2:-2, 2:-2]) <= TOL[dtype]
    assert solves >= 2 * mx * my and updates >= solves


def test_seed_net_only_for_the_exact_solver(nets):
    p, _ = problems("euler", 8, 8, 0.1, 0.1, mc.F32, (X, X, X, X))
    with mc.Context(p) as ctx:
        with pytest.raises(mc.McError):
            ctx.set_seed_net(nets["trained"])
