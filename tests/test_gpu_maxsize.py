"""A grid whose state arrays pass 2^31 elements (and 2^32 bytes).

The shallow-water step on 32768 x 32768 cells in FP32: a state plane holds
1.07e9 elements, so plane 2 starts past element 2^31 and plane 1 past byte
2^32.  Element offsets in every kernel of the step (ghost fill, cell speeds,
the fused step's stores and its tensor map strides) must be 64-bit.  The
input is generated on the device by torch (a dam break with seeded noise);
40 windows of 8 x 8 cells, including the last rows and columns, are
recomputed by the oracle from the step's filled input, and total mass is
conserved by the walls.
"""
import numpy as np
import pytest

import oracle
import paper_1308_1464_gb300 as mc
from gpu_util import TOL, field_scales, problems, window_step

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1308_1464_gb300.state import DeviceState  # noqa: E402

W = mc.BC_WALL


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1308_1464_gb300 import _build
    _build.build()
    oracle.build()


def test_step_beyond_2_31_elements():
    n = 32768
    dx = 2.0 / n
    p, op = problems("swe", n, n, dx, dx, mc.F32, (W, W, W, W))
    with mc.Context(p) as ctx:
        lay = ctx.layout
        assert 2 * lay.ld_field > 2 ** 31 and lay.ld_field * 4 > 2 ** 32
        a, b = DeviceState(ctx).zero_(), DeviceState(ctx).zero_()
        P = a.padded()
        xi = int(lay.x_offset)
        gen = torch.Generator(device="cuda").manual_seed(1308)
        c = (torch.arange(n, device="cuda", dtype=torch.float32) + 0.5) * dx - 1.0
        for j in range(0, n, 4096):   # row blocks, to bound the temporaries
            r2 = c[j: j + 4096, None] ** 2 + c[None, :] ** 2
            h = torch.where(r2 < 0.25, 2.0, 1.0)
            h += 1e-3 * torch.rand(h.shape, device="cuda", generator=gen)
            P[0, 2 + j: 2 + j + 4096, xi: xi + n] = h
            P[1, 2 + j: 2 + j + 4096, xi: xi + n] = 0.01 * (torch.rand(h.shape, device="cuda", generator=gen) - 0.5)
            P[2, 2 + j: 2 + j + 4096, xi: xi + n] = 0.01 * (torch.rand(h.shape, device="cuda", generator=gen) - 0.5)
            del r2, h
        torch.cuda.synchronize()
        dt = 0.8 * dx / 5.0   # speeds are below |u| + sqrt(9.81 * 2.001) < 5
        smax = ctx.step(a.ptr, b.ptr, dt)
        assert 0.0 < smax * dt <= 0.8
        Pb = b.padded()
        x0 = xi - 2
        m0 = P[0, 2:-2, xi: xi + n].double().sum().item()
        m1 = Pb[0, 2:-2, xi: xi + n].double().sum().item()
        rng = np.random.default_rng(17)
        w = h = 8
        spots = [(0, 0), (n - w, 0), (0, n - h), (n - w, n - h), (n // 2 - 4, n - h), (n - w, n // 2)]
        spots += [(int(rng.integers(0, n - w)), int(rng.integers(0, n - h))) for _ in range(34)]
        wins = []
        for (i0, j0) in spots:
            fin = P[:, j0: j0 + h + 4, x0 + i0: x0 + i0 + w + 4].cpu().numpy().astype(np.float64)
            got = Pb[:, 2 + j0: 2 + j0 + h, xi + i0: xi + i0 + w].cpu().numpy().astype(np.float64)
            wins.append((i0, j0, fin, got))
    for (i0, j0, fin, got) in wins:
        # the window and its two ghost layers, placed at the origin of a
        # small ghosted array for window_step
        want = window_step(op, fin, dt, 0, 0, w, h)
        S = field_scales("swe", fin[:, 2:-2, 2:-2])
        err = max(np.abs(got[m] - want[m]).max() / S[m] for m in range(3))
        assert err <= TOL[mc.F32], (i0, j0, err)
    assert abs(m1 - m0) / m0 <= 1e-6
