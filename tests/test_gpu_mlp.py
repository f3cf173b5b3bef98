"""GPU seed network: forward and gradient parity with the oracle's BF16
precision model, and what training buys the exact solver.

The gradient check uses inputs that are exact in BF16 and a network whose
standardisation is the identity, so both sides round the same operands; the
remaining differences are FP32 versus FP64 accumulation (tolerance 1e-3
relative to each tensor's scale)."""
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


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1308_1464_gb300 import _build
    _build.build()
    oracle.build()


def bf16_exact(a):
    """Round float values to BF16 (to nearest, ties to even) in numpy."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return u.view(np.float32).astype(np.float64)


def random_params(rng):
    p = np.zeros(mc.MLP_NPARAM, dtype=np.float32)
    W1 = rng.normal(scale=0.4, size=(16, 64))
    W1[10:] = 0.0
    p[0:1024] = W1.ravel()
    p[1024:1088] = rng.normal(scale=0.1, size=64)
    p[1088:5184] = rng.normal(scale=0.15, size=64 * 64)
    p[5184:5248] = rng.normal(scale=0.1, size=64)
    p[5248:5312] = rng.normal(scale=0.2, size=64)
    p[5312] = 0.05
    p[mc.MLP_NWEIGHT + 10:] = 1.0      # mu = 0, sigma = 1
    return p


def unpack(p):
    p = p.astype(np.float64)
    return (p[0:1024].reshape(16, 64), p[1024:1088], p[1088:5184].reshape(64, 64),
            p[5184:5248], p[5248:5312], p[5312:5313])


def test_forward_and_gradient_match_oracle():
    rng = np.random.default_rng(7)
    params = random_params(rng)
    net = mc.SeedNet()
    net.set_params(params.ctypes.data)
    n = 1000                                   # 62.5 chunks of 16 rows: ragged tail
    X10 = bf16_exact(rng.normal(size=(n, 10)))
    y = rng.normal(size=n)
    Xd = torch.from_numpy(X10.astype(np.float32)).cuda()
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    net.forward(n, Xd.data_ptr(), out.data_ptr())
    grads = torch.empty(mc.MLP_NWEIGHT, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    net.grad(n, Xd.data_ptr(), yd.data_ptr(), grads.data_ptr(), loss.data_ptr())
    torch.cuda.synchronize()
    X = np.zeros((n, 16))
    X[:, :10] = X10
    W = unpack(params)
    y32 = y.astype(np.float32).astype(np.float64)
    out_ref = oracle.mlp_forward(X, *W, bf16=True)
    o = out.cpu().numpy()
    assert np.abs(o - out_ref).max() <= 1e-3 * np.abs(out_ref).max()
    loss_ref, g_ref = oracle.mlp_backward(X, y32, *W, bf16=True)
    assert float(loss.cpu()) == pytest.approx(loss_ref, rel=1e-3)
    g = grads.cpu().numpy().astype(np.float64)
    pieces = [("W1", 0, 1024), ("b1", 1024, 1088), ("W2", 1088, 5184), ("b2", 5184, 5248),
              ("W3", 5248, 5312), ("b3", 5312, 5313)]
    for name, a, b in pieces:
        ref = g_ref[name].ravel()
        got = g[a:b]
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 1e-3 * scale, (name, np.abs(got - ref).max(), scale)


def oracle_training_set(n, seed, offset):
    """Interfaces and their oracle star pressures (vacuum rows dropped)."""
    st = [a.astype(np.float32) for a in workloads.riemann_states(n, seed=seed, offset=offset)]
    ps, us, it, fl = oracle.exact_batch(GAMMA, *[a.astype(np.float64) for a in st], tol=1e-12)
    keep = fl == 0
    return [a[keep] for a in st], ps[keep]


def test_training_reduces_newton_iterations():
    """Trained on oracle star states, the network's seed needs fewer Newton
    updates than the plain adaptive seed on held-out interfaces, and the
    solver still returns the same p*."""
    st, ps = oracle_training_set(1 << 16, seed=11, offset=0)
    n = st[0].size
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in st]
    psd = torch.from_numpy(ps.astype(np.float32)).cuda()
    feat = torch.empty((n, 10), dtype=torch.float32, device="cuda")
    tgt = torch.empty(n, dtype=torch.float32, device="cuda")
    mc.mlp_features(n, GAMMA, [d.data_ptr() for d in dev], psd.data_ptr(), feat.data_ptr(),
                    tgt.data_ptr())
    net = mc.SeedNet()
    params = np.zeros(mc.MLP_NPARAM, dtype=np.float32)
    rng = np.random.default_rng(0)
    params[:mc.MLP_NWEIGHT] = random_params(rng)[:mc.MLP_NWEIGHT] * 0.5
    params[mc.MLP_NWEIGHT + 10:] = 1.0
    net.set_params(params.ctypes.data)
    epochs = 25
    losses = np.zeros(epochs, dtype=np.float32)
    net.train(n, feat.data_ptr(), tgt.data_ptr(), batch=4096, epochs=epochs, lr=3e-3, seed=5,
              loss_out=losses.ctypes.data)
    assert losses[-1] < 0.2 * losses[0], losses

    # held-out interfaces
    test_st = [a.astype(np.float32) for a in workloads.riemann_states(1 << 15, seed=11,
                                                                        offset=1 << 20)]
    from test_gpu_exact import gpu_solve
    ps_m, _, it_m, fl_m, stats_m = gpu_solve(test_st, mc.SEED_MLP, net)
    ps_p, _, it_p, fl_p, stats_p = gpu_solve(test_st, mc.SEED_ADAPTIVE)
    ok = (fl_p & mc.RS_VACUUM) == 0
    np.testing.assert_allclose(ps_m[ok], ps_p[ok], rtol=1.2e-7, atol=0)
    mean_m, mean_p = it_m[ok].mean(), it_p[ok].mean()
    fallback = ((fl_m & mc.RS_FALLBACK) != 0)[ok].mean()
    print(f"mean Newton updates: learned {mean_m:.3f}, plain {mean_p:.3f}, fallback {fallback:.4f}")
    assert mean_m < mean_p
    assert fallback < 0.01


def test_params_round_trip():
    """set_params copies every value (the first ones included) from an array
    it holds for the whole call, temporaries too; get_params returns them."""
    from paper_1308_1464_gb300.seednet import initial_params
    net = mc.SeedNet()
    for seed in range(4):
        net.set_params(initial_params(mc, seed=seed))      # a temporary array
        np.testing.assert_array_equal(net.get_params(), initial_params(mc, seed=seed))
    with pytest.raises(ValueError):
        net.set_params(np.zeros(10, dtype=np.float32))
    net.close()


def test_training_is_deterministic():
    """Two trainings from the same initial parameters, data and seed give
    bitwise identical parameters and losses: the gradients are summed in a
    fixed order (per warp, per CTA, then CTA by CTA), with no float atomics,
    and so are the feature moments of the standardisation."""
    st, ps = oracle_training_set(1 << 14, seed=13, offset=0)
    n = st[0].size
    dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in st]
    psd = torch.from_numpy(ps.astype(np.float32)).cuda()
    feat = torch.empty((n, 10), dtype=torch.float32, device="cuda")
    tgt = torch.empty(n, dtype=torch.float32, device="cuda")
    mc.mlp_features(n, GAMMA, [d.data_ptr() for d in dev], psd.data_ptr(), feat.data_ptr(),
                    tgt.data_ptr())
    rng = np.random.default_rng(3)
    params = np.zeros(mc.MLP_NPARAM, dtype=np.float32)
    params[:mc.MLP_NWEIGHT] = random_params(rng)[:mc.MLP_NWEIGHT] * 0.5
    params[mc.MLP_NWEIGHT + 10:] = 1.0
    runs = []
    for _ in range(2):
        net = mc.SeedNet()
        net.set_params(params.ctypes.data)
        losses = np.zeros(4, dtype=np.float32)
        net.train(n, feat.data_ptr(), tgt.data_ptr(), batch=2048, epochs=4, lr=3e-3, seed=9,
                  fit_norm=True, loss_out=losses.ctypes.data)
        runs.append((net.get_params().copy(), losses.copy()))
        net.close()
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
