"""Pins of the oracle's seed network (CPU only).

* FP64 back-propagation equals central finite differences of the loss;
* the FP64 forward pass equals a numpy evaluation of the same layers;
* bfloat16 rounding (round to nearest, ties to even, 8 significant bits)
  reproduces hand-computed values;
* the feature map is consistent with its definitions (c = sqrt(gamma p/rho)).
"""
import math

import numpy as np
import pytest

from paper_1308_1464_gb300 import workloads

GAMMA = 1.4


def random_net(rng, scale=0.3):
    return {"W1": rng.normal(size=(16, 64)) * scale, "b1": rng.normal(size=64) * 0.1,
            "W2": rng.normal(size=(64, 64)) * scale / 4, "b2": rng.normal(size=64) * 0.1,
            "W3": rng.normal(size=64) * scale / 4, "b3": rng.normal(size=1) * 0.1}


def net_args(net):
    return [net[k] for k in ("W1", "b1", "W2", "b2", "W3", "b3")]


def test_forward_matches_numpy(oracle_mod):
    rng = np.random.default_rng(0)
    net = random_net(rng)
    X = np.zeros((9, 16))
    X[:, :10] = rng.normal(size=(9, 10))
    out = oracle_mod.mlp_forward(X, *net_args(net))
    h1 = np.maximum(X @ net["W1"] + net["b1"], 0)
    h2 = np.maximum(h1 @ net["W2"] + net["b2"], 0)
    np.testing.assert_allclose(out, h2 @ net["W3"] + net["b3"][0], rtol=1e-13, atol=1e-13)


def test_backward_matches_finite_differences(oracle_mod):
    rng = np.random.default_rng(1)
    net = random_net(rng)
    X = np.zeros((7, 16))
    X[:, :10] = rng.normal(size=(7, 10))
    y = rng.normal(size=7)
    loss, grads = oracle_mod.mlp_backward(X, y, *net_args(net))

    def L(n):
        o = oracle_mod.mlp_forward(X, *net_args(n))
        return np.mean((o - y) ** 2)

    assert loss == pytest.approx(L(net), rel=1e-13)
    h = 1e-6
    for key in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = net[key].reshape(-1)
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for k in idx:
            if key == "W1" and (k // 64) >= 10:
                continue  # padded input rows: zero input, zero gradient
            orig = flat[k]
            flat[k] = orig + h
            lp = L(net)
            flat[k] = orig - h
            lm = L(net)
            flat[k] = orig
            fd = (lp - lm) / (2 * h)
            g = grads[key].reshape(-1)[k]
            assert g == pytest.approx(fd, rel=1e-6, abs=1e-9), (key, k, g, fd)


@pytest.mark.parametrize("x,expected", [
    (1.0, 1.0),
    (1.0 + 2.0 ** -8, 1.0),                        # tie -> even (1.0)
    (1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -6),        # tie -> even (mantissa 2)
    (1.0 + 2.0 ** -8 + 2.0 ** -20, 1.0 + 2.0 ** -7),
    (-1.0 - 2.0 ** -8 - 2.0 ** -20, -1.0 - 2.0 ** -7),
    (3.14159, 3.140625),
    (0.0, 0.0),
])
def test_bf16_rounding(oracle_mod, x, expected):
    assert oracle_mod.round_bf16(x) == expected


def test_features(oracle_mod):
    st = [a[:5] for a in workloads.riemann_states(5, seed=2)]
    F = oracle_mod.mlp_features(GAMMA, *st)
    rl, ul, pl, rr, ur, pr = st
    np.testing.assert_allclose(F[:, 0], np.log(rl))
    np.testing.assert_allclose(F[:, 3], np.log(pr))
    cl = np.sqrt(GAMMA * pl / rl)
    cr = np.sqrt(GAMMA * pr / rr)
    np.testing.assert_allclose(F[:, 4], np.log(cl), rtol=1e-14)
    np.testing.assert_allclose(F[:, 6], ur - ul)
    np.testing.assert_allclose(F[:, 7], (ur - ul) / (cl + cr), rtol=1e-14)
    for k in range(5):
        ptr = oracle_mod.seed(oracle_mod.SEED_TR, GAMMA, *[a[k] for a in st])
        assert F[k, 8] == pytest.approx(math.log(ptr), rel=1e-14)
