"""Training of the pressure-seed network on the GPU (marshalling only).

The 10-64-64-1 network proposes ln(p*/p_TR) for an exact Euler Riemann
problem.  Its training data are seeded synthetic interfaces (workloads.py)
whose star pressures come from the library's exact solver run to 1e-12;
features, targets and the training itself (fused forward/backward on the
tensor cores, Adam) are the library's C-ABI calls.  Every step of the
arithmetic runs in the CUDA library; this module only allocates and calls.
"""
from __future__ import annotations

import time

import numpy as np


def initial_params(mc, seed: int = 0) -> np.ndarray:
    """Random initial parameters (layer scales 0.2 / 0.1 / 0.1, zero biases,
    identity standardisation until training sets it)."""
    rng = np.random.default_rng(seed)
    params = np.zeros(mc.MLP_NPARAM, dtype=np.float32)
    params[0:1024] = (rng.normal(size=(16, 64)) * 0.2 * (np.arange(16) < 10)[:, None]).ravel()
    params[1088:5184] = rng.normal(size=4096) * 0.1
    params[5248:5312] = rng.normal(size=64) * 0.1
    params[mc.MLP_NWEIGHT + 10:] = 1.0
    return params


def train_seed_net(ntrain: int = 1 << 22, epochs: int = 12, gamma: float = 1.4, offset: int = 1 << 26,
                   batch: int = 16384, lr: float = 2e-3, seed: int = 3, clip: float = 2.0,
                   lr_final: float = 4e-5):
    """-> (SeedNet, per-epoch losses, training seconds).  Adam with each
    step's gradient norm clipped to `clip` times its running mean and the
    learning rate decayed from lr to lr_final (cosine)."""
    import torch
    import paper_1308_1464_gb300 as mc
    from paper_1308_1464_gb300 import workloads

    states = [torch.from_numpy(a.astype(np.float32)).cuda()
              for a in workloads.riemann_states(ntrain, seed=1308, offset=offset)]
    ptrs = [s.data_ptr() for s in states]
    p_star = torch.empty(ntrain, dtype=torch.float32, device="cuda")
    u_star = torch.empty_like(p_star)
    iters = torch.empty(ntrain, dtype=torch.uint8, device="cuda")
    flags = torch.empty_like(iters)
    mc.riemann_exact(ntrain, gamma, ptrs, p_star.data_ptr(), u_star.data_ptr(), iters.data_ptr(),
                     flags.data_ptr(), mc.SEED_ADAPTIVE, None, 1e-12, 30, None)
    feat = torch.empty((ntrain, 10), dtype=torch.float32, device="cuda")
    tgt = torch.empty(ntrain, dtype=torch.float32, device="cuda")
    mc.mlp_features(ntrain, gamma, ptrs, p_star.data_ptr(), feat.data_ptr(), tgt.data_ptr())
    net = mc.SeedNet()
    net.set_params(initial_params(mc))
    losses = np.zeros(epochs, dtype=np.float32)
    t0 = time.perf_counter()
    net.train(ntrain, feat.data_ptr(), tgt.data_ptr(), batch=batch, epochs=epochs, lr=lr, seed=seed,
              loss_out=losses.ctypes.data, clip=clip, lr_final=lr_final)
    torch.cuda.synchronize()
    return net, losses, time.perf_counter() - t0
