"""Device state buffers in the library layout, held in torch tensors.

Marshalling only: allocation (torch), host<->device copies through the C ABI
(mc_upload / mc_download), and views of the padded array.  No arithmetic of
the method happens here.
"""
from __future__ import annotations

import numpy as np
import torch

from . import Context


class DeviceState:
    """One state array (ghost cells included) of a context's problem."""

    def __init__(self, ctx: Context, device: str = "cuda"):
        self.ctx = ctx
        lay = ctx.layout
        self.buf = torch.empty(int(lay.bytes), dtype=torch.uint8, device=device)
        self.np_dtype = np.float64 if lay.elem_bytes == 8 else np.float32
        self.t_dtype = torch.float64 if lay.elem_bytes == 8 else torch.float32

    @property
    def ptr(self) -> int:
        return self.buf.data_ptr()

    def zero_(self) -> "DeviceState":
        self.buf.zero_()
        return self

    def upload(self, interior: np.ndarray, stream: int = 0) -> "DeviceState":
        p = self.ctx.problem
        a = np.ascontiguousarray(interior, dtype=self.np_dtype)
        assert a.shape == (p.meqn, p.my, p.mx), (a.shape, (p.meqn, p.my, p.mx))
        self.ctx.upload(a.ctypes.data, self.ptr, stream)
        torch.cuda.synchronize()
        return self

    def download(self, stream: int = 0) -> np.ndarray:
        p = self.ctx.problem
        out = np.empty((p.meqn, p.my, p.mx), dtype=self.np_dtype)
        torch.cuda.synchronize()
        self.ctx.download(self.ptr, out.ctypes.data, stream)
        torch.cuda.synchronize()
        return out

    def padded(self) -> torch.Tensor:
        """(meqn, my + 4, ld_x) view of the device array."""
        p, lay = self.ctx.problem, self.ctx.layout
        return self.buf.view(self.t_dtype)[: lay.meqn * lay.ld_field].view(
            int(lay.meqn), p.my + 4, int(lay.ld_x))

    def with_ghosts(self) -> np.ndarray:
        """Host copy (meqn, my + 4, mx + 4) including the ghost layers."""
        p, lay = self.ctx.problem, self.ctx.layout
        x0 = int(lay.x_offset) - 2
        torch.cuda.synchronize()
        return self.padded()[:, :, x0: x0 + p.mx + 4].cpu().numpy()
