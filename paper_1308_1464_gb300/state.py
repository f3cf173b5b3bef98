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


class PatchSet:
    """All patches of a batch in two device buffers (ping-pong), each patch in
    the library layout at a 256-byte aligned offset.  Marshalling only."""

    def __init__(self, proto, patches, device: str = "cuda"):
        """patches: list of (mx, my, dx, dy, interior (meqn, my, mx) array)."""
        from . import layout_of
        import copy
        self.proto = proto
        self.specs = []
        off = 0
        for (mx, my, dx, dy, q) in patches:
            p = copy.copy(proto)
            p.mx, p.my, p.dx, p.dy = int(mx), int(my), float(dx), float(dy)
            lay = layout_of(p)
            self.specs.append((p, lay, off))
            off += (int(lay.bytes) + 255) // 256 * 256
        self.nbytes = off
        es = int(self.specs[0][1].elem_bytes)
        self.np_dtype = np.float64 if es == 8 else np.float32
        host = np.zeros(off // es, dtype=self.np_dtype)
        for (p, lay, o), (_, _, _, _, q) in zip(self.specs, patches):
            v = self._view(host, p, lay, o)
            v[:, 2:-2, int(lay.x_offset): int(lay.x_offset) + p.mx] = q
        self._host0 = torch.from_numpy(host.view(np.uint8))
        self.buf_a = self._host0.to(device)
        self.buf_b = torch.zeros_like(self.buf_a)

    def reset(self) -> None:
        """Restore the initial state into buffer a."""
        self.buf_a.copy_(self._host0)
        torch.cuda.synchronize()

    @staticmethod
    def _view(flat, p, lay, off):
        es = flat.itemsize
        n = int(lay.meqn * lay.ld_field)
        return flat[off // es: off // es + n].reshape(int(lay.meqn), p.my + 4, int(lay.ld_x))

    def pointers(self):
        """(mx, my, dx, dy, qa, qb) per patch, for Batch()."""
        a, b = self.buf_a.data_ptr(), self.buf_b.data_ptr()
        return [(p.mx, p.my, p.dx, p.dy, a + o, b + o) for (p, lay, o) in self.specs]

    def interiors(self, in_b: bool):
        """Host copies of every patch's interior from buffer b (or a)."""
        torch.cuda.synchronize()
        flat = (self.buf_b if in_b else self.buf_a).cpu().numpy().view(self.np_dtype)
        out = []
        for (p, lay, o) in self.specs:
            v = self._view(flat, p, lay, o)
            out.append(v[:, 2:-2, int(lay.x_offset): int(lay.x_offset) + p.mx].copy())
        return out
