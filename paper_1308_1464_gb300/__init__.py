"""GB300-native wave-propagation library: thin Python binding of include/manyclaw.h.

The compute path lives in the CUDA library ``_lib/libmanyclaw.so`` (built by
``__graft_entry__.build()`` or ``python -m paper_1308_1464_gb300._build``);
this module only marshals arguments to its C ABI.  It never falls back to a
CPU implementation: if the library is missing, ``lib()`` raises.

Device buffers are passed as integer addresses (e.g. ``tensor.data_ptr()``)
and streams as integer handles (``torch.cuda.current_stream().cuda_stream``);
PyTorch is only used by callers for device memory and streams.
"""
from __future__ import annotations

import ctypes
import os
import re

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libmanyclaw.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "manyclaw.h")

MC_OK, MC_EINVAL, MC_ECUDA, MC_ENOMEM, MC_ECFL, MC_ENONPHYS, MC_ETIMEOUT, MC_ENOTSUP = (
    0, -1, -2, -3, -4, -5, -6, -7)
ACOUSTICS, SWE_ROE, EULER_ROE, ADVECTION, ACOUSTICS_VAR, EULER_GODUNOV = 1, 2, 3, 4, 5, 6
LIM_NONE, LIM_MINMOD, LIM_SUPERBEE, LIM_VANLEER, LIM_MC = 0, 1, 2, 3, 4
BC_PERIODIC, BC_EXTRAP, BC_WALL, BC_GIVEN = 0, 1, 2, 3
F32, F64 = 0, 1


class McError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{status_string(status)}: {message}")
        self.status = status


class Problem(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int32), ("dtype", ctypes.c_int32), ("mx", ctypes.c_int32),
                ("my", ctypes.c_int32), ("mbc", ctypes.c_int32), ("limiter", ctypes.c_int32),
                ("order", ctypes.c_int32), ("transverse", ctypes.c_int32), ("efix", ctypes.c_int32),
                ("bc", ctypes.c_int32 * 4), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("param", ctypes.c_double * 4)]

    @classmethod
    def make(cls, solver, mx, my, dx, dy, dtype=F32, limiter=LIM_MC, order=2, transverse=1,
             efix=1, bc=(BC_PERIODIC,) * 4, param=(1.0, 4.0, 0.0, 0.0)):
        p = cls()
        p.solver, p.dtype, p.mx, p.my, p.mbc = solver, dtype, mx, my, 2
        p.limiter, p.order, p.transverse, p.efix = limiter, order, transverse, efix
        for k in range(4):
            p.bc[k] = int(bc[k])
            p.param[k] = float(param[k]) if k < len(param) else 0.0
        p.dx, p.dy = float(dx), float(dy)
        return p

    @property
    def meqn(self) -> int:
        """Planes of a state array (conserved fields, then material planes)."""
        return {EULER_ROE: 4, EULER_GODUNOV: 4, ADVECTION: 1, ACOUSTICS_VAR: 5}.get(self.solver, 3)


class AmrPatch(ctypes.Structure):
    _fields_ = [("ci0", ctypes.c_int32), ("cj0", ctypes.c_int32), ("cw", ctypes.c_int32),
                ("ch", ctypes.c_int32), ("qa", ctypes.c_void_p), ("qb", ctypes.c_void_p)]


class Layout(ctypes.Structure):
    _fields_ = [("x_offset", ctypes.c_int64), ("ld_x", ctypes.c_int64),
                ("ld_field", ctypes.c_int64), ("elem_bytes", ctypes.c_int64),
                ("meqn", ctypes.c_int64), ("bytes", ctypes.c_int64)]


_lib = None
_VP = ctypes.c_void_p
_DP = ctypes.POINTER(ctypes.c_double)
_IP = ctypes.POINTER(ctypes.c_int)


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER(Problem)
        L.mc_status_string.restype = ctypes.c_char_p
        L.mc_status_string.argtypes = [ctypes.c_int]
        L.mc_last_error.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
        L.mc_layout_of.argtypes = [P, ctypes.POINTER(Layout)]
        L.mc_create.argtypes = [P, ctypes.POINTER(_VP)]
        L.mc_destroy.argtypes = [_VP]
        L.mc_set_tile_rows.argtypes = [_VP, ctypes.c_int]
        L.mc_set_seed_net.argtypes = [_VP, _VP]
        L.mc_amr_fine_problem.argtypes = [P, ctypes.c_int32, ctypes.POINTER(AmrPatch), P]
        L.mc_amr_create.argtypes = [P, ctypes.c_int32, ctypes.POINTER(AmrPatch), ctypes.c_int32,
                                    ctypes.POINTER(_VP)]
        L.mc_amr_destroy.argtypes = [_VP]
        L.mc_amr_set_reflux.argtypes = [_VP, ctypes.c_int32]
        L.mc_amr_advance.argtypes = [_VP, _VP, _VP, ctypes.c_int32, ctypes.c_double,
                                     ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32), _VP]
        L.mc_newton_stats.argtypes = [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.c_int32, _VP]
        L.mc_guard_stats.argtypes = [_VP, ctypes.POINTER(ctypes.c_int64), ctypes.c_int32, _VP]
        L.mc_upload.argtypes = [_VP, _VP, _VP, _VP]
        L.mc_repack.argtypes = [_VP, _VP, _VP, ctypes.c_int32, _VP]
        L.mc_download.argtypes = [_VP, _VP, _VP, _VP]
        L.mc_bc_fill.argtypes = [_VP, _VP, _VP]
        L.mc_bc_fill_dir.argtypes = [_VP, _VP, ctypes.c_int32, _VP]
        L.mc_halo_elems.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]
        L.mc_halo_pack.argtypes = [_VP, _VP, ctypes.c_int32, _VP, _VP]
        L.mc_halo_unpack.argtypes = [_VP, _VP, ctypes.c_int32, _VP, _VP]
        L.mc_step.argtypes = [_VP, _VP, _VP, ctypes.c_double, _DP, _VP]
        L.mc_block_begin.argtypes = [_VP, ctypes.c_double, ctypes.c_double, _VP]
        L.mc_block_pack.argtypes = [_VP, _VP, _VP, ctypes.c_int32, _VP, _VP]
        L.mc_block_unpack.argtypes = [_VP, _VP, ctypes.c_int32, _VP, _VP, _VP]
        L.mc_block_fill_dir.argtypes = [_VP, _VP, _VP, ctypes.c_int32, _VP]
        L.mc_block_sweep.argtypes = [_VP, _VP, _VP, _VP, _VP]
        L.mc_block_dt_rule.argtypes = [_VP, _VP, ctypes.c_double, ctypes.c_double, _VP]
        L.mc_block_end.argtypes = [_VP, _DP, _DP, _IP, _IP, _IP, _VP]
        L.mc_sweep.argtypes = [_VP, _VP, _VP, ctypes.c_double, _VP]
        L.mc_step_noalloc.argtypes = [P, _VP, _VP, ctypes.c_double, _DP, _VP]
        L.mc_peak_run.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int64, _VP, _DP, _VP]
        L.mc_max_cell_speed.argtypes = [_VP, _VP, _DP, _VP]
        L.mc_advance.argtypes = [_VP, _VP, _VP, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 _DP, _DP, _IP, _IP, _VP]
        L.mc_advance_host.argtypes = [_VP, _VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, _DP, _DP, _IP, _VP]
        L.mc_mlp_create.argtypes = [ctypes.POINTER(_VP)]
        L.mc_mlp_destroy.argtypes = [_VP]
        L.mc_mlp_set_params.argtypes = [_VP, _VP]
        L.mc_mlp_get_params.argtypes = [_VP, _VP]
        L.mc_mlp_features.argtypes = [ctypes.c_int64, ctypes.c_double] + [_VP] * 9 + [_VP]
        L.mc_mlp_forward.argtypes = [_VP, ctypes.c_int64, _VP, _VP, _VP]
        L.mc_mlp_grad.argtypes = [_VP, ctypes.c_int64, _VP, _VP, _VP, _VP, _VP]
        L.mc_mlp_train.argtypes = [_VP, ctypes.c_int64, _VP, _VP, ctypes.POINTER(TrainCfg),
                                   _VP, _VP]
        L.mc_batch_create.argtypes = [P, ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(_VP)]
        L.mc_batch_destroy.argtypes = [_VP]
        L.mc_batch_set_tile_rows.argtypes = [_VP, ctypes.c_void_p]
        L.mc_batch_inject_stall.argtypes = [_VP, ctypes.c_int32]
        for fn in (L.mc_batch_advance, L.mc_batch_advance_plain, L.mc_batch_advance_steps):
            fn.argtypes = [_VP, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p, _IP, _VP]
        L.mc_riemann_exact.argtypes = [ctypes.c_int64, ctypes.c_double] + [_VP] * 10 + [
            ctypes.c_int, _VP, ctypes.c_double, ctypes.c_int, _VP, _VP]
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().mc_status_string(int(status)).decode()


def last_error() -> str:
    buf = ctypes.create_string_buffer(512)
    lib().mc_last_error(buf, 512)
    return buf.value.decode()


def check(status: int) -> None:
    if status != MC_OK:
        raise McError(status, last_error())


def layout_of(p: Problem) -> Layout:
    lay = Layout()
    check(lib().mc_layout_of(ctypes.byref(p), ctypes.byref(lay)))
    return lay


class Context:
    """A problem bound to the current CUDA device (mc_create / mc_destroy)."""

    def __init__(self, problem: Problem):
        self.problem = problem
        self.layout = layout_of(problem)
        h = _VP()
        check(lib().mc_create(ctypes.byref(problem), ctypes.byref(h)))
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().mc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_tile_rows(self, rows: int) -> None:
        check(lib().mc_set_tile_rows(self._h, int(rows)))

    def set_seed_net(self, net) -> None:
        """Attach a SeedNet (or None) to the exact-solution Euler solver."""
        self._seed_net = net   # keep it alive while attached
        check(lib().mc_set_seed_net(self._h, net.handle if net is not None else None))

    # ---- device-side block stepping (mc_block_*)
    def block_begin(self, t: float, dt: float, stream: int = 0) -> None:
        check(lib().mc_block_begin(self._h, float(t), float(dt), _VP(stream)))

    def block_pack(self, qa: int, qb: int, side: int, buf: int, stream: int = 0) -> None:
        check(lib().mc_block_pack(self._h, _VP(qa), _VP(qb), int(side), _VP(buf), _VP(stream)))

    def block_unpack(self, buf: int, side: int, qa: int, qb: int, stream: int = 0) -> None:
        check(lib().mc_block_unpack(self._h, _VP(buf), int(side), _VP(qa), _VP(qb), _VP(stream)))

    def block_fill_dir(self, qa: int, qb: int, direction: int, stream: int = 0) -> None:
        check(lib().mc_block_fill_dir(self._h, _VP(qa), _VP(qb), int(direction), _VP(stream)))

    def block_sweep(self, qa: int, qb: int, smax_dev: int, stream: int = 0) -> None:
        check(lib().mc_block_sweep(self._h, _VP(qa), _VP(qb), _VP(smax_dev), _VP(stream)))

    def block_dt_rule(self, smax_dev: int, cfl_desired: float, cfl_max: float, stream: int = 0) -> None:
        check(lib().mc_block_dt_rule(self._h, _VP(smax_dev), float(cfl_desired), float(cfl_max),
                                     _VP(stream)))

    def block_end(self, stream: int = 0):
        """-> (t, dt, cur, naccepted, nrejected); synchronises."""
        t, dt = ctypes.c_double(), ctypes.c_double()
        cur, na, nr = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().mc_block_end(self._h, ctypes.byref(t), ctypes.byref(dt), ctypes.byref(cur),
                                 ctypes.byref(na), ctypes.byref(nr), _VP(stream)))
        return t.value, dt.value, cur.value, na.value, nr.value

    def guard_stats(self, reset: bool = True, stream: int = 0) -> int:
        """Interior edges the FP64 guard recomputed since the last reset."""
        n = ctypes.c_int64()
        check(lib().mc_guard_stats(self._h, ctypes.byref(n), int(reset), _VP(stream)))
        return n.value

    def newton_stats(self, reset: bool = True, stream: int = 0):
        """(Newton updates, normal solves) counted since the last reset."""
        u, n = ctypes.c_int64(), ctypes.c_int64()
        check(lib().mc_newton_stats(self._h, ctypes.byref(u), ctypes.byref(n), int(reset), _VP(stream)))
        return u.value, n.value

    def upload(self, host_dense_ptr: int, q_dev: int, stream: int = 0) -> None:
        check(lib().mc_upload(self._h, _VP(host_dense_ptr), _VP(q_dev), _VP(stream)))

    def download(self, q_dev: int, host_dense_ptr: int, stream: int = 0) -> None:
        check(lib().mc_download(self._h, _VP(q_dev), _VP(host_dense_ptr), _VP(stream)))

    def repack(self, src_dev: int, dst_dev: int, to_layout: bool, stream: int = 0) -> None:
        check(lib().mc_repack(self._h, _VP(src_dev), _VP(dst_dev), int(bool(to_layout)), _VP(stream)))

    def bc_fill(self, q_dev: int, stream: int = 0) -> None:
        check(lib().mc_bc_fill(self._h, _VP(q_dev), _VP(stream)))

    def bc_fill_dir(self, q_dev: int, direction: int, stream: int = 0) -> None:
        check(lib().mc_bc_fill_dir(self._h, _VP(q_dev), int(direction), _VP(stream)))

    def halo_elems(self, side: int) -> int:
        n = ctypes.c_int64(0)
        check(lib().mc_halo_elems(ctypes.byref(self.problem), int(side), ctypes.byref(n)))
        return n.value

    def halo_pack(self, q_dev: int, side: int, buf_dev: int, stream: int = 0) -> None:
        check(lib().mc_halo_pack(self._h, _VP(q_dev), int(side), _VP(buf_dev), _VP(stream)))

    def halo_unpack(self, buf_dev: int, side: int, q_dev: int, stream: int = 0) -> None:
        check(lib().mc_halo_unpack(self._h, _VP(buf_dev), int(side), _VP(q_dev), _VP(stream)))

    def step(self, q_in: int, q_out: int, dt: float, want_smax: bool = True, stream: int = 0):
        smax = ctypes.c_double(0.0)
        check(lib().mc_step(self._h, _VP(q_in), _VP(q_out), float(dt),
                            ctypes.byref(smax) if want_smax else None, _VP(stream)))
        return smax.value if want_smax else None

    def sweep(self, q_in: int, q_out: int, dt: float, stream: int = 0) -> None:
        check(lib().mc_sweep(self._h, _VP(q_in), _VP(q_out), float(dt), _VP(stream)))

    def max_cell_speed(self, q: int, stream: int = 0) -> float:
        s = ctypes.c_double(0.0)
        check(lib().mc_max_cell_speed(self._h, _VP(q), ctypes.byref(s), _VP(stream)))
        return s.value

    def advance(self, qa: int, qb: int, nsteps: int, cfl_desired: float, cfl_max: float,
                t: float, dt: float, stream: int = 0):
        """-> (t, dt, result_in_b, nrejected)"""
        tt, dd = ctypes.c_double(t), ctypes.c_double(dt)
        inb, nrej = ctypes.c_int(0), ctypes.c_int(0)
        check(lib().mc_advance(self._h, _VP(qa), _VP(qb), int(nsteps), float(cfl_desired),
                               float(cfl_max), ctypes.byref(tt), ctypes.byref(dd),
                               ctypes.byref(inb), ctypes.byref(nrej), _VP(stream)))
        return tt.value, dd.value, bool(inb.value), nrej.value

    def advance_host(self, host_q0: int, host_q: int, qa: int, qb: int, nsteps: int,
                     cfl_desired: float, cfl_max: float, t: float, dt: float, stream: int = 0):
        """-> (t, dt, nrejected)"""
        tt, dd, nrej = ctypes.c_double(t), ctypes.c_double(dt), ctypes.c_int(0)
        check(lib().mc_advance_host(self._h, _VP(host_q0), _VP(host_q), _VP(qa), _VP(qb),
                                    int(nsteps), float(cfl_desired), float(cfl_max),
                                    ctypes.byref(tt), ctypes.byref(dd), ctypes.byref(nrej),
                                    _VP(stream)))
        return tt.value, dd.value, nrej.value


def header_functions(path: str = HEADER) -> list[str]:
    """Names of the functions include/manyclaw.h declares."""
    with open(path) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(mc_[a-z0-9_]+)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


# ---------------------------------------------------------------- exact solver

SEED_ADAPTIVE, SEED_PV, SEED_TR, SEED_TS, SEED_PVTR, SEED_MLP = range(6)
NEWTON_MIXED = 16   # added to a seed mode: FP32 Newton stage, then FP64 updates
RS_OK, RS_VACUUM, RS_NOCONV, RS_FALLBACK = 0, 1, 2, 4
MLP_NWEIGHT = 16 * 64 + 64 + 64 * 64 + 64 + 64 + 1
MLP_NPARAM = MLP_NWEIGHT + 20


class TrainCfg(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int64), ("epochs", ctypes.c_int32), ("lr", ctypes.c_float),
                ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("fit_norm", ctypes.c_int32), ("clip", ctypes.c_float),
                ("lr_final", ctypes.c_float)]


class SeedNet:
    """Device-resident pressure-seed network (mc_mlp_*)."""

    def __init__(self):
        h = _VP()
        check(lib().mc_mlp_create(ctypes.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().mc_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params) -> None:
        """params: a host array of MLP_NPARAM values (held for the duration of
        the call), or the address of one."""
        if isinstance(params, int):
            check(lib().mc_mlp_set_params(self._h, _VP(params)))
            return
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        if a.size != MLP_NPARAM:
            raise ValueError(f"expected {MLP_NPARAM} parameters, got {a.size}")
        check(lib().mc_mlp_set_params(self._h, _VP(a.ctypes.data)))

    def get_params(self, host_ptr: int | None = None):
        """Copies the parameters to the address given, or returns a new array."""
        if host_ptr is not None:
            check(lib().mc_mlp_get_params(self._h, _VP(host_ptr)))
            return None
        import numpy as np
        a = np.empty(MLP_NPARAM, dtype=np.float32)
        check(lib().mc_mlp_get_params(self._h, _VP(a.ctypes.data)))
        return a

    def forward(self, n: int, features: int, out: int, stream: int = 0) -> None:
        check(lib().mc_mlp_forward(self._h, int(n), _VP(features), _VP(out), _VP(stream)))

    def grad(self, n: int, features: int, target: int, grads: int, loss: int, stream: int = 0):
        check(lib().mc_mlp_grad(self._h, int(n), _VP(features), _VP(target), _VP(grads),
                                _VP(loss), _VP(stream)))

    def train(self, n: int, features: int, target: int, batch: int = 8192, epochs: int = 10,
              lr: float = 2e-3, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8,
              seed: int = 1, fit_norm: bool = True, loss_out: int = 0, stream: int = 0,
              clip: float = 2.0, lr_final: float | None = None) -> None:
        cfg = TrainCfg(int(batch), int(epochs), lr, beta1, beta2, eps, int(seed), int(fit_norm),
                       float(clip), float(lr if lr_final is None else lr_final))
        check(lib().mc_mlp_train(self._h, int(n), _VP(features), _VP(target), ctypes.byref(cfg),
                                 _VP(loss_out) if loss_out else None, _VP(stream)))


def mlp_features(n: int, gamma: float, states, p_star: int, features: int, target: int,
                 stream: int = 0) -> None:
    """states: six device pointers (rho_l, u_l, p_l, rho_r, u_r, p_r)."""
    check(lib().mc_mlp_features(int(n), float(gamma), *[_VP(s) for s in states],
                                _VP(p_star) if p_star else None, _VP(features),
                                _VP(target) if target else None, _VP(stream)))


def riemann_exact(n: int, gamma: float, states, p_star: int, u_star: int, iters: int, flags: int,
                  seed_mode: int = SEED_ADAPTIVE, net: "SeedNet | None" = None, tol: float = 1e-8,
                  max_iter: int = 30, stats: int = 0, stream: int = 0) -> None:
    """Exact Euler Riemann solves of n interfaces (device SoA pointers)."""
    check(lib().mc_riemann_exact(int(n), float(gamma), *[_VP(s) for s in states], _VP(p_star),
                                 _VP(u_star), _VP(iters) if iters else None,
                                 _VP(flags) if flags else None, int(seed_mode),
                                 net.handle if net is not None else None, float(tol),
                                 int(max_iter), _VP(stats) if stats else None, _VP(stream)))


def step_noalloc(problem: Problem, q_in: int, q_out: int, dt: float, want_smax: bool = True,
                 stream: int = 0):
    """mc_step_noalloc: one step without a context, allocating no device memory."""
    smax = ctypes.c_double(0.0)
    check(lib().mc_step_noalloc(ctypes.byref(problem), _VP(q_in), _VP(q_out), float(dt),
                                ctypes.byref(smax) if want_smax else None, _VP(stream)))
    return smax.value if want_smax else None


PEAK_FFMA, PEAK_FFMA2, PEAK_DFMA, PEAK_RSQRT, PEAK_RCP, PEAK_IADD, PEAK_ISSUE = range(7)


def peak_run(kind: int, blocks_per_sm: int, iters: int, sink: int, stream: int = 0) -> float:
    """mc_peak_run: launch one throughput microbenchmark; returns its operation count."""
    ops = ctypes.c_double(0.0)
    check(lib().mc_peak_run(int(kind), int(blocks_per_sm), int(iters), _VP(sink), ctypes.byref(ops),
                            _VP(stream)))
    return ops.value


# ---------------------------------------------------------------- batched patches

class PatchC(ctypes.Structure):
    _fields_ = [("mx", ctypes.c_int32), ("my", ctypes.c_int32), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("qa", ctypes.c_void_p), ("qb", ctypes.c_void_p)]


class Batch:
    """Uneven wall-bounded patches advanced together (mc_batch_*).  patches:
    sequence of (mx, my, dx, dy, qa_ptr, qb_ptr)."""

    def __init__(self, proto: Problem, patches):
        L = lib()
        arr = (PatchC * len(patches))(*[PatchC(int(mx), int(my), float(dx), float(dy), int(qa),
                                               int(qb)) for (mx, my, dx, dy, qa, qb) in patches])
        h = _VP()
        check(L.mc_batch_create(ctypes.byref(proto), arr, len(patches), ctypes.byref(h)))
        self._h = h
        self.npatch = len(patches)

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().mc_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tile_rows(self, rows) -> None:
        arr = (ctypes.c_int32 * self.npatch)(*[int(r) for r in rows])
        check(lib().mc_batch_set_tile_rows(self._h, arr))

    def _run(self, fn, nsteps, cfl, want_t, stream):
        t = (ctypes.c_double * self.npatch)() if want_t else None
        inb = ctypes.c_int(0)
        check(fn(self._h, int(nsteps), float(cfl), t, ctypes.byref(inb), _VP(stream)))
        return (list(t) if want_t else None), bool(inb.value)

    def advance(self, nsteps: int, cfl: float = 0.9, want_t: bool = False, stream: int = 0):
        """One persistent launch in a graph -> (t per patch or None, result_in_b)."""
        return self._run(lib().mc_batch_advance, nsteps, cfl, want_t, stream)

    def inject_stall(self, patch: int) -> None:
        """Test hook: the next advance's waits for this patch run out (MC_ETIMEOUT)."""
        check(lib().mc_batch_inject_stall(self._h, int(patch)))

    def advance_steps(self, nsteps: int, cfl: float = 0.9, want_t: bool = False, stream: int = 0):
        """One launch per step over all patches, in a graph -> (t per patch or None, result_in_b)."""
        return self._run(lib().mc_batch_advance_steps, nsteps, cfl, want_t, stream)

    def advance_plain(self, nsteps: int, cfl: float = 0.9, want_t: bool = False, stream: int = 0):
        """One launch per patch per step -> (t per patch or None, result_in_b)."""
        return self._run(lib().mc_batch_advance_plain, nsteps, cfl, want_t, stream)


def amr_fine_problem(coarse: Problem, ratio: int, ci0: int, cj0: int, cw: int, ch: int) -> Problem:
    """The problem of a fine patch over coarse cells [ci0, ci0+cw) x [cj0, cj0+ch)."""
    out = Problem()
    patch = AmrPatch(ci0, cj0, cw, ch, None, None)
    check(lib().mc_amr_fine_problem(ctypes.byref(coarse), int(ratio), ctypes.byref(patch),
                                    ctypes.byref(out)))
    return out


class Amr:
    """Refined patches on a coarse grid (mc_amr_*).  patches: list of
    (ci0, cj0, cw, ch, qa_ptr, qb_ptr)."""

    def __init__(self, coarse: Problem, ratio: int, patches, reflux: bool = False):
        arr = (AmrPatch * max(1, len(patches)))(*[AmrPatch(*pt) for pt in patches])
        h = _VP()
        check(lib().mc_amr_create(ctypes.byref(coarse), int(ratio), arr, len(patches), ctypes.byref(h)))
        self._h = h
        self.set_reflux(reflux)

    def set_reflux(self, on: bool) -> None:
        """Flux correction of the coarse cells outside the patches."""
        check(lib().mc_amr_set_reflux(self._h, int(bool(on))))

    def close(self) -> None:
        if getattr(self, "_h", None):
            lib().mc_amr_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def advance(self, qc_a: int, qc_b: int, nsteps: int, dt: float, stream: int = 0):
        """-> (coarse result in b, fine result in b)."""
        cb, fb = ctypes.c_int32(), ctypes.c_int32()
        check(lib().mc_amr_advance(self._h, _VP(qc_a), _VP(qc_b), int(nsteps), float(dt),
                                   ctypes.byref(cb), ctypes.byref(fb), _VP(stream)))
        return bool(cb.value), bool(fb.value)
