"""FP64 CPU oracle of the wave-propagation method (plain C, loaded by ctypes).

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
restatement of the method that the CUDA library is checked against.  Only the
test-suite, the smoke check and the benchmark's CPU-baseline leg may import
it; the product library never does, and nothing here imports the product.

The paper (arXiv 1308.1464) describes the Riemann and limiter kernels in words
(§1.1, §1.2, Table 1, §2) and names Clawpack for the mathematics, so the
formulas are restated from LeVeque (2002) and Toro (exact Euler solver); each C
file cites the sections it follows.

Arrays are numpy float64, planar ``q[m, j, i]`` with ``mbc`` ghost layers on
every side: shape ``(meqn, my + 2*mbc, mx + 2*mbc)``.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["rp.c", "step.c", "exact.c", "mlp.c", "amr.c"]
_LIBDIR = os.path.join(_HERE, "_lib")

ACOUSTICS, SWE, EULER, ADVECTION, ACOUSTICS_VAR, EULER_GODUNOV = 1, 2, 3, 4, 5, 6
LIM_NONE, LIM_MINMOD, LIM_SUPERBEE, LIM_VANLEER, LIM_MC = 0, 1, 2, 3, 4
BC_PERIODIC, BC_EXTRAP, BC_WALL, BC_GIVEN = 0, 1, 2, 3
SEED_ADAPTIVE, SEED_PV, SEED_TR, SEED_TS, SEED_PVTR, SEED_GIVEN = range(6)
RS_OK, RS_VACUUM, RS_NOCONV, RS_FALLBACK = 0, 1, 2, 4
NIN, KIN, NH = 10, 16, 64


def _source_hash() -> str:
    h = hashlib.sha1()
    for name in _SOURCES + ["mcref.h"]:
        with open(os.path.join(_HERE, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_lib/ (gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    out = os.path.join(_LIBDIR, f"libmcref_{_source_hash()}.so")
    if os.path.exists(out) and not force:
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-o", tmp] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


class _Problem(ctypes.Structure):
    _fields_ = [("solver", ctypes.c_int), ("mx", ctypes.c_int), ("my", ctypes.c_int),
                ("mbc", ctypes.c_int), ("dx", ctypes.c_double), ("dy", ctypes.c_double),
                ("limiter", ctypes.c_int), ("order", ctypes.c_int),
                ("transverse", ctypes.c_int), ("efix", ctypes.c_int),
                ("bc", ctypes.c_int * 4), ("param", ctypes.c_double * 4)]


@dataclass
class Problem:
    solver: int
    mx: int
    my: int
    dx: float
    dy: float
    limiter: int = LIM_MC
    order: int = 2
    transverse: int = 1
    efix: int = 1
    bc: tuple = (BC_PERIODIC,) * 4
    param: tuple = (1.0, 4.0, 0.0, 0.0)
    mbc: int = 2
    _c: _Problem = field(default=None, repr=False, compare=False)

    @property
    def meqn(self) -> int:
        return {EULER: 4, EULER_GODUNOV: 4, ADVECTION: 1}.get(self.solver, 3)

    @property
    def nplane(self) -> int:
        """Planes of a state array: the conserved fields, then (variable-
        coefficient acoustics) the density and sound speed of each cell."""
        return self.meqn + (2 if self.solver == ACOUSTICS_VAR else 0)

    @property
    def mwaves(self) -> int:
        return {ACOUSTICS: 2, ACOUSTICS_VAR: 2, ADVECTION: 1}.get(self.solver, 3)

    @property
    def shape(self) -> tuple:
        return (self.nplane, self.my + 2 * self.mbc, self.mx + 2 * self.mbc)

    def c(self) -> _Problem:
        s = _Problem()
        s.solver, s.mx, s.my, s.mbc = self.solver, self.mx, self.my, self.mbc
        s.dx, s.dy = self.dx, self.dy
        s.limiter, s.order, s.transverse, s.efix = self.limiter, self.order, self.transverse, self.efix
        for k in range(4):
            s.bc[k] = int(self.bc[k])
            s.param[k] = float(self.param[k]) if k < len(self.param) else 0.0
        return s


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER(_Problem)
        L.mcref_rpn2.argtypes = [P, ctypes.c_int, _D, _D, _D, _D, _D, _D]
        L.mcref_rpt2.argtypes = [P, ctypes.c_int, _D, _D, _D, _D, _D]
        L.mcref_rpt2_var.argtypes = [P, ctypes.c_int, _D, _D, _D, _D, _D, _D]
        L.mcref_exact_sample.argtypes = [ctypes.c_double] * 9 + [_D, _D, _D]
        L.mcref_exact_sample.restype = None
        L.mcref_flux.argtypes = [P, ctypes.c_int, _D, _D]
        L.mcref_flux.restype = None
        L.mcref_philim.argtypes = [ctypes.c_int, ctypes.c_double]
        L.mcref_philim.restype = ctypes.c_double
        L.mcref_bc_fill.argtypes = [P, _D]
        L.mcref_bc_fill.restype = None
        L.mcref_step.argtypes = [P, _D, _D, ctypes.c_double, _D, ctypes.c_int]
        L.mcref_max_cell_speed.argtypes = [P, _D]
        L.mcref_max_cell_speed.restype = ctypes.c_double
        L.mcref_advance.argtypes = [P, _D, _D, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                    _D, _D, ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_int), ctypes.c_int]
        dd = [ctypes.c_double] * 7
        L.mcref_seed.argtypes = [ctypes.c_int] + dd
        L.mcref_seed.restype = ctypes.c_double
        L.mcref_pressure_function.argtypes = dd + [ctypes.c_double, _D, _D]
        L.mcref_pressure_function.restype = None
        L.mcref_exact_riemann.argtypes = dd + [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_int, _D, _D, ctypes.POINTER(ctypes.c_int)]
        L.mcref_exact_bisect.argtypes = dd + [_D, _D]
        L.mcref_exact_batch.argtypes = [ctypes.c_int64, ctypes.c_double] + [_D] * 6 + [
            ctypes.c_int, _D, ctypes.c_double, ctypes.c_int, _D, _D, _I32, _I32, ctypes.c_int]
        L.mcref_exact_batch.restype = None
        L.mcref_mlp_features.argtypes = dd + [_D]
        L.mcref_mlp_features.restype = None
        L.mcref_mlp_forward.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D, _D, _D,
                                        ctypes.c_int, _D, _D, _D]
        L.mcref_mlp_forward.restype = None
        L.mcref_mlp_backward.argtypes = [ctypes.c_int64, _D, _D, _D, _D, _D, _D, _D, _D,
                                         ctypes.c_int] + [_D] * 6
        L.mcref_mlp_backward.restype = ctypes.c_double
        L.mcref_round_bf16.argtypes = [ctypes.c_double]
        L.mcref_round_bf16.restype = ctypes.c_double
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- pointwise

def rpn2(prob: Problem, direction: int, ql, qr):
    """Normal Riemann solve across one edge -> (waves[mw, meqn], s[mw], amdq, apdq, flags)."""
    ql, qr = _f64(ql), _f64(qr)
    wave = np.zeros((prob.mwaves, prob.meqn))
    s = np.zeros(prob.mwaves)
    amdq = np.zeros(prob.meqn)
    apdq = np.zeros(prob.meqn)
    flags = lib().mcref_rpn2(ctypes.byref(prob.c()), direction, _p(ql), _p(qr), _p(wave), _p(s),
                             _p(amdq), _p(apdq))
    return wave, s, amdq, apdq, flags


def rpt2(prob: Problem, direction: int, ql, qr, asdq):
    ql, qr, asdq = _f64(ql), _f64(qr), _f64(asdq)
    bm = np.zeros(prob.meqn)
    bp = np.zeros(prob.meqn)
    lib().mcref_rpt2(ctypes.byref(prob.c()), direction, _p(ql), _p(qr), _p(asdq), _p(bm), _p(bp))
    return bm, bp


def rpt2_var(prob: Problem, direction: int, qlo, qc, qhi, asdq):
    """Variable-coefficient acoustics: split asdq entering cell qc between its
    neighbours qlo and qhi across the other direction -> (bm, bp)."""
    qlo, qc, qhi, asdq = _f64(qlo), _f64(qc), _f64(qhi), _f64(asdq)
    bm = np.zeros(prob.meqn)
    bp = np.zeros(prob.meqn)
    lib().mcref_rpt2_var(ctypes.byref(prob.c()), direction, _p(qlo), _p(qc), _p(qhi), _p(asdq),
                         _p(bm), _p(bp))
    return bm, bp


class _AmrPatch(ctypes.Structure):
    _fields_ = [("ci0", ctypes.c_int), ("cj0", ctypes.c_int), ("cw", ctypes.c_int), ("ch", ctypes.c_int)]


def _amr_lib():
    L = lib()
    if not getattr(L, "_amr_ready", False):
        P = ctypes.POINTER(_Problem)
        AP = ctypes.POINTER(_AmrPatch)
        DPP = ctypes.POINTER(_D)
        L.mcref_fine_problem.argtypes = [P, ctypes.c_int, AP, P]
        L.mcref_fine_problem.restype = None
        L.mcref_amr_fill_ghosts.argtypes = [P, ctypes.c_int, _D, _D, ctypes.c_double, AP, ctypes.c_int, DPP]
        L.mcref_amr_fill_ghosts.restype = None
        L.mcref_amr_average_down.argtypes = [P, ctypes.c_int, AP, ctypes.c_int, DPP, _D]
        L.mcref_amr_average_down.restype = None
        L.mcref_amr_step.argtypes = [P, ctypes.c_int, AP, ctypes.c_int, _D, _D, DPP, ctypes.c_double,
                                     ctypes.c_int, ctypes.c_int]
        L.mcref_edge_flux.argtypes = [P, _D, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, _D]
        L.mcref_edge_flux.restype = None
        L._amr_ready = True
    return L


def fine_problem(coarse: Problem, ratio: int, patch) -> Problem:
    """The fine patch's problem: coarse sizes / ratio, ghosts given."""
    ci0, cj0, cw, ch = patch
    return Problem(coarse.solver, ratio * cw, ratio * ch, coarse.dx / ratio, coarse.dy / ratio,
                   limiter=coarse.limiter, order=coarse.order, transverse=coarse.transverse,
                   efix=coarse.efix, bc=(BC_GIVEN,) * 4, param=coarse.param, mbc=coarse.mbc)


def _patch_array(patches):
    arr = (_AmrPatch * max(1, len(patches)))()
    for k, (ci0, cj0, cw, ch) in enumerate(patches):
        arr[k] = _AmrPatch(ci0, cj0, cw, ch)
    return arr


def amr_fill_ghosts(coarse: Problem, ratio, qc0, qc1, alpha, patches, qf):
    """Fill the ghost layers of the patch arrays qf (list, modified in place)."""
    qc0, qc1 = _f64(qc0), _f64(qc1)
    ptrs = (_D * max(1, len(qf)))(*[_p(a) for a in qf])
    _amr_lib().mcref_amr_fill_ghosts(ctypes.byref(coarse.c()), int(ratio), _p(qc0), _p(qc1),
                                     float(alpha), _patch_array(patches), len(patches), ptrs)


def amr_average_down(coarse: Problem, ratio, patches, qf, qc):
    qc = _f64(qc).copy()
    ptrs = (_D * max(1, len(qf)))(*[_p(a) for a in qf])
    _amr_lib().mcref_amr_average_down(ctypes.byref(coarse.c()), int(ratio), _patch_array(patches),
                                      len(patches), ptrs, _p(qc))
    return qc


def amr_step(coarse: Problem, ratio, patches, qc, qf, dt, nthreads=1, reflux=False):
    """One coarse step with ratio fine steps per patch -> (qc_new, flags); the
    patch arrays in the list qf are advanced in place.  reflux: correct the
    coarse cells outside the patches with the mean fine fluxes."""
    qc = _f64(qc)
    out = np.zeros_like(qc)
    for a in qf:
        assert a.dtype == np.float64 and a.flags.c_contiguous
    ptrs = (_D * max(1, len(qf)))(*[_p(a) for a in qf])
    flags = _amr_lib().mcref_amr_step(ctypes.byref(coarse.c()), int(ratio), _patch_array(patches),
                                      len(patches), _p(qc), _p(out), ptrs, float(dt), int(bool(reflux)),
                                      int(nthreads))
    return out, flags


def edge_flux(prob: Problem, q, dt: float, direction: int, i: int, j: int):
    """Flux through the edge of `direction` with high cell (i, j) implied by
    the step of q (ghosts filled) with dt."""
    q = _f64(q)
    F = np.zeros(prob.meqn)
    _amr_lib().mcref_edge_flux(ctypes.byref(prob.c()), _p(q), float(dt), int(direction), int(i),
                               int(j), _p(F))
    return F


def exact_sample(gamma, rl, ul, pl, rr, ur, pr, pstar, ustar):
    """(rho, u, p) of the exact 1D Riemann solution at x/t = 0."""
    out = [ctypes.c_double() for _ in range(3)]
    lib().mcref_exact_sample(*(float(v) for v in (gamma, rl, ul, pl, rr, ur, pr, pstar, ustar)),
                             *(ctypes.byref(o) for o in out))
    return tuple(o.value for o in out)


def flux(prob: Problem, direction: int, q):
    q = _f64(q)
    f = np.zeros(prob.meqn)
    lib().mcref_flux(ctypes.byref(prob.c()), direction, _p(q), _p(f))
    return f


def philim(limiter: int, theta: float) -> float:
    return lib().mcref_philim(limiter, float(theta))


# ---------------------------------------------------------------- grid

def bc_fill(prob: Problem, q):
    q = _f64(q).copy()
    lib().mcref_bc_fill(ctypes.byref(prob.c()), _p(q))
    return q


def step(prob: Problem, q, dt: float, nthreads: int = 1):
    """One CTU step -> (q_new with ghosts filled, smax, flags).  Courant = dt*smax."""
    q = _f64(q)
    assert q.shape == prob.shape, (q.shape, prob.shape)
    out = np.zeros_like(q)
    smax = ctypes.c_double(0.0)
    flags = lib().mcref_step(ctypes.byref(prob.c()), _p(q), _p(out), float(dt), ctypes.byref(smax),
                             int(nthreads))
    return out, smax.value, flags


def max_cell_speed(prob: Problem, q) -> float:
    q = _f64(q)
    return lib().mcref_max_cell_speed(ctypes.byref(prob.c()), _p(q))


def advance(prob: Problem, q, nsteps: int, cfl_desired: float, cfl_max: float, t: float, dt: float,
            nthreads: int = 1):
    """Variable-dt run with reject/retake -> (q, t, dt, nrejected, flags)."""
    qa = _f64(q).copy()
    qb = np.zeros_like(qa)
    tt, dd = ctypes.c_double(t), ctypes.c_double(dt)
    inb, nrej = ctypes.c_int(0), ctypes.c_int(0)
    flags = lib().mcref_advance(ctypes.byref(prob.c()), _p(qa), _p(qb), int(nsteps),
                                float(cfl_desired), float(cfl_max), ctypes.byref(tt),
                                ctypes.byref(dd), ctypes.byref(inb), ctypes.byref(nrej),
                                int(nthreads))
    return (qb if inb.value else qa), tt.value, dd.value, nrej.value, flags


# ---------------------------------------------------------------- exact solver

def seed(mode: int, gamma, rl, ul, pl, rr, ur, pr) -> float:
    return lib().mcref_seed(mode, gamma, rl, ul, pl, rr, ur, pr)


def pressure_function(gamma, rl, ul, pl, rr, ur, pr, p):
    f, fd = ctypes.c_double(), ctypes.c_double()
    lib().mcref_pressure_function(gamma, rl, ul, pl, rr, ur, pr, p, ctypes.byref(f), ctypes.byref(fd))
    return f.value, fd.value


def exact_riemann(gamma, rl, ul, pl, rr, ur, pr, seed_mode=SEED_ADAPTIVE, p_given=0.0,
                  tol=1e-8, max_iter=30):
    ps, us, it = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    flag = lib().mcref_exact_riemann(gamma, rl, ul, pl, rr, ur, pr, seed_mode, p_given, tol,
                                     max_iter, ctypes.byref(ps), ctypes.byref(us), ctypes.byref(it))
    return ps.value, us.value, it.value, flag


def exact_bisect(gamma, rl, ul, pl, rr, ur, pr):
    ps, us = ctypes.c_double(), ctypes.c_double()
    flag = lib().mcref_exact_bisect(gamma, rl, ul, pl, rr, ur, pr, ctypes.byref(ps), ctypes.byref(us))
    return ps.value, us.value, flag


def exact_batch(gamma, rl, ul, pl, rr, ur, pr, seed_mode=SEED_ADAPTIVE, p_given=None, tol=1e-8,
                max_iter=30, nthreads=None):
    arrs = [_f64(a) for a in (rl, ul, pl, rr, ur, pr)]
    n = arrs[0].size
    pg = _f64(p_given) if p_given is not None else None
    ps, us = np.zeros(n), np.zeros(n)
    it = np.zeros(n, np.int32)
    fl = np.zeros(n, np.int32)
    if nthreads is None:
        nthreads = len(os.sched_getaffinity(0))
    lib().mcref_exact_batch(n, gamma, *[_p(a) for a in arrs], seed_mode, _p(pg), tol, max_iter,
                            _p(ps), _p(us), it.ctypes.data_as(_I32), fl.ctypes.data_as(_I32),
                            int(nthreads))
    return ps, us, it, fl


# ---------------------------------------------------------------- network

def mlp_features(gamma, rl, ul, pl, rr, ur, pr):
    """Raw features, shape (n, 10)."""
    arrs = [np.atleast_1d(_f64(a)) for a in (rl, ul, pl, rr, ur, pr)]
    n = arrs[0].size
    out = np.zeros((n, NIN))
    f = np.zeros(NIN)
    L = lib()
    for k in range(n):
        L.mcref_mlp_features(gamma, *[float(a[k]) for a in arrs], _p(f))
        out[k] = f
    return out


def mlp_forward(X, W1, b1, W2, b2, W3, b3, bf16=False, return_hidden=False):
    X = _f64(X)
    B = X.shape[0]
    out = np.zeros(B)
    H1 = np.zeros((B, NH)) if return_hidden else None
    H2 = np.zeros((B, NH)) if return_hidden else None
    lib().mcref_mlp_forward(B, _p(X), _p(_f64(W1)), _p(_f64(b1)), _p(_f64(W2)), _p(_f64(b2)),
                            _p(_f64(W3)), _p(_f64(np.atleast_1d(b3))), int(bf16), _p(out), _p(H1),
                            _p(H2))
    return (out, H1, H2) if return_hidden else out


def mlp_backward(X, y, W1, b1, W2, b2, W3, b3, bf16=False):
    """-> (loss, dict of gradients)."""
    X, y = _f64(X), _f64(y)
    g = {"W1": np.zeros((KIN, NH)), "b1": np.zeros(NH), "W2": np.zeros((NH, NH)),
         "b2": np.zeros(NH), "W3": np.zeros(NH), "b3": np.zeros(1)}
    loss = lib().mcref_mlp_backward(X.shape[0], _p(X), _p(y), _p(_f64(W1)), _p(_f64(b1)),
                                    _p(_f64(W2)), _p(_f64(b2)), _p(_f64(W3)),
                                    _p(_f64(np.atleast_1d(b3))), int(bf16), _p(g["W1"]),
                                    _p(g["b1"]), _p(g["W2"]), _p(g["b2"]), _p(g["W3"]), _p(g["b3"]))
    return loss, g


def round_bf16(x: float) -> float:
    return lib().mcref_round_bf16(float(x))
