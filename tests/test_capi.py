"""C-ABI checks that need no GPU: the library loads, exports every function
include/manyclaw.h declares, validates problems and computes layouts."""
import ctypes

import pytest

import paper_1308_1464_gb300 as mc


@pytest.fixture(scope="module")
def L():
    from paper_1308_1464_gb300 import _build
    _build.build()
    return mc.lib()


def test_exports_every_declared_function(L):
    names = mc.header_functions()
    assert len(names) >= 12, names
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/manyclaw.h but not exported"


def test_status_strings(L):
    assert mc.status_string(0) == "MC_OK"
    for st in range(-7, 0):
        assert mc.status_string(st).startswith("MC_E")


def base_problem(**kw):
    args = dict(solver=mc.SWE_ROE, mx=100, my=50, dx=0.01, dy=0.02, dtype=mc.F32,
                bc=(mc.BC_WALL,) * 4, param=(9.81, 0, 0, 0))
    args.update(kw)
    return mc.Problem.make(**args)


def test_layout(L):
    lay = mc.layout_of(base_problem())
    assert lay.elem_bytes == 4 and lay.meqn == 3
    assert lay.x_offset * 4 % 16 == 0 and lay.x_offset >= 2
    assert lay.ld_x * 4 % 128 == 0 and lay.ld_x >= lay.x_offset + 100 + 2
    assert lay.ld_field == lay.ld_x * 54
    assert lay.bytes == 3 * lay.ld_field * 4
    lay = mc.layout_of(base_problem(dtype=mc.F64, solver=mc.EULER_ROE, param=(1.4, 0, 0, 0)))
    assert lay.elem_bytes == 8 and lay.meqn == 4 and lay.x_offset * 8 % 16 == 0
    lay = mc.layout_of(base_problem(solver=mc.ADVECTION, param=(1.0, -0.5, 0, 0), limiter=mc.LIM_VANLEER,
                                    transverse=2))
    assert lay.meqn == 1 and lay.bytes == lay.ld_field * 4


@pytest.mark.parametrize("kw", [
    dict(solver=7), dict(solver=0), dict(dtype=3), dict(mx=0), dict(my=-1), dict(limiter=5),
    dict(limiter=-1), dict(order=3), dict(transverse=3),
    dict(bc=(mc.BC_PERIODIC, mc.BC_WALL, 0, 0)), dict(dx=0.0), dict(param=(0.0, 0, 0, 0)),
    dict(solver=mc.EULER_ROE, param=(1.0, 0, 0, 0)), dict(bc=(4, 2, 2, 2)),
    dict(mx=1, bc=(mc.BC_GIVEN, mc.BC_WALL, mc.BC_WALL, mc.BC_WALL)),
])
def test_invalid_problems_rejected(L, kw):
    p = base_problem(**kw)
    lay = mc.Layout()
    st = L.mc_layout_of(ctypes.byref(p), ctypes.byref(lay))
    assert st == mc.MC_EINVAL
    assert mc.last_error()


def test_mbc_must_be_two(L):
    p = base_problem()
    p.mbc = 3
    with pytest.raises(mc.McError):
        mc.layout_of(p)


def test_null_arguments(L):
    assert L.mc_layout_of(None, None) == mc.MC_EINVAL
    assert L.mc_step(None, None, None, 0.1, None, None) == mc.MC_EINVAL
    assert L.mc_destroy(None) == mc.MC_OK


def test_halo_strip_sizes(L):
    """Strips of a block: two interior columns by my rows (x sides), two rows
    across the padded width mx + 4 (y sides), all planes."""
    p = base_problem(mx=30, my=7, bc=(mc.BC_GIVEN, mc.BC_WALL, mc.BC_GIVEN, mc.BC_GIVEN))
    mc.layout_of(p)
    n = ctypes.c_int64()
    for side, want in ((0, 3 * 7 * 2), (1, 3 * 7 * 2), (2, 3 * 2 * 34), (3, 3 * 2 * 34)):
        assert L.mc_halo_elems(ctypes.byref(p), side, ctypes.byref(n)) == mc.MC_OK
        assert n.value == want
    assert L.mc_halo_elems(ctypes.byref(p), 4, ctypes.byref(n)) == mc.MC_EINVAL
    assert L.mc_halo_pack(None, None, 0, None, None) == mc.MC_EINVAL
    assert L.mc_bc_fill_dir(None, None, 0, None) == mc.MC_EINVAL
