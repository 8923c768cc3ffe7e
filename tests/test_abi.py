"""The C-ABI library builds, loads and exports every function declared in
include/bzcoll.h; host-side argument checks answer without touching a GPU."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_2103_14890_gb300 import build, binding
    build.build()
    return binding.load()


def test_exports_every_declared_function(lib):
    from paper_2103_14890_gb300 import binding
    names = binding.header_functions()
    assert "collide_batch" in names and "imex_stage_local" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    from paper_2103_14890_gb300 import binding
    src = open(binding.__file__).read()
    for n in binding.header_functions():
        assert '"%s"' % n in src, n


def test_host_side_argument_errors(lib):
    from paper_2103_14890_gb300 import binding as b
    out = ctypes.c_void_p()
    assert lib.init_velocity_grid(4, 32, 10.0, ctypes.byref(out)) == b.EINVAL
    assert b"dim" in lib.bz_last_error()
    assert lib.init_velocity_grid(2, 33, 10.0, ctypes.byref(out)) == b.EINVAL
    assert lib.init_velocity_grid(2, 32, -1.0, ctypes.byref(out)) == b.EINVAL
    assert lib.init_velocity_grid(2, 32, 1.0, None) == b.EINVAL
    assert lib.build_kernel_modes(None, 1.0, 0.0, 0, ctypes.byref(out)) == b.EINVAL
    assert lib.collide_batch(None, 1, 0, None, None, 4, None) == b.EINVAL
    assert b"modes" in lib.bz_last_error()
    assert lib.imex_step(None, 0, 0, 0.1, 1.0, None, None, None, 4, 1, 0, None) == b.EINVAL
    assert lib.imex_stage_local(None, 0, 1, 0, 0.1, 1.0, None, None, None, None, None, 4, 1, 0, None) == b.EINVAL
    info = (ctypes.c_int64 * 8)()
    assert lib.bz_modes_info(None, info) == b.EINVAL
    assert lib.bz_modes_beta(None, None) == b.EINVAL
    assert lib.bz_profile_read(None, 0, None, None, 0) == b.EINVAL
    assert lib.build_fast_modes(None, 0.0, 8, ctypes.byref(out)) == b.EINVAL
    assert lib.build_fast_modes(None, 0.0, 8, None) == b.EINVAL
    assert lib.bz_fast_info(None, (ctypes.c_int64 * 4)()) == b.EINVAL
    assert lib.build_fv_mesh(0, None, 1, None, None, 2, ctypes.byref(out)) == b.EINVAL
    assert lib.build_fv_mesh_periodic(0, None, 1, None, None, 2, 10.0, 10.0, ctypes.byref(out)) == b.EINVAL
    assert lib.bz_modes_set_penalty(None, 3.0) == b.EINVAL
    xy = (ctypes.c_double * 6)(0, 0, 1, 0, 0, 1)
    ptr = (ctypes.c_int64 * 2)(0, 3)
    vtx = (ctypes.c_int64 * 3)(0, 1, 2)
    assert lib.build_fv_mesh_periodic(3, xy, 1, ptr, vtx, 2, -1.0, 0.0, ctypes.byref(out)) == b.EINVAL
    for order in (0, 4):                                     # orders 1, 2, 3 only
        assert lib.build_fv_mesh(3, xy, 1, ptr, vtx, order, ctypes.byref(out)) == b.EINVAL
    assert lib.transport_residual(None, None, 1, None, None, None) == b.EINVAL
    assert lib.bz_mesh_info(None, (ctypes.c_int64 * 5)()) == b.EINVAL
    assert lib.imex_step_fv(None, None, 0, 0, 0.1, 1.0, None, None, 1, 0, None) == b.EINVAL


def test_missing_library_fails_loudly(tmp_path):
    from paper_2103_14890_gb300 import binding as b
    saved = b._lib
    try:
        b._lib = None
        with pytest.raises(b.BzError):
            b.load(str(tmp_path / "absent.so"))
    finally:
        b._lib = saved


def test_alloc_injection_hook_host_side(lib):
    """The fault-injection hook and the allocation counters answer on the
    host: arming and disarming return BZ_OK; with no handle alive and no pool
    created the library holds nothing."""
    from paper_2103_14890_gb300 import binding as b
    assert lib.bz_inject_alloc_failure(3) == b.OK
    assert lib.bz_inject_alloc_failure(-1) == b.OK
    live, used = ctypes.c_int64(-7), ctypes.c_uint64(7)
    assert lib.bz_alloc_stats(ctypes.byref(live), ctypes.byref(used)) == b.OK
    assert live.value == 0 and used.value == 0
    assert lib.bz_alloc_stats(None, None) == b.OK
