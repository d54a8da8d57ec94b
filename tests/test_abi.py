"""The C ABI library loads, exports every function include/rad.h declares
and validates its arguments on the host (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def R():
    from paper_2606_26268_b300 import build
    build.build()
    import paper_2606_26268_b300 as R
    return R


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rad.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rad_[a-z_]+)\s*\(", src)))


def test_every_declared_function_is_exported(R):
    L = R.lib()
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(R.EXPORTS)


def _grid(R, n=(8, 1, 1), ndim=1, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
    xs = [np.linspace(lo[d], hi[d], n[d] + 1) for d in range(3)]
    g = R.rad_grid()
    g.ndim = ndim
    for d in range(3):
        g.n[d] = n[d]
        g.xface[d] = xs[d].ctypes.data
    return g, xs


def test_async_host_transfers_validate_their_arguments(R):
    """The asynchronous host transfers check their arguments before touching
    the device: NULL pointers and unknown fields are RAD_EINVAL, a context
    without a workspace RAD_ENOMEM."""
    L = R.lib()
    g, xs = _grid(R)
    o = R.rad_opacity()
    p = R.default_params()
    ctx = C.c_void_p()
    assert L.rad_create(C.byref(g), 0, C.byref(o), C.byref(p), C.byref(ctx)) == R.RAD_OK
    buf = np.zeros(8)
    ptr = C.c_void_p(buf.ctypes.data)
    assert L.rad_set_gas_host_async(ctx, None, ptr, ptr) == R.RAD_EINVAL
    assert L.rad_set_rad_host_async(ctx, ptr, None) == R.RAD_EINVAL
    assert L.rad_read_host_async(ctx, 0, None, buf.nbytes) == R.RAD_EINVAL
    assert L.rad_read_host_async(ctx, 9, ptr, buf.nbytes) == R.RAD_EINVAL
    assert L.rad_read_host_async(ctx, 0, ptr, buf.nbytes) == R.RAD_ENOMEM
    assert L.rad_set_gas_host_async(ctx, ptr, ptr, ptr) == R.RAD_ENOMEM
    L.rad_destroy(ctx)


def test_host_side_validation(R):
    L = R.lib()
    g, xs = _grid(R)
    o = R.rad_opacity()
    p = R.default_params()
    ctx = C.c_void_p()
    assert L.rad_create(C.byref(g), 0, C.byref(o), C.byref(p), C.byref(ctx)) == R.RAD_OK
    size = C.c_size_t()
    assert L.rad_workspace_size(ctx, C.byref(size)) == R.RAD_OK and size.value > 0
    dt = C.c_double()
    assert L.rad_dt(ctx, C.byref(dt)) == R.RAD_OK
    assert dt.value == pytest.approx(0.4 / 8.0)
    # no workspace bound yet: stepping and reading refuse
    assert L.rad_step(ctx, 0.0, 1) == R.RAD_ENOMEM
    assert L.rad_step(ctx, 0.0, -1) == R.RAD_EINVAL
    L.rad_destroy(ctx)
    bad = []
    p2 = R.default_params(); p2.chat = -1.0; bad.append((g, 0, o, p2))
    p3 = R.default_params(); p3.c = 0.5; bad.append((g, 0, o, p3))            # c < chat
    p4 = R.default_params(); p4.ncomp = 4; bad.append((g, 0, o, p4))
    p5 = R.default_params(); p5.precision = 7; bad.append((g, 0, o, p5))
    p6 = R.default_params(); p6.e_floor = 0.0; bad.append((g, 0, o, p6))
    bad.append((g, 5, o, p))                                                   # geometry
    o2 = R.rad_opacity(); o2.kind = R.RAD_OPAC_TABLE; bad.append((g, 0, o2, p))  # no table
    g2, xs2 = _grid(R, (8, 2, 1), 1); bad.append((g2, 0, o, p))                 # n[1] != 1
    g3, xs3 = _grid(R); xs3[0][3] = xs3[0][2]; bad.append((g3, 0, o, p))        # not increasing
    g4, xs4 = _grid(R); g4.bc_lo[0] = 1; bad.append((g4, 0, o, p))              # half periodic
    for (gg, geom, oo, pp) in bad:
        c2 = C.c_void_p()
        assert L.rad_create(C.byref(gg), geom, C.byref(oo), C.byref(pp), C.byref(c2)) == R.RAD_EINVAL
        assert not c2.value
    assert L.rad_create(None, 0, C.byref(o), C.byref(p), C.byref(ctx)) == R.RAD_EINVAL
    assert L.rad_strerror(R.RAD_ENOCONV).decode().startswith("coupling")


def test_missing_library_fails_loudly(R, tmp_path, monkeypatch):
    import importlib
    monkeypatch.setattr(R, "LIB_PATH", str(tmp_path / "nope.so"))
    monkeypatch.setattr(R, "_lib", None)
    with pytest.raises(RuntimeError):
        R.lib()


def test_options_boundaries_and_gas_are_validated_on_the_host(R):
    L = R.lib()
    g, xs = _grid(R)
    o = R.rad_opacity()
    ctx = C.c_void_p()

    def create(gg, geom, pp):
        c2 = C.c_void_p()
        st = L.rad_create(C.byref(gg), geom, C.byref(o), C.byref(pp), C.byref(c2))
        if c2.value:
            L.rad_destroy(c2)
        return st

    for field, value in (("reconstruction", 2), ("face_fix", 3), ("riemann", 2),
                         ("implicit_mode", 3), ("hydro", 2), ("reconstruction", -1)):
        p = R.default_params()
        setattr(p, field, value)
        assert create(g, 0, p) == R.RAD_EINVAL, field
    # the gas step is Cartesian only
    p = R.default_params()
    p.hydro = 1
    gc, xc = _grid(R)
    xs_keep = np.linspace(0.5, 1.5, 9)  # radii > 0
    gc.xface[0] = xs_keep.ctypes.data
    assert create(gc, R.RAD_CYLINDRICAL, p) == R.RAD_EUNSUPPORTED
    assert create(g, 0, p) == R.RAD_OK
    # boundary kinds and states
    p = R.default_params()
    gb, xb = _grid(R)
    gb.bc_lo[0] = 5
    assert create(gb, 0, p) == R.RAD_EINVAL
    gb.bc_lo[0] = R.RAD_BC_FIXED
    for state, ok in (((1.0, 0.5, 0.0, 0.0, 1.0), True), ((1.0, 1.5, 0.0, 0.0, 1.0), False),
                      ((1.0, 0.5, 0.0, 0.0, 0.0), False), ((0.0, 0.0, 0.0, 0.0, 1.0), False),
                      ((1.0, 0.0, 0.5, 0.0, 1.0), False)):  # F_1 beyond ncomp = 1
        pp = R.default_params()
        pp.ncomp = 1
        for q in range(5):
            gb.bc_value[q] = state[q]
        assert create(gb, 0, pp) == (R.RAD_OK if ok else R.RAD_EINVAL), state
    gb.bc_lo[0] = R.RAD_BC_LTE
    for q in range(5):
        gb.bc_value[q] = (0.0, 0.0, 0.0, 0.0, 0.0)[q]
    assert create(gb, 0, p) == R.RAD_EINVAL        # T_b = 0
    gb.bc_value[4] = 1.0
    assert create(gb, 0, p) == R.RAD_OK
    gb.bc_lo[0] = R.RAD_BC_REFLECTIVE
    gb.bc_hi[0] = R.RAD_BC_PERIODIC
    assert create(gb, 0, p) == R.RAD_EINVAL        # periodic on one side only


def test_general_form_offers_the_right_launch_shapes(R):
    """Split 3D Cartesian: ten shapes in the default form and with evolved
    gas (the TMA-staged ones read the gas step's output), four with a face
    option of Sect. 2.5 (the register-tiled kernel only)."""
    L = R.lib()
    g, xs = _grid(R, (16, 16, 16), 3)
    o = R.rad_opacity()

    def shapes(**kw):
        p = R.default_params()
        p.precision = R.RAD_FP32_SPLIT
        for k, v in kw.items():
            setattr(p, k, v)
        c2 = C.c_void_p()
        assert L.rad_create(C.byref(g), 0, C.byref(o), C.byref(p), C.byref(c2)) == R.RAD_OK
        nv = C.c_int()
        assert L.rad_get_launch(c2, None, None, C.byref(nv)) == R.RAD_OK
        L.rad_destroy(c2)
        return nv.value

    assert shapes() == 10
    assert shapes(hydro=1) == 10
    assert shapes(irradiation=1) == 10
    assert shapes(implicit_mode=R.RAD_ABSORPTION_ONLY) == 10
    assert shapes(reconstruction=R.RAD_LIMO3) == 4
    assert shapes(face_fix=R.RAD_FIX_PLUTO, hydro=1) == 4


@pytest.mark.parametrize("geometry", [1, 2])
def test_curvilinear_grids_offer_the_tma_staged_shapes_in_the_split_form(R, geometry):
    """Split 3D cylindrical and spherical grids: the register-tiled shape and
    the TMA-staged non-overlapping 32x8 at 2 and 3 CTAs/SM and 16x16 at 3; FP64, or a face
    option of Sect. 2.5: the register-tiled shape only."""
    L = R.lib()
    g, xs = _grid(R, (16, 16, 16), 3, lo=(1.0, 0.5, 0.0), hi=(2.0, 2.5, 1.0))
    o = R.rad_opacity()

    def shapes(**kw):
        p = R.default_params()
        for k, v in kw.items():
            setattr(p, k, v)
        c2 = C.c_void_p()
        assert L.rad_create(C.byref(g), geometry, C.byref(o), C.byref(p), C.byref(c2)) == R.RAD_OK
        nv = C.c_int()
        assert L.rad_get_launch(c2, None, None, C.byref(nv)) == R.RAD_OK
        L.rad_destroy(c2)
        return nv.value

    assert shapes(precision=R.RAD_FP32_SPLIT) == 4
    assert shapes(precision=R.RAD_FP32_SPLIT, irradiation=1) == 4
    assert shapes(precision=R.RAD_FP32_SPLIT, reconstruction=R.RAD_LIMO3) == 1
    assert shapes(precision=R.RAD_FP64) == 1


def test_record_pointers_off_a_16_byte_boundary_are_refused(R):
    """Records are read and written as float4: a pointer that is not 16-byte
    aligned (an offset view starting inside a record) is refused on the host
    with RAD_EINVAL before anything is launched or the workspace is looked
    at, for every entry point that takes one."""
    L = R.lib()
    g, xs = _grid(R)
    o = R.rad_opacity()
    p = R.default_params()
    ctx = C.c_void_p()
    assert L.rad_create(C.byref(g), 0, C.byref(o), C.byref(p), C.byref(ctx)) == R.RAD_OK
    odd = C.c_void_p(0x10004)   # never dereferenced: refused on the host
    out = C.c_void_p(0x20000)
    loss = C.c_float()
    assert L.rad_mlp_grad(ctx, odd, 16, None, C.byref(loss)) == R.RAD_EINVAL
    assert L.rad_mlp_train(ctx, odd, 16, 1, 8, C.c_float(1e-3), 0, None) == R.RAD_EINVAL
    assert L.rad_mlp_predict(ctx, odd, 16, out) == R.RAD_EINVAL
    assert L.rad_mlp_predict_tc(ctx, odd, 16, out) == R.RAD_EINVAL
    assert L.rad_log_bind(ctx, odd, 16, 1) == R.RAD_EINVAL
    assert L.rad_mlp_grad_noalloc(out, odd, 16, out, out, None) == R.RAD_EINVAL
    # an aligned pointer gets past the check (no workspace bound: RAD_ENOMEM)
    assert L.rad_mlp_predict(ctx, C.c_void_p(0x10010), 16, out) == R.RAD_ENOMEM
    L.rad_destroy(ctx)


def test_wait_limit_setter_validates_its_context(R):
    L = R.lib()
    assert L.rad_set_wait_limit(None, 1) == R.RAD_EINVAL


def test_debug_build_exports_the_same_entry_points_and_the_release_build_refuses_the_check(R):
    """The debug build (librad_debug.so, RAD_DEBUG_CHECKS) exports every
    function include/rad.h declares; its index check reports RAD_EBOUNDS,
    which rad_strerror names.  The release build compiles the checks out and
    answers rad_debug_check_index with RAD_EUNSUPPORTED, on the host."""
    from paper_2606_26268_b300 import build
    lib = build.build(debug=True)
    D = C.CDLL(lib)
    for name in declared_functions():
        assert hasattr(D, name), name
    L = R.lib()
    L.rad_strerror.restype = C.c_char_p
    assert b"index check" in L.rad_strerror(R.RAD_EBOUNDS)
    g, xs = _grid(R)
    o = R.rad_opacity()
    p = R.default_params()
    ctx = C.c_void_p()
    assert L.rad_create(C.byref(g), 0, C.byref(o), C.byref(p), C.byref(ctx)) == R.RAD_OK
    assert L.rad_debug_check_index(ctx, 0) == R.RAD_EUNSUPPORTED
    assert L.rad_debug_check_index(None, 0) == R.RAD_EINVAL
    L.rad_destroy(ctx)
