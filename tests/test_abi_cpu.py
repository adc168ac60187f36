"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function include/qsmg.h declares (no compute calls here)."""
import ctypes

from paper_1904_03808_gb300 import binding, build


def test_library_exports_every_declared_function():
    path = build.build()
    L = ctypes.CDLL(path)
    names = binding.header_functions()
    assert {"mg_setup", "mg_solve", "qs_step", "mg_free"} <= set(names)
    for n in names:
        assert hasattr(L, n), n
    # the binding knows every declared symbol
    assert set(names) <= set(binding._SIGS)


def test_status_strings_without_gpu():
    L = binding.lib()
    assert L.mg_status_str(0) == b"ok"
    assert L.mg_status_str(2) == b"unsupported grid shape"


def test_setup_rejects_bad_shapes_without_touching_the_gpu():
    L = binding.lib()
    out = ctypes.c_void_p()
    o = binding.mg_opts(0, 2, 2, 50, 4)
    m = binding.mg_moduli(122e9, 37.4e9)
    for (nx, ny, nz) in ((7, 8, 8), (8, 8, 3), (2, 8, 8), (8, 8, 0)):
        g = binding.mg_grid(nx, ny, nz, 1e-3)
        st = L.mg_setup(ctypes.byref(g), ctypes.byref(m), None, None, ctypes.byref(o), None,
                        ctypes.byref(out))
        assert st == binding.MG_ERR_SHAPE, (nx, ny, nz)
    g = binding.mg_grid(8, 8, 8, 1e-3)
    bad = binding.mg_opts(7, 2, 2, 50, 4)
    assert L.mg_setup(ctypes.byref(g), ctypes.byref(m), None, None, ctypes.byref(bad), None,
                      ctypes.byref(out)) == binding.MG_ERR_ARG
    assert L.mg_solve(None, None, None, 1e-10, None) == binding.MG_ERR_ARG


def test_setup_rejects_a_coarsest_level_beyond_the_dense_solve():
    """Coarsening stops once a dimension would fall below 4 cells; the level
    left must fit the dense coarsest solve (3072 unknowns).  A slender
    768 x 768 x 192 grid stops at 24 x 24 x 6 (8640 unknowns) and 384 x 24 x 16
    at 96 x 6 x 4 (5184): both are refused before any device work, with the
    level named in the error string."""
    L = binding.lib()
    out = ctypes.c_void_p()
    o = binding.mg_opts(0, 2, 2, 50, 4)
    m = binding.mg_moduli(122e9, 37.4e9)
    for shape, level in (((768, 768, 192), b"24x24x6"), ((384, 24, 16), b"96x6x4")):
        g = binding.mg_grid(*shape, 1e-3)
        st = L.mg_setup(ctypes.byref(g), ctypes.byref(m), None, None, ctypes.byref(o), None,
                        ctypes.byref(out))
        assert st == binding.MG_ERR_SHAPE, shape
        assert level in L.mg_last_error(), L.mg_last_error()
        assert not out.value


def test_missing_library_fails_loudly(monkeypatch):
    """No CPU fallback: without the built CUDA library the binding raises."""
    import pytest
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "lib_path", lambda: "/nonexistent/libqsmg.so")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        binding.lib()


def test_reverse_mode_entry_points_reject_null_arguments_without_gpu():
    L = binding.lib()
    assert L.qs_step_adjoint(None, None, 1.0, 1e-10, 1.0, None, None, None,
                             None) == binding.MG_ERR_ARG
    W = ctypes.c_double()
    assert L.qs_plastic_work_grad(None, None, 4, 1.0, 1e-10, 2, None, ctypes.byref(W),
                                  None) == binding.MG_ERR_ARG
    assert L.qs_plastic_work(None, None, 4, 1.0, 1e-10, 2, None, ctypes.byref(W),
                             None) == binding.MG_ERR_ARG
    assert L.qs_plastic_work_backward(None, None, 0.0, 0, 4, 1.0, 1e-10, 2, None,
                                      None) == binding.MG_ERR_ARG
    assert b"null" in L.mg_last_error()


def test_qs_run_rejects_null_arguments_without_gpu():
    L = binding.lib()
    assert L.qs_run(None, None, 2, 1.0, 1e-10, None) == binding.MG_ERR_ARG
    assert L.qs_step(None, None, 1.0, 1e-10, None) == binding.MG_ERR_ARG


def test_explicit_step_rejects_null_arguments_without_gpu():
    L = binding.lib()
    assert L.qs_explicit_step(None, None, 1e-9, 6125.0, 1.0, 1) == binding.MG_ERR_ARG


def test_plastic_work_is_an_autograd_function_over_the_c_entry_point():
    import torch
    cls = binding._plastic_work_class()
    assert issubclass(cls, torch.autograd.Function)
    from paper_1904_03808_gb300 import plastic_work
    assert plastic_work is binding.plastic_work
