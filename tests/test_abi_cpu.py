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
