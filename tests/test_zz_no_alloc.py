"""The allocation-free entry point mg_residual_restrict_static.

Some callers cannot allocate device memory: their device memory belongs to
another allocator with a fixed budget, or they run on a latency-critical
path where cudaFree's implicit device synchronisation is not acceptable.  For
them the library offers the finest-level residual + restriction with its
intermediate residual in a fixed array compiled into the library.  This test
calls it through the C ABI twice in a row (the second call must not see the
first call's leftovers) and compares each result with the allocating entry
points mg_residual + mg_restrict, which use a buffer made by mg_setup.

This file sorts last so that a run stopping at the first failure has already
run every other test.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_03808_gb300 import Context, binding, inputs as I  # noqa: E402

K, MU = I.TABLE1["K"], I.TABLE1["mu"]


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("shape", [(32, 32, 32), (24, 16, 8)])
def test_static_variant_matches_allocating_entry_points(shape):
    nx, ny, nz = shape
    L = binding.lib()
    ctx = Context(nx, ny, nz, 1e-3, K, MU)
    stream = torch.cuda.current_stream()
    g = binding.mg_grid(nx, ny, nz, 1e-3)
    m = binding.mg_moduli(K, MU)
    rng = np.random.default_rng(17)
    for call in range(2):  # two calls in a row share the static array
        b = torch.from_numpy(rng.uniform(-1, 1, (3, nz + 1, ny, nx))).cuda()
        x = torch.from_numpy(rng.uniform(-1, 1, (3, nz + 1, ny, nx)) * (call + 1)).cuda()
        r = torch.zeros_like(b)
        ctx.residual(0, b, x, r)
        want = torch.zeros((3, nz // 2 + 1, ny // 2, nx // 2), dtype=torch.float64, device="cuda")
        ctx.restrict(0, r, want)
        got = torch.full_like(want, float("nan"))
        st = L.mg_residual_restrict_static(C.byref(g), C.byref(m), C.c_void_p(b.data_ptr()),
                                           C.c_void_p(x.data_ptr()), C.c_void_p(got.data_ptr()),
                                           C.c_void_p(stream.cuda_stream))
        assert st == binding.MG_OK, L.mg_last_error()
        torch.cuda.synchronize()
        assert _rel(got, want) <= 1e-12, call
        assert bool((got[:, 0] == 0).all()) and bool((got[:, nz // 2] == 0).all())
    ctx.close()


def test_static_variant_rejects_grids_beyond_its_array():
    L = binding.lib()
    g = binding.mg_grid(96, 96, 96, 1e-3)
    m = binding.mg_moduli(K, MU)
    dummy = C.c_void_p(1)  # never dereferenced: the size check comes first
    st = L.mg_residual_restrict_static(C.byref(g), C.byref(m), dummy, dummy, dummy, None)
    assert st == binding.MG_ERR_SHAPE
    assert b"static scratch" in L.mg_last_error()
