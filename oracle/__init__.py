"""Python face of the FP64 CPU oracle (``qs_oracle.c``).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline / reference legs use it; the product path never imports it.  It
shares no code with the CUDA library: it is compiled from its own C source
with gcc and called through ctypes on numpy arrays.

Array layouts: corner fields (3, nz+1, ny, nx); cell stress (6, nz, ny, nx)
in the order xx, yy, zz, yz, xz, xy; cell scalars (nz, ny, nx); float64.
Stencil tables: (27, 3, 3) with offset index (dz+1)*9 + (dy+1)*3 + (dx+1).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qs_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libqs_oracle.so")
_lib = None

_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


# -O3 without -march=native and without contraction into fused multiply-adds,
# so that the oracle computes the expressions as written and gives the same
# rounding on every host (x86-64 and aarch64 alike)
_CFLAGS = ["-O3", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile qs_oracle.c with gcc (OpenMP across the nodes of one colour
    pass and of one pointwise loop)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    stamp = _OUT + ".flags"
    flags = " ".join(_CFLAGS)
    stale = (not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC) or
             not os.path.exists(stamp) or open(stamp).read() != flags)
    if force or stale:
        tmp = _OUT + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc"] + _CFLAGS + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
        with open(stamp, "w") as f:
            f.write(flags)
    return _OUT


class STZ(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("tau0", "eps0", "c0", "Delta_K", "Omega", "T", "chi_inf", "ez_K", "sY", "l", "kB")]


class BC(C.Structure):
    _fields_ = [("kind", C.c_int)] + [(n, C.c_double) for n in
                                      ("U_B", "t_ramp", "omega", "R", "lambda_w")]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.ora_threads.restype = C.c_int
        L.ora_fine_stencil.argtypes = [C.c_double, C.c_double, _D]
        L.ora_galerkin.argtypes = [_D, _D]
        for f in (L.ora_apply,):
            f.argtypes = [C.c_int, C.c_int, C.c_int, _D, _D, _D]
        L.ora_residual.argtypes = [C.c_int, C.c_int, C.c_int, _D, _D, _D, _D]
        L.ora_norm2.argtypes = [C.c_int, C.c_int, C.c_int, _D]
        L.ora_norm2.restype = C.c_double
        L.ora_gs_colour.argtypes = [C.c_int, C.c_int, C.c_int, _D, _D, _D, C.c_int]
        L.ora_restrict.argtypes = [C.c_int, C.c_int, C.c_int, _D, _D]
        L.ora_prolong_add.argtypes = [C.c_int, C.c_int, C.c_int, _D, _D]
        L.ora_mg_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int, C.c_int]
        L.ora_mg_create.restype = C.c_void_p
        L.ora_mg_free.argtypes = [C.c_void_p]
        L.ora_mg_levels.argtypes = [C.c_void_p]
        L.ora_mg_level_dims.argtypes = [C.c_void_p, C.c_int, _I]
        L.ora_mg_stencil.argtypes = [C.c_void_p, C.c_int, _D]
        L.ora_mg_dense.argtypes = [C.c_void_p, C.c_int, _D]
        L.ora_mg_coarse_size.argtypes = [C.c_void_p]
        L.ora_mg_vcycle.argtypes = [C.c_void_p, _D, _D]
        L.ora_mg_solve.argtypes = [C.c_void_p, _D, _D, C.c_double, C.c_int, _I, _D]
        L.ora_cholesky.argtypes = [_D, C.c_long]
        L.ora_dpl.argtypes = [C.POINTER(STZ), C.c_double, C.c_double]
        L.ora_dpl.restype = C.c_double
        L.ora_cell_gradient.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, _D, _D]
        L.ora_stress_star.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                      C.POINTER(STZ), _D, _D, _D, _D, _D, _D]
        L.ora_chi_update.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                     C.POINTER(STZ), _D, _D, _D, _D, _D]
        L.ora_div_rhs.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, _D, _D]
        L.ora_stress_final.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double,
                                       C.c_double, _D, _D, _D]
        L.ora_wall_fill.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(BC), C.c_double, _D]
        L.ora_qs_step.argtypes = [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double,
                                  C.POINTER(STZ), C.POINTER(BC), C.c_double, _D, _D, _D,
                                  C.c_double, C.c_int, _I, _D]
        L.ora_stress_star_adv.argtypes = L.ora_stress_star.argtypes + [C.c_int]
        L.ora_qs_step_adv.argtypes = L.ora_qs_step.argtypes + [C.c_int]
        L.ora_eno.argtypes = [_D, C.c_double, C.c_double]
        L.ora_eno.restype = C.c_double
        L.ora_explicit_step.argtypes = [C.c_int, C.c_int, C.c_int] + [C.c_double] * 6 + [
            C.POINTER(STZ), C.POINTER(BC), C.c_double, _D, _D, _D]
    return _lib


def threads() -> int:
    return lib().ora_threads()


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _dims(x: np.ndarray):
    c, nz1, ny, nx = x.shape
    assert c == 3
    return nx, ny, nz1 - 1


def fine_stencil(lam: float, mu: float) -> np.ndarray:
    S = np.zeros((27, 3, 3))
    lib().ora_fine_stencil(lam, mu, _p(S))
    return S


def galerkin(S: np.ndarray) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.float64)
    Sc = np.zeros((27, 3, 3))
    lib().ora_galerkin(_p(S), _p(Sc))
    return Sc


def apply(S: np.ndarray, x: np.ndarray) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.float64)
    y = np.zeros_like(x)
    lib().ora_apply(*_dims(x), _p(S), _p(x), _p(y))
    return y


def residual(S, b, x) -> np.ndarray:
    S = np.ascontiguousarray(S, dtype=np.float64)
    r = np.zeros_like(x)
    lib().ora_residual(*_dims(x), _p(S), _p(b), _p(x), _p(r))
    return r


def norm2(r) -> float:
    return lib().ora_norm2(*_dims(r), _p(r))


def gs_colour(S, b, x, colour: int) -> None:
    S = np.ascontiguousarray(S, dtype=np.float64)
    lib().ora_gs_colour(*_dims(x), _p(S), _p(b), _p(x), colour)


def restrict(r) -> np.ndarray:
    nx, ny, nz = _dims(r)
    bc = np.zeros((3, nz // 2 + 1, ny // 2, nx // 2))
    lib().ora_restrict(nx, ny, nz, _p(r), _p(bc))
    return bc


def prolong_add(xc, x) -> None:
    lib().ora_prolong_add(*_dims(x), _p(xc), _p(x))


class MG:
    """Oracle multigrid hierarchy for an nx*ny*nz-cell grid (section 3.6)."""

    def __init__(self, nx, ny, nz, lam, mu, nu1=2, nu2=2):
        self.h = lib().ora_mg_create(nx, ny, nz, lam, mu, nu1, nu2)
        if not self.h:
            raise ValueError("unsupported grid %dx%dx%d" % (nx, ny, nz))
        self.shape = (nx, ny, nz)

    def close(self):
        if self.h:
            lib().ora_mg_free(self.h)
            self.h = None

    def __del__(self):
        self.close()

    @property
    def levels(self) -> int:
        return lib().ora_mg_levels(self.h)

    def dims(self, l):
        d = (C.c_int * 3)()
        lib().ora_mg_level_dims(self.h, l, d)
        return tuple(d)

    def stencil(self, l) -> np.ndarray:
        S = np.zeros((27, 3, 3))
        lib().ora_mg_stencil(self.h, l, _p(S))
        return S

    def dense(self, l) -> np.ndarray:
        nx, ny, nz = self.dims(l)
        n = 3 * nx * ny * (nz - 1)
        A = np.zeros((n, n))
        lib().ora_mg_dense(self.h, l, _p(A))
        return A

    def vcycle(self, b, x) -> None:
        lib().ora_mg_vcycle(self.h, _p(b), _p(x))

    def solve(self, b, x, tol=1e-10, max_cycles=100):
        """In-place solve; returns (status, cycles, history)."""
        cyc = C.c_int(0)
        hist = np.zeros(max_cycles + 1)
        st = lib().ora_mg_solve(self.h, _p(b), _p(x), tol, max_cycles, C.byref(cyc), _p(hist))
        return st, cyc.value, hist[: cyc.value + 1].copy()


def dpl(stz: STZ, sbar: float, chi: float) -> float:
    return lib().ora_dpl(C.byref(stz), sbar, chi)


def cell_gradient(v, h) -> np.ndarray:
    nx, ny, nz = _dims(v)
    L = np.zeros((nz, ny, nx, 3, 3))
    lib().ora_cell_gradient(nx, ny, nz, h, _p(v), _p(L))
    return L


def stress_star(v, sig, chi, h, dt, mu, stz, advect=False):
    """Eq. (27); advect adds -(u.grad) sigma (ENO, Eq. 33) to the rate."""
    nx, ny, nz = _dims(v)
    ss = np.zeros_like(sig)
    D = np.zeros_like(chi)
    sb = np.zeros_like(chi)
    lib().ora_stress_star_adv(nx, ny, nz, h, dt, mu, C.byref(stz), _p(v), _p(sig), _p(chi),
                              _p(ss), _p(D), _p(sb), 1 if advect else 0)
    return ss, D, sb


def chi_update(sig, chi, D, sb, h, dt, stz):
    nz, ny, nx = chi.shape
    out = np.zeros_like(chi)
    lib().ora_chi_update(nx, ny, nz, h, dt, C.byref(stz), _p(sig), _p(chi), _p(D), _p(sb), _p(out))
    return out


def div_rhs(sig_star, h, dt, mu):
    _, nz, ny, nx = sig_star.shape
    b = np.zeros((3, nz + 1, ny, nx))
    lib().ora_div_rhs(nx, ny, nz, h, dt, mu, _p(sig_star), _p(b))
    return b


def stress_final(v, sig_star, h, dt, lam, mu):
    nx, ny, nz = _dims(v)
    sig = np.zeros_like(sig_star)
    lib().ora_stress_final(nx, ny, nz, h, dt, lam, mu, _p(v), _p(sig_star), _p(sig))
    return sig


def wall_fill(v, h, bc: BC, t: float) -> None:
    lib().ora_wall_fill(*_dims(v), h, C.byref(bc), t, _p(v))


def qs_step(mg: MG, v, sig, chi, h, dt, lam, mu, stz: STZ, bc: BC, t, tol=1e-10, max_cycles=100,
            advect=False):
    """One projection step in place (advect: the stress advection of
    stress_star); returns (status, cycles, history)."""
    cyc = C.c_int(0)
    hist = np.zeros(max_cycles + 1)
    st = lib().ora_qs_step_adv(mg.h, h, dt, lam, mu, C.byref(stz), C.byref(bc), t, _p(v),
                               _p(sig), _p(chi), tol, max_cycles, C.byref(cyc), _p(hist),
                               1 if advect else 0)
    return st, cyc.value, hist[: cyc.value + 1].copy()


def eno(f5, u, h) -> float:
    """ENO first derivative of Eq. (33) from the 5 values at offsets -2..2."""
    f = np.ascontiguousarray(f5, dtype=np.float64)
    assert f.shape == (5,)
    return lib().ora_eno(_p(f), float(u), float(h))


def explicit_step(v, sig, chi, h, dt, rho, lam, mu, kappa, stz: STZ, bc: BC, t) -> None:
    """One explicit forward-Euler step (section 3.2, Eqs. 24-26) in place."""
    nx, ny, nz = _dims(v)
    lib().ora_explicit_step(nx, ny, nz, h, dt, rho, lam, mu, kappa, C.byref(stz), C.byref(bc), t,
                            _p(v), _p(sig), _p(chi))
