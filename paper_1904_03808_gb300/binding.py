"""Thin ctypes binding of the C ABI in include/qsmg.h.

Argument marshalling only: every step of the solve and of the projection
step runs in the CUDA library ``_build/libqsmg.so``.  There is no CPU
fallback; if the library is missing or fails to load this module raises.
Torch tensors are accepted wherever the ABI takes a device pointer: they must
be contiguous float64 (float32 for the FP32 smoother entry) CUDA tensors.
"""
from __future__ import annotations

import ctypes as C
import os
import re

from . import build as _build

_lib = None

MG_OK, MG_ERR_ARG, MG_ERR_SHAPE, MG_ERR_CUDA, MG_ERR_OOM, MG_ERR_NOCONV, MG_ERR_NONFINITE, \
    MG_ERR_STATE = range(8)
MG_FP64, MG_MIXED = 0, 1
MG_FLAG_COLOUR_PASSES = 1
MG_FLAG_NO_GRAPH = 2
MG_FLAG_FUSED_SWEEP = 4
MG_FLAG_UNFUSED_TRANSFERS = 8
MG_FLAG_ADVECT_STRESS = 16
MG_HIST = 128


class mg_grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("h", C.c_double)]


class mg_moduli(C.Structure):
    _fields_ = [("K", C.c_double), ("mu", C.c_double)]


class mg_bc(C.Structure):
    _fields_ = [("kind", C.c_int)] + [(n, C.c_double) for n in
                                      ("U_B", "t_ramp", "omega", "R", "lambda_w")]


class stz_params(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("tau0", "eps0", "c0", "Delta_K", "Omega", "T", "chi_inf", "ez_K", "sY", "l", "kB")]


class mg_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int),
                ("max_cycles", C.c_int), ("inner_cycles", C.c_int), ("flags", C.c_int)]


class mg_stats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("outer_iters", C.c_int), ("rel_resid", C.c_double),
                ("bnorm", C.c_double), ("resid_hist", C.c_double * MG_HIST)]


class qs_state(C.Structure):
    _fields_ = [("v", C.c_void_p), ("sigma", C.c_void_p), ("chi", C.c_void_p),
                ("t", C.c_double), ("step", C.c_long)]


class QSMGError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = "%s: %s (%s)" % (where, lib().mg_status_str(status).decode(),
                                lib().mg_last_error().decode())
        super().__init__(msg)


_P = C.c_void_p
_SIGS = {
    "mg_setup": (C.c_int, [C.POINTER(mg_grid), C.POINTER(mg_moduli), C.POINTER(mg_bc),
                           C.POINTER(stz_params), C.POINTER(mg_opts), _P, C.POINTER(_P)]),
    "mg_solve": (C.c_int, [_P, _P, _P, C.c_double, C.POINTER(mg_stats)]),
    "qs_step": (C.c_int, [_P, C.POINTER(qs_state), C.c_double, C.c_double, C.POINTER(mg_stats)]),
    "qs_run": (C.c_int, [_P, C.POINTER(qs_state), C.c_int, C.c_double, C.c_double,
                         C.POINTER(mg_stats)]),
    "mg_free": (None, [_P]),
    "mg_status_str": (C.c_char_p, [C.c_int]),
    "mg_last_error": (C.c_char_p, []),
    "mg_num_levels": (C.c_int, [_P]),
    "mg_level_dims": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int)]),
    "mg_level_stencil": (C.c_int, [_P, C.c_int, C.POINTER(C.c_double)]),
    "mg_residual": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "mg_residual32": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "mg_residual_restrict32": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "mg_smooth": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, C.c_int, C.c_int]),
    "mg_restrict": (C.c_int, [_P, C.c_int, _P, _P]),
    "mg_prolong_add": (C.c_int, [_P, C.c_int, _P, _P]),
    "mg_vcycle": (C.c_int, [_P, _P, _P]),
    "qs_stress_predict": (C.c_int, [_P, _P, _P, _P, C.c_double, _P, _P, _P]),
    "qs_chi_update": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, _P]),
    "qs_rhs": (C.c_int, [_P, _P, C.c_double, _P]),
    "qs_stress_correct": (C.c_int, [_P, _P, _P, C.c_double, _P]),
    "qs_wall_fill": (C.c_int, [_P, _P, C.c_double]),
    "qs_step_adjoint": (C.c_int, [_P, C.POINTER(qs_state), C.c_double, C.c_double, C.c_double,
                                  _P, _P, _P, C.POINTER(mg_stats)]),
    "qs_plastic_work_grad": (C.c_int, [_P, C.POINTER(qs_state), C.c_int, C.c_double, C.c_double,
                                       C.c_int, _P, C.POINTER(C.c_double), C.POINTER(mg_stats)]),
    "qs_plastic_work": (C.c_int, [_P, C.POINTER(qs_state), C.c_int, C.c_double, C.c_double,
                                  C.c_int, _P, C.POINTER(C.c_double), C.POINTER(mg_stats)]),
    "qs_plastic_work_backward": (C.c_int, [_P, _P, C.c_double, C.c_long, C.c_int, C.c_double,
                                           C.c_double, C.c_int, _P, C.POINTER(mg_stats)]),
    "qs_explicit_step": (C.c_int, [_P, C.POINTER(qs_state), C.c_double, C.c_double, C.c_double,
                                   C.c_int]),
    "mg_profile": (C.c_int, [_P, C.c_int]),
    "mg_profile_read": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_long),
                                  C.POINTER(C.c_long)]),
    "mg_launch_count": (C.c_long, []),
    "mg_residual_restrict_static": (C.c_int, [C.POINTER(mg_grid), C.POINTER(mg_moduli), _P, _P,
                                              _P, _P]),
}


def lib_path() -> str:
    return _build.LIB


def lib():
    """Load libqsmg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError("CUDA library %s is missing: run paper_1904_03808_gb300.build.build() "
                               "(no CPU fallback exists)" % path)
        L = C.CDLL(path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def header_functions():
    """Names of the functions include/qsmg.h declares."""
    h = os.path.join(os.path.dirname(_build.HERE), "include", "qsmg.h")
    text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
    return sorted(set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", text)) -
                  {"if", "sizeof", "defined", "for", "while", "return"})


def _ptr(t, dtype=None):
    import torch
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError("expected dtype %s, got %s" % (dtype, t.dtype))
    return C.c_void_p(t.data_ptr())


def _check(status, where):
    if status != MG_OK:
        raise QSMGError(status, where)


class Context:
    """Owns one mg_ctx: a multigrid hierarchy for an nx*ny*nz-cell grid."""

    def __init__(self, nx, ny, nz, h, K, mu, bc=None, stz=None, precision=MG_FP64, nu1=2, nu2=2,
                 max_cycles=100, inner_cycles=0, flags=0, stream=None):
        import torch
        L = lib()
        self.shape = (nx, ny, nz)
        g = mg_grid(nx, ny, nz, h)
        m = mg_moduli(K, mu)
        o = mg_opts(precision, nu1, nu2, max_cycles, inner_cycles, flags)
        b = mg_bc(**bc) if isinstance(bc, dict) else bc
        z = stz_params(**stz) if isinstance(stz, dict) else stz
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h_ = C.c_void_p()
        st = L.mg_setup(C.byref(g), C.byref(m), C.byref(b) if b is not None else None,
                        C.byref(z) if z is not None else None, C.byref(o),
                        C.c_void_p(stream.cuda_stream), C.byref(h_))
        _check(st, "mg_setup")
        self.h = h_
        self.precision = precision

    def close(self):
        if getattr(self, "h", None):
            lib().mg_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def levels(self) -> int:
        return lib().mg_num_levels(self.h)

    def level_dims(self, level):
        d = (C.c_int * 3)()
        _check(lib().mg_level_dims(self.h, level, d), "mg_level_dims")
        return tuple(d)

    def level_stencil(self, level):
        import numpy as np
        S = np.zeros((27, 3, 3))
        _check(lib().mg_level_stencil(self.h, level, S.ctypes.data_as(C.POINTER(C.c_double))),
               "mg_level_stencil")
        return S

    def solve(self, rhs, v, tol=1e-10, raise_on_error=True):
        """mg_solve: v (in/out) and rhs are (3, nz+1, ny, nx) float64 CUDA tensors."""
        import torch
        s = mg_stats()
        st = lib().mg_solve(self.h, _ptr(rhs, torch.float64), _ptr(v, torch.float64), tol,
                            C.byref(s))
        if raise_on_error:
            _check(st, "mg_solve")
        return st, s

    def step(self, state: qs_state, dt, tol=1e-10, raise_on_error=True):
        s = mg_stats()
        st = lib().qs_step(self.h, C.byref(state), dt, tol, C.byref(s))
        if raise_on_error:
            _check(st, "qs_step")
        return st, s

    def run(self, state: qs_state, nsteps, dt, tol=1e-10, raise_on_error=True):
        """qs_run: nsteps projection steps in one call; returns (status, list
        of each step's mg_stats)."""
        n = int(nsteps)
        arr = (mg_stats * max(n, 1))()
        st = lib().qs_run(self.h, C.byref(state), n, dt, tol, arr)
        if raise_on_error:
            _check(st, "qs_run")
        return st, [arr[i] for i in range(n)]

    def explicit_step(self, state: qs_state, dt, rho, kappa, nsteps=1, raise_on_error=True):
        """qs_explicit_step: nsteps steps of the explicit method (section 3.2)."""
        st = lib().qs_explicit_step(self.h, C.byref(state), dt, rho, kappa, int(nsteps))
        if raise_on_error:
            _check(st, "qs_explicit_step")
        return st

    def step_adjoint(self, state: qs_state, dt, vbar, sigbar, chibar, tol=1e-10, work_weight=1.0,
                     raise_on_error=True):
        """qs_step_adjoint: vbar, sigbar, chibar (float64 CUDA tensors) hold the
        adjoints of the step's output on entry and of its input on return."""
        s = mg_stats()
        st = lib().qs_step_adjoint(self.h, C.byref(state), dt, tol, work_weight, _ptr(vbar),
                                   _ptr(sigbar), _ptr(chibar), C.byref(s))
        if raise_on_error:
            _check(st, "qs_step_adjoint")
        return st, s

    def plastic_work_grad(self, state: qs_state, nsteps, dt, chibar, tol=1e-10,
                          checkpoint_every=8, raise_on_error=True):
        """qs_plastic_work_grad: returns (status, W, stats); chibar receives
        dW/dchi0 and state is advanced by nsteps steps."""
        s = mg_stats()
        W = C.c_double()
        st = lib().qs_plastic_work_grad(self.h, C.byref(state), int(nsteps), dt, tol,
                                        int(checkpoint_every), _ptr(chibar), C.byref(W),
                                        C.byref(s))
        if raise_on_error:
            _check(st, "qs_plastic_work_grad")
        return st, W.value, s

    def checkpoint_size(self, nsteps, checkpoint_every):
        """Doubles of the checkpoint buffer qs_plastic_work fills."""
        nx, ny, nz = self.shape
        seg = min(int(checkpoint_every), int(nsteps))
        ncp = (int(nsteps) + seg - 1) // seg
        return ncp * (3 * (nz + 1) * ny * nx + 7 * nz * ny * nx)

    def plastic_work(self, state: qs_state, nsteps, dt, tol=1e-10, checkpoint_every=8,
                     checkpoints=None, raise_on_error=True):
        """qs_plastic_work: returns (status, W, stats); state is advanced by
        nsteps steps; checkpoints (float64 CUDA tensor of checkpoint_size
        doubles, or None) receives a copy of the state every checkpoint_every
        steps."""
        s = mg_stats()
        W = C.c_double()
        if checkpoints is not None and checkpoints.numel() < self.checkpoint_size(
                nsteps, checkpoint_every):
            raise ValueError("checkpoint buffer too small")
        st = lib().qs_plastic_work(self.h, C.byref(state), int(nsteps), dt, tol,
                                   int(checkpoint_every), _ptr(checkpoints), C.byref(W), C.byref(s))
        if raise_on_error:
            _check(st, "qs_plastic_work")
        return st, W.value, s

    def plastic_work_backward(self, checkpoints, t0, step0, nsteps, dt, chibar, tol=1e-10,
                              checkpoint_every=8, raise_on_error=True):
        """qs_plastic_work_backward: chibar receives dW/dchi0 from the
        checkpoints of a plastic_work call with the same arguments."""
        s = mg_stats()
        if checkpoints.numel() < self.checkpoint_size(nsteps, checkpoint_every):
            raise ValueError("checkpoint buffer too small")
        st = lib().qs_plastic_work_backward(self.h, _ptr(checkpoints), float(t0), int(step0),
                                            int(nsteps), dt, tol, int(checkpoint_every),
                                            _ptr(chibar), C.byref(s))
        if raise_on_error:
            _check(st, "qs_plastic_work_backward")
        return st, s

    def profile(self, enable=True):
        _check(lib().mg_profile(self.h, int(enable)), "mg_profile")

    def profile_read(self):
        ms, sw, la = C.c_double(), C.c_long(), C.c_long()
        _check(lib().mg_profile_read(self.h, C.byref(ms), C.byref(sw), C.byref(la)),
               "mg_profile_read")
        return ms.value, sw.value, la.value

    # -- component entry points (parity tests) --
    def residual(self, level, b, x, r):
        import torch
        _check(lib().mg_residual(self.h, level, _ptr(b, torch.float64), _ptr(x, torch.float64),
                                 _ptr(r, torch.float64)), "mg_residual")

    def residual32(self, level, b, x, r):
        import torch
        _check(lib().mg_residual32(self.h, level, _ptr(b, torch.float32), _ptr(x, torch.float32),
                                   _ptr(r, torch.float32)), "mg_residual32")

    def residual_restrict32(self, level, b, x, bc):
        """mg_residual_restrict32: bc = T^T (b - A x) in FP32 (float32 tensors)."""
        import torch
        _check(lib().mg_residual_restrict32(self.h, level, _ptr(b, torch.float32),
                                            _ptr(x, torch.float32), _ptr(bc, torch.float32)),
               "mg_residual_restrict32")

    def smooth(self, level, b, x, nsweeps, descending=False):
        import torch
        prec = MG_FP64 if x.dtype == torch.float64 else MG_MIXED
        _check(lib().mg_smooth(self.h, level, _ptr(b, x.dtype), _ptr(x, x.dtype), nsweeps,
                               int(descending), prec), "mg_smooth")

    def restrict(self, level, r, bc):
        import torch
        _check(lib().mg_restrict(self.h, level, _ptr(r, torch.float64), _ptr(bc, torch.float64)),
               "mg_restrict")

    def prolong_add(self, level, xc, x):
        import torch
        _check(lib().mg_prolong_add(self.h, level, _ptr(xc, torch.float64), _ptr(x, torch.float64)),
               "mg_prolong_add")

    def vcycle(self, b, x):
        import torch
        _check(lib().mg_vcycle(self.h, _ptr(b, torch.float64), _ptr(x, torch.float64)), "mg_vcycle")

    def stress_predict(self, v, sig, chi, dt, sig_star, dpl, sbar):
        _check(lib().qs_stress_predict(self.h, _ptr(v), _ptr(sig), _ptr(chi), dt, _ptr(sig_star),
                                       _ptr(dpl), _ptr(sbar)), "qs_stress_predict")

    def chi_update(self, sig, chi, dpl, sbar, dt, chi_new):
        _check(lib().qs_chi_update(self.h, _ptr(sig), _ptr(chi), _ptr(dpl), _ptr(sbar), dt,
                                   _ptr(chi_new)), "qs_chi_update")

    def rhs(self, sig_star, dt, b):
        _check(lib().qs_rhs(self.h, _ptr(sig_star), dt, _ptr(b)), "qs_rhs")

    def stress_correct(self, v, sig_star, dt, sig):
        _check(lib().qs_stress_correct(self.h, _ptr(v), _ptr(sig_star), dt, _ptr(sig)),
               "qs_stress_correct")

    def wall_fill(self, v, t):
        _check(lib().qs_wall_fill(self.h, _ptr(v), t), "qs_wall_fill")


def plastic_work(ctx: "Context", v0, sigma0, chi0, t0, nsteps, dt, tol=1e-10, checkpoint_every=8):
    """The plastic work W of nsteps projection steps from (v0, sigma0, chi0)
    at time t0, differentiable with respect to chi0 (a torch.autograd.Function
    over qs_plastic_work / qs_plastic_work_backward; the inputs are copied,
    not advanced).  The forward pass runs the steps only, keeping checkpoints
    when chi0 requires a gradient; the backward pass runs the reverse sweep
    from them."""
    return _PlasticWork.apply(chi0, ctx, v0, sigma0, t0, nsteps, dt, tol, checkpoint_every)


def _plastic_work_class():
    import torch

    class PlasticWork(torch.autograd.Function):
        @staticmethod
        def forward(fctx, chi0, ctx, v0, sigma0, t0, nsteps, dt, tol, checkpoint_every):
            # the library works on ctx.stream: order it after the work that
            # produced the inputs and the copies below on the current stream
            with torch.cuda.stream(ctx.stream):
                ctx.stream.wait_stream(torch.cuda.current_stream(chi0.device))
                v = v0.detach().clone()
                sig = sigma0.detach().clone()
                chi = chi0.detach().clone()
                cp = None
                if fctx.needs_input_grad[0]:
                    cp = torch.empty(ctx.checkpoint_size(nsteps, checkpoint_every),
                                     dtype=torch.float64, device=chi0.device)
                state = make_state(v, sig, chi, t0)
                _, W, _ = ctx.plastic_work(state, nsteps, dt, tol=tol,
                                           checkpoint_every=checkpoint_every, checkpoints=cp)
            fctx.lib_ctx = ctx
            fctx.args = (t0, nsteps, dt, tol, checkpoint_every)
            if cp is not None:
                fctx.save_for_backward(cp)
            return torch.tensor(W, dtype=torch.float64, device=chi0.device)

        @staticmethod
        def backward(fctx, gW):
            (cp,) = fctx.saved_tensors
            ctx = fctx.lib_ctx
            t0, nsteps, dt, tol, every = fctx.args
            with torch.cuda.stream(ctx.stream):
                ctx.stream.wait_stream(torch.cuda.current_stream(cp.device))
                grad = torch.empty(ctx.shape[::-1], dtype=torch.float64, device=cp.device)
                ctx.plastic_work_backward(cp, t0, 0, nsteps, dt, grad, tol=tol,
                                          checkpoint_every=every)
            torch.cuda.current_stream(cp.device).wait_stream(ctx.stream)
            return (gW * grad,) + (None,) * 8

    return PlasticWork


class _Lazy:
    def __init__(self, make):
        self._make, self._cls = make, None

    def apply(self, *args):
        if self._cls is None:
            self._cls = self._make()
        return self._cls.apply(*args)


_PlasticWork = _Lazy(_plastic_work_class)


def launch_count() -> int:
    """Kernels the library has launched since it was loaded."""
    return lib().mg_launch_count()


def make_state(v, sigma, chi, t=0.0, step=0) -> qs_state:
    """qs_state over caller-owned CUDA tensors (kept alive by the caller)."""
    import torch
    return qs_state(_ptr(v, torch.float64), _ptr(sigma, torch.float64), _ptr(chi, torch.float64),
                    t, step)
