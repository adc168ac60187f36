"""GPU parity of the reverse mode: qs_step_adjoint, qs_plastic_work(_backward,
_grad) and the plastic_work autograd Function, called through the C ABI,
against the gradient oracle (autograd of the step equations restated in
FP64 PyTorch CPU operations, oracle/adjoint.py) and against central
differences of the GPU's own forward run.

Tolerances (derived from the arithmetic):
- one adjoint step, FP64, adjoint solve to 1e-13: 1e-10 relative (the
  solve's truncation, times the operator's condition number at these sizes,
  stays below that; every other operation is FP64 rounding);
- dW/dchi0 over several steps, FP64, solves to 1e-12: 1e-9 relative (the
  forward states differ from the oracle's, solved to 1e-13, by ~1e-11
  relative; the STZ rate's exponential sensitivity to sbar turns that into
  ~1e-10 relative in D^pl);
- mixed precision, solves to 1e-11: 1e-7 relative;
- central differences with step eps: Richardson (4 f(eps/2) - f(eps)) / 3
  to 1e-6 relative at small sizes; at the 64^3 x 40-step configuration with
  eps = 1e-3 K the difference quotient's rounding floor (a few ulps of W over
  2 eps) is the bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from oracle import adjoint as A  # noqa: E402
from paper_1904_03808_gb300 import (MG_FP64, MG_MIXED, Context, inputs as I,  # noqa: E402
                                    make_state, plastic_work)

MU = I.TABLE1["mu"]
K = I.TABLE1["K"]
LAM = I.lame_lambda(K, MU)


def g(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def c(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    """max of the norm-wise and the element-wise relative difference."""
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    d = (a - b).ravel()
    nb = max(np.linalg.norm(b.ravel()), 1e-300)
    mb = max(np.abs(b).max(), 1e-300)
    return max(np.linalg.norm(d) / nb, np.abs(d).max() / mb)


def _state(n, nz=None, ny=None, preload=1.2e9, steps=10, strain=0.02, seed=3, lc=2.0):
    w = I.Workload(n, steps=steps, strain=strain, preload=preload, chi_mean=600.0, chi_std=30.0,
                   lc_cells=lc, seed=seed, nz=nz)
    if ny is not None:
        w.ny = ny
    v, sig, chi, t = w.initial_state()
    return w, v, sig, chi, t


def _perturbed(w, v, sig, seed=9):
    # every velocity-gradient and stress component present, cells on both
    # sides of yield (the preload halved in one half of the box)
    rng = np.random.default_rng(seed)
    v = v + 1e-3 * w.U_B * rng.standard_normal(v.shape)
    sig = sig + 1e8 * rng.standard_normal(sig.shape)
    sig[4, :, :, : w.nx // 2] *= 0.5
    return v, sig


def _dev_state(v, sig, chi, t):
    """Device copies of a state and the qs_state over them (the state holds
    raw pointers only, so the tensors are returned to be kept alive)."""
    vg, sg, cg = g(v), g(sig), g(chi)
    return (vg, sg, cg), make_state(vg, sg, cg, t)


def _ctx(w, precision=MG_FP64, max_cycles=120):
    return Context(w.nx, w.ny, w.nz, w.h, K, MU, bc=w.bc_values(), stz=w.stz,
                   precision=precision, max_cycles=max_cycles, inner_cycles=0)


@pytest.mark.parametrize("shape", [(8, 8, 6), (16, 8, 8), (8, 8, 2)])
@pytest.mark.parametrize("path", ["v", "sigma", "chi", "work", "all"])
def test_step_adjoint_matches_autograd(shape, path):
    """One qs_step_adjoint against autograd of the oracle's step for random
    output adjoints, one path of the step at a time (velocity, stress, chi,
    plastic work) and all together; interior velocity planes (the walls are
    prescribed and carry no adjoint)."""
    nx, ny, nz = shape
    w, v, sig, chi, t = _state(nx, nz=nz, ny=ny)
    v, sig = _perturbed(w, v, sig)
    p, bc = O.STZ(**w.stz), O.BC(**w.bc_values())
    _, D, _ = O.stress_star(v, sig, chi, w.h, w.dt, MU, p)
    assert (D > 0).sum() > 10 and (D == 0).sum() > 10  # both sides of yield
    rng = np.random.default_rng(21)
    vbar = rng.standard_normal(v.shape) * (path in ("v", "all"))
    vbar[:, [0, nz]] = 0.0
    sigbar = rng.standard_normal(sig.shape) * (path in ("sigma", "all"))
    chibar = rng.standard_normal(chi.shape) * (path in ("chi", "all"))
    ww = 0.7 if path in ("work", "all") else 0.0

    T = torch.from_numpy
    vt, st_, ct = (T(a.copy()).requires_grad_(True) for a in (v, sig, chi))
    mg = O.MG(nx, ny, nz, LAM, MU)
    v1, s1, c1, work = A.step(mg, vt, st_, ct, w.h, w.dt, LAM, MU, p, bc, t, tol=1e-13)
    loss = (v1 * T(vbar)).sum() + (s1 * T(sigbar)).sum() + (c1 * T(chibar)).sum() + ww * work
    gv, gs, gc = torch.autograd.grad(loss, (vt, st_, ct), allow_unused=True)
    gv = np.zeros_like(v) if gv is None else gv.numpy()
    gs = np.zeros_like(sig) if gs is None else gs.numpy()
    gc = np.zeros_like(chi) if gc is None else gc.numpy()

    ctx = _ctx(w)
    vg, sg, cg = g(v), g(sig), g(chi)
    state = make_state(vg, sg, cg, t)
    vb, sb, cb = g(vbar), g(sigbar), g(chibar)
    st, s = ctx.step_adjoint(state, w.dt, vb, sb, cb, tol=1e-13, work_weight=ww)
    assert st == 0
    # the forward state is not modified
    assert np.array_equal(c(vg), v) and np.array_equal(c(sg), sig) and np.array_equal(c(cg), chi)
    gvi = gv[:, 1:nz]
    if np.any(gvi):
        assert rel(c(vb)[:, 1:nz], gvi) <= 1e-10, path
    else:
        assert not np.any(c(vb)[:, 1:nz])
    assert not np.any(c(vb)[:, [0, nz]])
    assert rel(c(sb), gs) <= 1e-10, path
    assert rel(c(cb), gc) <= 1e-10, path
    ctx.close()


def _oracle_grad(w, v, sig, chi, t, steps):
    return A.plastic_work_gradient((w.nx, w.ny, w.nz), v, sig, chi, w.h, w.dt, LAM, MU,
                                   O.STZ(**w.stz), O.BC(**w.bc_values()), t, steps)


@pytest.mark.parametrize("precision,every,tol,bar", [(MG_FP64, 1, 1e-12, 1e-9),
                                                     (MG_FP64, 2, 1e-12, 1e-9),
                                                     (MG_FP64, 8, 1e-12, 1e-9),
                                                     (MG_MIXED, 2, 1e-11, 1e-7)])
def test_plastic_work_gradient_matches_oracle(precision, every, tol, bar):
    """dW/dchi0 of 5 steps at 16 x 8 x 8 cells (ragged last segment for
    checkpoints every 2), FP64 and mixed, against the oracle gradient; the
    state is advanced as by 5 qs_step calls."""
    steps = 5
    w, v, sig, chi, t = _state(16, nz=8, ny=8)
    W_o, g_o = _oracle_grad(w, v, sig, chi, t, steps)
    assert W_o > 0 and np.abs(g_o).max() > 0
    ctx = _ctx(w, precision)
    vg, sg, cg = g(v), g(sig), g(chi)
    state = make_state(vg, sg, cg, t)
    grad = torch.full_like(cg, float("nan"))
    st, W, s = ctx.plastic_work_grad(state, steps, w.dt, grad, tol=tol, checkpoint_every=every)
    assert st == 0 and state.step == steps
    assert W == pytest.approx(W_o, rel=bar)
    assert rel(c(grad), g_o) <= bar, rel(c(grad), g_o)
    # the advanced state: the oracle's forward run to the same tolerance
    mg = O.MG(w.nx, w.ny, w.nz, LAM, MU)
    p, bc = O.STZ(**w.stz), O.BC(**w.bc_values())
    tt = t
    for _ in range(steps):
        O.qs_step(mg, v, sig, chi, w.h, w.dt, LAM, MU, p, bc, tt, tol=1e-13, max_cycles=400)
        tt += w.dt
    assert rel(c(cg), chi) <= bar and rel(c(sg), sig) <= bar
    ctx.close()


def test_split_forward_backward_equals_combined():
    """qs_plastic_work (checkpoints into a caller buffer) then
    qs_plastic_work_backward gives bitwise the W and dW/dchi0 of
    qs_plastic_work_grad; a forward call without checkpoints gives the same
    W and final state."""
    steps, every = 7, 3
    w, v, sig, chi, t = _state(16, nz=8)
    ctx = _ctx(w)
    outs = []
    for mode in ("grad", "split", "forward"):
        vg, sg, cg = g(v), g(sig), g(chi)
        state = make_state(vg, sg, cg, t)
        grad = torch.zeros_like(cg)
        if mode == "grad":
            _, W, _ = ctx.plastic_work_grad(state, steps, w.dt, grad, tol=1e-12,
                                            checkpoint_every=every)
        elif mode == "split":
            cp = torch.full((ctx.checkpoint_size(steps, every),), float("nan"),
                            dtype=torch.float64, device="cuda")
            _, W, _ = ctx.plastic_work(state, steps, w.dt, tol=1e-12, checkpoint_every=every,
                                       checkpoints=cp)
            ctx.plastic_work_backward(cp, t, 0, steps, w.dt, grad, tol=1e-12,
                                      checkpoint_every=every)
        else:
            _, W, _ = ctx.plastic_work(state, steps, w.dt, tol=1e-12, checkpoint_every=every)
            grad = None
        outs.append((W, None if grad is None else c(grad), c(vg), c(sg), c(cg), state.t))
    (W0, g0, *s0), (W1, g1, *s1), (W2, _, *s2) = outs
    assert W0 == W1 == W2
    assert np.array_equal(g0, g1)
    for a, b, d in zip(s0, s1, s2):
        assert np.array_equal(a, b) and np.array_equal(a, d)
    ctx.close()


def _gpu_work(ctx, w, v, sig, chi, t, steps, tol):
    keep, state = _dev_state(v, sig, chi, t)
    _, W, _ = ctx.plastic_work(state, steps, w.dt, tol=tol, checkpoint_every=steps)
    return W


def test_gradient_against_central_differences_small():
    """Three single cells and a random direction at 16 x 8 x 8, 4 steps, FP64:
    Richardson-combined central differences of the GPU forward run."""
    steps = 4
    w, v, sig, chi, t = _state(16, nz=8, ny=8)
    ctx = _ctx(w)
    keep, state = _dev_state(v, sig, chi, t)
    grad = torch.zeros((w.nz, w.ny, w.nx), dtype=torch.float64, device="cuda")
    ctx.plastic_work_grad(state, steps, w.dt, grad, tol=1e-13, checkpoint_every=2)
    gr = c(grad)

    def central(d, eps):
        return (_gpu_work(ctx, w, v, sig, chi + eps * d, t, steps, 1e-13) -
                _gpu_work(ctx, w, v, sig, chi - eps * d, t, steps, 1e-13)) / (2 * eps)

    # along a direction that moves every cell the Richardson combination
    # keeps an eps^4 term of ~2e-6 relative at eps = 1 K: steps of 0.5 and
    # 0.25 K bring it 16 times lower
    dirn = np.random.default_rng(4).standard_normal(chi.shape)
    want = float(np.sum(gr * dirn))
    f1, f2 = central(dirn, 0.5), central(dirn, 0.25)
    assert (4 * f2 - f1) / 3 == pytest.approx(want, rel=1e-6)
    for cell in ((0, 0, 0), (3, 5, 2), (7, 1, 14)):
        e = np.zeros_like(chi)
        e[cell] = 1.0
        f1, f2 = central(e, 1.0), central(e, 0.5)
        assert (4 * f2 - f1) / 3 == pytest.approx(gr[cell], rel=1e-6, abs=1e-6 * np.abs(gr).max())
    ctx.close()


def test_autograd_function_equals_c_gradient():
    """plastic_work(...).backward() gives the C gradient; a call whose chi0
    needs no gradient returns the same W; the inputs are not advanced."""
    steps, every = 4, 2
    w, v, sig, chi, t = _state(16, nz=8)
    ctx = _ctx(w)
    v0, s0 = g(v), g(sig)
    chi0 = g(chi).requires_grad_(True)
    W = plastic_work(ctx, v0, s0, chi0, t, steps, w.dt, tol=1e-12, checkpoint_every=every)
    (3.0 * W).backward()
    keep, state = _dev_state(v, sig, chi, t)
    grad = torch.zeros_like(chi0)
    _, Wc, _ = ctx.plastic_work_grad(state, steps, w.dt, grad, tol=1e-12, checkpoint_every=every)
    assert float(W) == Wc
    assert torch.equal(chi0.grad, 3.0 * grad)
    W2 = plastic_work(ctx, v0, s0, g(chi), t, steps, w.dt, tol=1e-12, checkpoint_every=every)
    assert float(W2) == Wc and not W2.requires_grad
    assert np.array_equal(c(v0), v) and np.array_equal(c(chi0), chi)
    ctx.close()


def test_config4_gradient_64_cubed_40_steps():
    """The differentiation workload: 64^3 cells, 40 FP64 steps of simple shear
    from an STZ-active preload, dW/dchi0 with checkpoints every 8 steps,
    against central differences with eps = 1e-3 K of the GPU forward run on
    16 random cells (seed 4).  The solves run to 1e-13, so the forward map is
    smooth in chi0 to rounding; the bound is the difference quotient's
    rounding floor, 64 ulps of W over 2 eps, plus 1e-6 relative."""
    steps, every, eps = 40, 8, 1e-3
    w, v, sig, chi, t = _state(64, steps=steps, seed=4, lc=4.0)
    ctx = _ctx(w)
    keep, state = _dev_state(v, sig, chi, t)
    grad = torch.zeros((w.nz, w.ny, w.nx), dtype=torch.float64, device="cuda")
    _, W, _ = ctx.plastic_work_grad(state, steps, w.dt, grad, tol=1e-13, checkpoint_every=every)
    gr = c(grad)
    assert W > 0 and np.isfinite(gr).all()
    floor = 64 * np.finfo(np.float64).eps * W / (2 * eps)
    rng = np.random.default_rng(4)
    cells = [tuple(int(rng.integers(0, m)) for m in chi.shape) for _ in range(16)]
    for cell in cells:
        e = np.zeros_like(chi)
        e[cell] = eps
        fd = (_gpu_work(ctx, w, v, sig, chi + e, t, steps, 1e-13) -
              _gpu_work(ctx, w, v, sig, chi - e, t, steps, 1e-13)) / (2 * eps)
        assert abs(fd - gr[cell]) <= 1e-6 * abs(gr[cell]) + floor, (cell, fd, gr[cell], floor)
    ctx.close()


def test_config4_gradient_matches_oracle_64_cubed():
    """dW/dchi0 at 64^3 over 8 FP64 steps (checkpoints every 3: a ragged last
    segment) against the oracle gradient."""
    steps = 8
    w, v, sig, chi, t = _state(64, steps=40, seed=4, lc=4.0)
    W_o, g_o = _oracle_grad(w, v, sig, chi, t, steps)
    ctx = _ctx(w)
    keep, state = _dev_state(v, sig, chi, t)
    grad = torch.zeros((w.nz, w.ny, w.nx), dtype=torch.float64, device="cuda")
    _, W, _ = ctx.plastic_work_grad(state, steps, w.dt, grad, tol=1e-12, checkpoint_every=3)
    assert W == pytest.approx(W_o, rel=1e-9)
    assert rel(c(grad), g_o) <= 1e-9, rel(c(grad), g_o)
    ctx.close()
