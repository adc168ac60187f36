"""Pins of the gradient oracle (``oracle/adjoint.py``): its PyTorch restatement
of each step equation against the C oracle, the whole step against the C
oracle's ``qs_step``, and dW/dchi^0 of the plastic work against central
finite differences of the C oracle's own forward run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from oracle import adjoint as A  # noqa: E402
from paper_1904_03808_gb300 import inputs as I  # noqa: E402

MU = I.TABLE1["mu"]
LAM = I.lame_lambda(I.TABLE1["K"], MU)


def rel(a, b):
    return np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel())


def _state(n=8, nz=None, preload=1.2e9, steps=10, seed=3):
    w = I.Workload(n, steps=steps, preload=preload, chi_mean=600.0, chi_std=30.0, lc_cells=2.0,
                   seed=seed, nz=nz)
    v, sig, chi, t = w.initial_state()
    return w, v, sig, chi, t


def _perturbed(w, v, sig, seed=9):
    # a velocity field with every gradient component present, and a stress
    # with every component present, so that each term of Eq. 27 is exercised
    # (the preload halved in one half of the box keeps those cells elastic)
    rng = np.random.default_rng(seed)
    v = v + 1e-3 * w.U_B * rng.standard_normal(v.shape)
    sig = sig + 1e8 * rng.standard_normal(sig.shape)
    sig[4, :, :, : w.nx // 2] *= 0.5
    return v, sig


def test_step_pieces_match_the_c_oracle():
    w, v, sig, chi, t = _state(8, nz=6)
    v, sig = _perturbed(w, v, sig)
    p = O.STZ(**w.stz)
    ss_c, D_c, sb_c = O.stress_star(v, sig, chi, w.h, w.dt, MU, p)
    T = torch.from_numpy
    ss, D, sb = A.stress_star(T(v), T(sig), T(chi), w.h, w.dt, MU, p)
    assert (D_c > 0).sum() > 10 and (D_c == 0).sum() > 10  # both sides of yield
    assert rel(ss.numpy(), ss_c) <= 1e-14
    assert rel(D.numpy(), D_c) <= 1e-13
    assert rel(sb.numpy(), sb_c) <= 1e-14
    L_c = O.cell_gradient(v, w.h)
    L = A.cell_gradient(T(v), w.h).permute(2, 3, 4, 0, 1).numpy()
    assert rel(L, L_c) <= 1e-14
    chi_c = O.chi_update(sig, chi, D_c, sb_c, w.h, w.dt, p)
    assert rel(A.chi_update(T(sig), T(chi), T(D_c), T(sb_c), w.h, w.dt, p).numpy(), chi_c) <= 1e-14
    b_c = O.div_rhs(ss_c, w.h, w.dt, MU)
    assert rel(A.div_rhs(T(ss_c), w.h, w.dt, MU).numpy(), b_c) <= 1e-14
    s1_c = O.stress_final(v, ss_c, w.h, w.dt, LAM, MU)
    assert rel(A.stress_final(T(v), T(ss_c), w.h, w.dt, LAM, MU).numpy(), s1_c) <= 1e-14


def test_whole_steps_match_the_c_oracle():
    w, v, sig, chi, t = _state(8)
    p = O.STZ(**w.stz)
    bc = O.BC(**w.bc_values())
    mg = O.MG(w.nx, w.ny, w.nz, LAM, MU)
    vt, st_, ct = (torch.from_numpy(a.copy()) for a in (v, sig, chi))
    for _ in range(3):
        s, _, _ = O.qs_step(mg, v, sig, chi, w.h, w.dt, LAM, MU, p, bc, t, tol=1e-13,
                            max_cycles=200)
        assert s == 0
        vt, st_, ct, work = A.step(mg, vt, st_, ct, w.h, w.dt, LAM, MU, p, bc, t)
        t += w.dt
        assert rel(vt.numpy(), v) <= 1e-11
        assert rel(st_.numpy(), sig) <= 1e-12
        assert rel(ct.numpy(), chi) <= 1e-14
        assert float(work) > 0.0


def _c_plastic_work(w, v, sig, chi, t, steps):
    # the objective from the C oracle's forward run: the D^pl and sbar of
    # each step's state, then the step itself
    p = O.STZ(**w.stz)
    bc = O.BC(**w.bc_values())
    mg = O.MG(w.nx, w.ny, w.nz, LAM, MU)
    v, sig, chi = v.copy(), sig.copy(), chi.copy()
    W = 0.0
    for _ in range(steps):
        _, D, sb = O.stress_star(v, sig, chi, w.h, w.dt, MU, p)
        W += 2.0 * float(np.sum(D * sb)) * w.dt * w.h ** 3
        s, _, _ = O.qs_step(mg, v, sig, chi, w.h, w.dt, LAM, MU, p, bc, t, tol=1e-13,
                            max_cycles=200)
        assert s == 0
        t += w.dt
    return W


def _grad(w, v, sig, chi, t, steps):
    return A.plastic_work_gradient((w.nx, w.ny, w.nz), v, sig, chi, w.h, w.dt, LAM, MU,
                                   O.STZ(**w.stz), O.BC(**w.bc_values()), t, steps)


def test_plastic_work_gradient_against_central_differences():
    """Directional derivative along a random chi perturbation, and three
    single cells, against central differences of the C oracle's forward run:
    the difference error falls as eps^2, and the Richardson combination of
    two step sizes agrees to 1e-6."""
    steps = 3
    w, v, sig, chi, t = _state(8)
    W, g = _grad(w, v, sig, chi, t, steps)
    assert W == pytest.approx(_c_plastic_work(w, v, sig, chi, t, steps), rel=1e-12)

    def central(d, eps):
        return (_c_plastic_work(w, v, sig, chi + eps * d, t, steps) -
                _c_plastic_work(w, v, sig, chi - eps * d, t, steps)) / (2 * eps)

    dirn = np.random.default_rng(4).standard_normal(chi.shape)
    want = float(np.sum(g * dirn))
    f1, f2 = central(dirn, 1.0), central(dirn, 0.5)
    e1, e2 = abs(f1 - want) / abs(want), abs(f2 - want) / abs(want)
    assert 0.2 < e2 / e1 < 0.3, (e1, e2)  # second order in eps
    assert (4 * f2 - f1) / 3 == pytest.approx(want, rel=1e-6)
    for cell in ((0, 0, 0), (3, 5, 2), (7, 1, 6)):
        e = np.zeros_like(chi)
        e[cell] = 1.0
        f1, f2 = central(e, 1.0), central(e, 0.5)
        assert (4 * f2 - f1) / 3 == pytest.approx(g[cell], rel=1e-6), cell


def test_gradient_reaches_later_steps_through_the_solve():
    """chi^0 acts on step 2's plastic work through sigma^1, hence through the
    projection solve of step 1 and its adjoint: dropping the adjoint solve
    (a planted omission) changes the gradient."""
    w, v, sig, chi, t = _state(8)
    _, g = _grad(w, v, sig, chi, t, 2)
    back = A._Solve.backward
    try:
        A._Solve.backward = staticmethod(lambda ctx, gv: (torch.zeros_like(gv), None, None, None))
        _, g0 = _grad(w, v, sig, chi, t, 2)
    finally:
        A._Solve.backward = back
    assert rel(g0, g) > 1e-6


def test_gradient_vanishes_below_yield():
    """No cell above yield: D^pl = 0 everywhere, W = 0, and the subgradient
    taken at the yield cut-off is 0."""
    w, v, sig, chi, t = _state(8, preload=0.0)
    W, g = _grad(w, v, sig, chi, t, 2)
    assert W == 0.0
    assert not np.any(g)


def test_solve_adjoint_is_the_same_solve():
    """<solve(a), b> = <a, solve(b)> with zero walls: the backward pass of the
    wrapped solve is exact for the symmetric scaled operator."""
    rng = np.random.default_rng(6)
    n = 8
    mg = O.MG(n, n, n, LAM, MU)
    a, b = (rng.standard_normal((3, n + 1, n, n)) for _ in range(2))
    for x in (a, b):
        x[:, [0, n]] = 0.0
    za, zb = np.zeros_like(a), np.zeros_like(b)
    mg.solve(a, za, tol=1e-14, max_cycles=400)
    mg.solve(b, zb, tol=1e-14, max_cycles=400)
    assert float(np.sum(za * b)) == pytest.approx(float(np.sum(a * zb)), rel=1e-12)
    bt = torch.from_numpy(a.copy()).requires_grad_(True)
    out = A._Solve.apply(bt, torch.zeros_like(bt), mg, 1e-14)
    (gb,) = torch.autograd.grad((out * torch.from_numpy(b)).sum(), bt)
    assert rel(gb.numpy()[:, 1:n], zb[:, 1:n]) <= 1e-12
