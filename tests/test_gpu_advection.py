"""GPU parity of the optional stress advection (MG_FLAG_ADVECT_STRESS):
sigma* of Eq. (27) plus -(u.grad) sigma (ENO, Eq. 33), through the C ABI,
against the oracle's predictor and whole steps with the same option.

States have the STZ rate active and velocity noise of both signs, so every
ENO branch is taken.  Whole steps use a fixed cycle count on both sides
(tol = 0), so the bar is FP64 rounding: 1e-12 element-wise and norm-wise.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_1904_03808_gb300 import Context, inputs as I, make_state  # noqa: E402
from paper_1904_03808_gb300 import binding  # noqa: E402

MU = I.TABLE1["mu"]
K = I.TABLE1["K"]
LAM = I.lame_lambda(K, MU)
TOL64 = 1e-12
ADV = binding.MG_FLAG_ADVECT_STRESS


def g(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def c(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    d = (np.asarray(a) - np.asarray(b)).ravel()
    b = np.asarray(b).ravel()
    return max(np.linalg.norm(d) / max(np.linalg.norm(b), 1e-300),
               np.abs(d).max(initial=0.0) / max(np.abs(b).max(initial=0.0), 1e-300))


def _state(n, nz=None, seed=3):
    w = I.Workload(n, steps=10, strain=0.02, preload=1.2e9, nz=nz, seed=seed)
    v, sig, chi, t = w.initial_state()
    rng = np.random.default_rng(seed)
    v[:, 1:w.nz] += 1e-2 * w.U_B * rng.normal(size=v[:, 1:w.nz].shape)
    sig += 5e7 * rng.normal(size=sig.shape)
    return w, v, sig, chi, t


def _ctx(w, flags, **kw):
    return Context(w.nx, w.ny, w.nz, w.h, K, MU, bc=w.bc_values(), stz=w.stz, flags=flags, **kw)


@pytest.mark.parametrize("n,nz", [(16, None), (24, 8), (32, 16)])
def test_stress_predictor_with_advection(n, nz):
    w, v, sig, chi, t = _state(n, nz)
    p = O.STZ(**w.stz)
    ss_o, D_o, sb_o = O.stress_star(v, sig, chi, w.h, w.dt, MU, p, advect=True)
    plain = O.stress_star(v, sig, chi, w.h, w.dt, MU, p)[0]
    assert rel(ss_o, plain) > 1e-9  # the term is far above the bar
    ctx = _ctx(w, ADV)
    vg, sg, cg = g(v), g(sig), g(chi)
    ss, D, sb = torch.zeros_like(sg), torch.zeros_like(cg), torch.zeros_like(cg)
    ctx.stress_predict(vg, sg, cg, w.dt, ss, D, sb)
    assert rel(c(ss), ss_o) <= TOL64
    assert rel(c(D), D_o) <= TOL64 and rel(c(sb), sb_o) <= TOL64
    ctx.close()


@pytest.mark.parametrize("n,nz,steps", [(16, None, 3), (24, 8, 3)])
def test_steps_with_advection(n, nz, steps):
    """Several steps in one qs_run (the correction/predictor fusion with the
    advection pass after each predictor) against the oracle's steps."""
    w, v, sig, chi, t = _state(n, nz)
    shape = (w.nx, w.ny, w.nz)
    mg = O.MG(*shape, LAM, MU)
    p = O.STZ(**w.stz)
    bc = O.BC(**w.bc_values())
    cyc = 10
    v0, s0, c0, t0 = v.copy(), sig.copy(), chi.copy(), t
    vg, sg, cg = g(v), g(sig), g(chi)
    state = make_state(vg, sg, cg, t)
    for _ in range(steps):
        st, n_o, _ = O.qs_step(mg, v, sig, chi, w.h, w.dt, LAM, MU, p, bc, t, tol=0.0,
                               max_cycles=cyc, advect=True)
        assert st == 0 and n_o == cyc
        t += w.dt
    ctx = _ctx(w, ADV, max_cycles=cyc)
    st, stats = ctx.run(state, steps, w.dt, tol=0.0)
    assert st == 0 and [s_.cycles for s_ in stats] == [cyc] * steps
    assert rel(c(vg), v) <= TOL64
    assert rel(c(sg), sig) <= TOL64
    assert rel(c(cg), chi) <= TOL64
    ctx.close()
    # the same steps without the option end far outside the bar
    for _ in range(steps):
        O.qs_step(mg, v0, s0, c0, w.h, w.dt, LAM, MU, p, bc, t0, tol=0.0, max_cycles=cyc)
        t0 += w.dt
    assert rel(s0, sig) > 1e-9 and rel(v0, v) > 1e-9


def test_reverse_mode_rejects_advection():
    w, v, sig, chi, t = _state(16)
    ctx = _ctx(w, ADV)
    vg, sg, cg = g(v), g(sig), g(chi)
    state = make_state(vg, sg, cg, t)
    vb, sb_, cb = torch.zeros_like(vg), torch.zeros_like(sg), torch.zeros_like(cg)
    st, _ = ctx.step_adjoint(state, w.dt, vb, sb_, cb, raise_on_error=False)
    assert st == binding.MG_ERR_ARG
    st, _, _ = ctx.plastic_work_grad(state, 2, w.dt, torch.zeros_like(cg), raise_on_error=False)
    assert st == binding.MG_ERR_ARG
    assert b"advection" in binding.lib().mg_last_error()
    ctx.close()
