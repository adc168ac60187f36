"""GPU parity of the explicit method (section 3.2: forward Euler of Eqs.
24-26 with ENO advection, Eq. 33) through the C ABI (qs_explicit_step)
against the oracle's step on the same seeded states: element-wise and
norm-wise to 1e-12 (FP64 rounding: the two sides sum the same terms in
different orders; every ENO branch decision compares the same FP64 values).
The states carry an STZ-active stress, velocity noise with both signs and
kinks (so every ENO branch is taken), non-zero walls, nx != ny, and the
disc walls of section 5."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from paper_1904_03808_gb300 import MG_FP64, Context, inputs as I, make_state  # noqa: E402

MU = I.TABLE1["mu"]
K = I.TABLE1["K"]
LAM = I.lame_lambda(K, MU)
RHO = I.TABLE1["rho"]


def rel(a, b):
    d = (a - b).ravel()
    return max(np.linalg.norm(d) / max(np.linalg.norm(b.ravel()), 1e-300),
               np.abs(d).max() / max(np.abs(b).max(), 1e-300))


def _setup(nx, ny, nz, kind, seed=5):
    w = I.Workload(nx, steps=10, strain=0.02, preload=1.3e9, chi_mean=600.0, chi_std=30.0,
                   lc_cells=2.0, seed=seed, nz=nz, kind=kind)
    w.ny = ny
    if kind:
        w.omega = 2.0 * math.pi / (1.0e4 * w.ts)
    v, sig, chi, t = w.initial_state()
    rng = np.random.default_rng(seed)
    U = max(w.U_B, 1.0)
    v += 0.3 * U * rng.standard_normal(v.shape)
    sig += 5e7 * rng.standard_normal(sig.shape)
    # the explicit time step and damping of section 4: dt = t_s h^2 / (20 L^2),
    # kappa = kappa' h with kappa' = 4.8 L / t_s
    dt = w.ts * w.h * w.h / (20.0 * w.L * w.L)
    kappa = 4.8 * w.L / w.ts * w.h
    return w, v, sig, chi, t, dt, kappa


@pytest.mark.parametrize("shape,kind", [((16, 16, 8), 0), ((24, 16, 12), 0), ((16, 16, 16), 1)])
def test_explicit_steps_match_oracle(shape, kind):
    nx, ny, nz = shape
    w, v, sig, chi, t, dt, kappa = _setup(nx, ny, nz, kind)
    p, bc = O.STZ(**w.stz), O.BC(**w.bc_values())
    _, D, _ = O.stress_star(v, sig, chi, w.h, dt, MU, p)
    assert (D > 0).mean() > 0.3  # the STZ rate is active
    ctx = Context(nx, ny, nz, w.h, K, MU, bc=w.bc_values(), stz=w.stz, precision=MG_FP64)
    vg, sg, cg = (torch.from_numpy(a.copy()).cuda() for a in (v, sig, chi))
    state = make_state(vg, sg, cg, t)
    for n in range(4):
        O.explicit_step(v, sig, chi, w.h, dt, RHO, LAM, MU, kappa, p, bc, t)
        t += dt
        ctx.explicit_step(state, dt, RHO, kappa, nsteps=1)
        assert state.step == n + 1 and abs(state.t - t) <= 1e-15 * abs(t)
        for got, want in ((vg, v), (sg, sig), (cg, chi)):
            assert rel(got.cpu().numpy(), want) <= 1e-12, n
    # several steps in one call equal as many single steps
    for _ in range(3):
        O.explicit_step(v, sig, chi, w.h, dt, RHO, LAM, MU, kappa, p, bc, t)
        t += dt
    ctx.explicit_step(state, dt, RHO, kappa, nsteps=3)
    for got, want in ((vg, v), (sg, sig), (cg, chi)):
        assert rel(got.cpu().numpy(), want) <= 1e-12
    ctx.close()


def test_explicit_step_arguments():
    nx = ny = nz = 8
    w, v, sig, chi, t, dt, kappa = _setup(nx, ny, nz, 0)
    ctx = Context(nx, ny, nz, w.h, K, MU, bc=w.bc_values(), stz=w.stz, precision=MG_FP64)
    vg, sg, cg = (torch.from_numpy(a.copy()).cuda() for a in (v, sig, chi))
    state = make_state(vg, sg, cg, t)
    assert ctx.explicit_step(state, dt, RHO, kappa, nsteps=0) == 0
    assert np.array_equal(vg.cpu().numpy(), v) and state.step == 0
    for args in ((-dt, RHO, kappa), (dt, 0.0, kappa), (dt, RHO, -1.0)):
        assert ctx.explicit_step(state, *args, nsteps=1, raise_on_error=False) == 1
    ctx.close()
    bare = Context(nx, ny, nz, w.h, K, MU, precision=MG_FP64)  # no walls / STZ parameters
    assert bare.explicit_step(state, dt, RHO, kappa, nsteps=1, raise_on_error=False) == 1
    bare.close()
