"""Pins of the oracle's optional stress advection in the quasi-static
predictor: Eq. (27) plus the -(u.grad) sigma term of the general
constitutive law of section 2, with u the mean corner velocity of the cell
and ENO derivatives (Eq. 33), the cell ghosts of the explicit method
beyond the z boundaries.

Each pin is a closed form:
- Uniform velocity (L = 0, stress below yield): sigma* = sigma - dt u.grad sigma,
  exact for a stress quadratic in x (at cells two or more from the periodic
  wrap) and for a stress linear in z (every layer, the wall layers included),
  for either sign of u.
- A simple-shear velocity v_x = g z + U with a stress affine in x and z:
  sigma* = sigma + dt (-(u.grad) sigma + L sigma + sigma L^T - tr(L) sigma)
  with u = v at the cell centre, against numpy matrix products, away from
  the x wrap.
- advect = False is the plain Eq. (27) bit for bit, and so is advect = True
  when the velocity is zero.
A dropped advection term, a wrong sign, the advecting velocity taken at a
corner instead of the cell centre, or a wrong ghost each fail one of these.
"""
import numpy as np
import pytest

import oracle as O
from paper_1904_03808_gb300 import inputs as I

MU = I.TABLE1["mu"]


def _stz():
    return O.STZ(**I.stz_values(0.0))


def _state(nx, ny, nz):
    v = np.zeros((3, nz + 1, ny, nx))
    sig = np.zeros((6, nz, ny, nx))
    chi = np.full((nz, ny, nx), 600.0)
    return v, sig, chi


@pytest.mark.parametrize("U", [0.7, -1.3])
def test_uniform_velocity_advects_quadratic_x_and_linear_z_stress(U):
    nx, ny, nz = 16, 4, 8
    h, dt = 1e-3, 1e-5
    p = _stz()
    v, sig, chi = _state(nx, ny, nz)
    v[0] = U
    xc = (np.arange(nx) + 0.5) * h
    qa, qb, qc = 3e9, -2e6, 5e5  # below yield everywhere
    sig[4] = (qa * xc * xc + qb * xc + qc)[None, None, :]
    ss, D, _ = O.stress_star(v, sig, chi, h, dt, MU, p, advect=True)
    assert not D.any()
    want = qa * xc * xc + qb * xc + qc - dt * U * (2 * qa * xc + qb)
    assert np.allclose(ss[4][:, :, 2:nx - 2], want[None, None, 2:nx - 2], rtol=1e-13)
    assert np.array_equal(ss[[0, 1, 2, 3, 5]], sig[[0, 1, 2, 3, 5]])
    # z, with both wall layers (linear ghosts continue the profile)
    v, sig, chi = _state(nx, ny, nz)
    v[2] = U
    zc = (np.arange(nz) + 0.5) * h
    sig[1] = (4e8 * zc + 7e5)[:, None, None]
    ss, _, _ = O.stress_star(v, sig, chi, h, dt, MU, p, advect=True)
    want = 4e8 * zc + 7e5 - dt * U * 4e8
    assert np.allclose(ss[1], want[:, None, None] * np.ones((1, ny, nx)), rtol=1e-13)


@pytest.mark.parametrize("g,U", [(300.0, 0.4), (-250.0, -0.6)])
def test_shear_flow_with_affine_stress_matches_the_closed_form(g, U):
    nx, ny, nz = 16, 4, 8
    h, dt = 1e-3, 1e-6
    p = _stz()
    v, sig, chi = _state(nx, ny, nz)
    z = np.arange(nz + 1) * h
    v[0] = (g * z + U)[:, None, None]
    zc = (np.arange(nz) + 0.5) * h
    xc = (np.arange(nx) + 0.5) * h
    # affine stress: sigma_c = a_c + bx_c x + bz_c z
    rng = np.random.default_rng(2)
    a, bx, bz = rng.normal(size=6) * 2e5, rng.normal(size=6) * 1e8, rng.normal(size=6) * 1e8
    for c in range(6):
        sig[c] = a[c] + bx[c] * xc[None, None, :] + bz[c] * zc[:, None, None]
    ss, D, _ = O.stress_star(v, sig, chi, h, dt, MU, p, advect=True)
    assert not D.any()
    L = np.zeros((3, 3))
    L[0, 2] = g
    idx = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
    for k in range(nz):
        ux = g * zc[k] + U  # the velocity at the cell centre
        for i in range(2, nx - 2):
            s = np.zeros((3, 3))
            for c, (r_, q_) in enumerate(idx):
                s[r_, q_] = s[q_, r_] = sig[c, k, 0, i]
            rate = L @ s + s @ L.T - np.trace(L) * s
            for c, (r_, q_) in enumerate(idx):
                want = s[r_, q_] + dt * (rate[r_, q_] - ux * bx[c])
                got = ss[c, k, 1, i]
                assert abs(got - want) <= 1e-12 * max(abs(want), 1.0), (c, k, i)


def test_advection_off_or_at_rest_is_plain_eq27():
    w = I.Workload(16, steps=10, strain=0.02, preload=1.2e9, seed=3)
    v, sig, chi, _ = w.initial_state()
    rng = np.random.default_rng(1)
    v[:, 1:w.nz] += 1e-3 * w.U_B * rng.normal(size=v[:, 1:w.nz].shape)
    sig += 5e7 * rng.normal(size=sig.shape)
    p = O.STZ(**w.stz)
    plain = O.stress_star(v, sig, chi, w.h, w.dt, MU, p)
    off = O.stress_star(v, sig, chi, w.h, w.dt, MU, p, advect=False)
    for x, y in zip(plain, off):
        assert np.array_equal(x, y)
    on = O.stress_star(v, sig, chi, w.h, w.dt, MU, p, advect=True)
    assert not np.array_equal(on[0], plain[0])  # the term is there
    assert np.array_equal(on[1], plain[1]) and np.array_equal(on[2], plain[2])
    v0 = np.zeros_like(v)
    a = O.stress_star(v0, sig, chi, w.h, w.dt, MU, p)
    b = O.stress_star(v0, sig, chi, w.h, w.dt, MU, p, advect=True)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
