"""Pins of the explicit-method oracle (section 3.2, Eqs. 24-26; ENO
advection, Eq. 33): each against a closed form the method must reproduce.

- ENO derivative: each of its three branches is exact on the quadratic it
  selects, and the branch goes to the smooth side (a planted wrong
  coefficient or a swapped upwind test fails these).
- Linearised elastic waves: a standing shear mode and a standing
  longitudinal mode between the walls evolve, step by step, by the scheme's
  own closed-form 2 x 2 amplification (staggered divergence and gradient of
  Eq. 31, the Laplacian damping of Eq. 32), which fixes the sign and size of
  div sigma / rho, of C:D (mu, lambda + 2 mu, lambda) and of kappa.
- Advection: a field quadratic in x is advected exactly at points away from
  the periodic wrap, and a field linear in z exactly up to the walls (the
  ghost extrapolation continues linear fields), for either sign of the
  velocity; velocity advected by velocity likewise.
- Uniform simple shear: a linear velocity profile with uniform stress and
  chi stays linear, and stress and chi follow a 0-D forward-Euler recursion
  of Eqs. 25-26 (elastic loading C:D, rotation terms, STZ relaxation).
- A general constant velocity gradient with a uniform stress: the closed
  form of Eq. 25's rate (the sign of the tr(L) term included).
- The reflected velocity ghosts beyond a wall: for a quadratic profile the
  corner next to the wall takes the one-sided stencil through the ghost.
Planting a wrong tr(L) sign, an even instead of odd wall reflection, a
swapped ENO upwind test, a wrong sign of div sigma or a wrong C:D factor in
the oracle each fails at least one of these tests.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1904_03808_gb300 import inputs as I

MU = I.TABLE1["mu"]
LAM = I.lame_lambda(I.TABLE1["K"], MU)
RHO = I.TABLE1["rho"]


# ------------------------------------------------------------------ ENO

@pytest.mark.parametrize("seed", range(5))
def test_eno_branches_exact_on_the_smooth_side(seed):
    rng = np.random.default_rng(seed)
    h = rng.uniform(0.3, 2.0)
    a, b, c = rng.normal(size=3)
    x = h * np.arange(-2, 3)
    q = a * x * x + b * x + c
    dq = b  # q'(0)
    kink = 3.0 * abs(a) * h * h + 1.0
    # u < 0: upwind side is +x; a kink at -h makes the centre rougher
    f = q.copy()
    f[1] += np.sign(a) * kink
    assert O.eno(f, -1.0, h) == pytest.approx(dq, abs=1e-12 * (1 + abs(dq)))
    # u > 0: upwind side is -x; a kink at +h
    f = q.copy()
    f[3] += np.sign(a) * kink
    assert O.eno(f, 1.0, h) == pytest.approx(dq, abs=1e-12 * (1 + abs(dq)))
    # upwind side rougher than the centre: the centred difference, exact on
    # the quadratic through -h, 0, h
    f = q.copy()
    f[4] += kink * 10.0
    assert O.eno(f, -1.0, h) == pytest.approx(dq, abs=1e-12 * (1 + abs(dq)))
    f = q.copy()
    f[0] += kink * 10.0
    assert O.eno(f, 1.0, h) == pytest.approx(dq, abs=1e-12 * (1 + abs(dq)))
    # no flow: centred
    assert O.eno(q, 0.0, h) == pytest.approx(dq, abs=1e-12 * (1 + abs(dq)))
    # a plain quadratic: every branch test fails, centred, exact
    assert O.eno(q, 1.0, h) == pytest.approx(dq, abs=1e-12 * (1 + abs(dq)))


def test_eno_one_sided_differs_from_centred_on_kinked_data():
    """The kinked cases above really exercise the one-sided stencils: on the
    same data the centred difference is off."""
    h = 1.0
    x = np.arange(-2, 3.0)
    q = x * x
    f = q.copy()
    f[1] += 5.0
    assert O.eno(f, -1.0, h) == pytest.approx(0.0, abs=1e-13)
    assert abs((f[3] - f[1]) / 2.0) > 1.0


# ------------------------------------------------------------ set-up helpers

def _stz(l=0.0):
    return O.STZ(**I.stz_values(l))


def _bc(U_B=0.0, t_ramp=1.0):
    return O.BC(kind=0, U_B=U_B, t_ramp=t_ramp, omega=0.0, R=1.0 / 3.0, lambda_w=1.0)


def _state(nx, ny, nz):
    v = np.zeros((3, nz + 1, ny, nx))
    sig = np.zeros((6, nz, ny, nx))
    chi = np.full((nz, ny, nx), 600.0)
    return v, sig, chi


# -------------------------------------------------------- linearised waves

@pytest.mark.parametrize("mode,m", [("shear", 1), ("shear", 3), ("longitudinal", 1),
                                    ("longitudinal", 2)])
def test_standing_wave_follows_the_discrete_amplification(mode, m):
    """Standing modes between the walls (zero wall velocity), uniform in x and
    y, with amplitudes small enough that the quadratic terms (rotation,
    advection) are below 1e-14 of the linear ones and the STZ rate is zero.
    With theta = pi m / nz, s = sin(theta / 2):
      a' = a - (2 dt / (rho h)) s b - (4 kappa dt / h^2) s^2 a,
      b' = b + (2 M dt / h) s a,
    for v_comp(k) = a sin(theta k) and sigma(k + 1/2) = b cos(theta (k + 1/2)),
    M = mu (shear: v_x, sigma_xz) or lambda + 2 mu (longitudinal: v_z,
    sigma_zz, with sigma_xx = sigma_yy following lambda)."""
    nx, ny, nz = 4, 4, 16
    h = 1.25e-3
    cp = math.sqrt((LAM + 2 * MU) / RHO)
    dt = 0.2 * h / cp
    kappa = 0.05 * h * h / dt
    theta = math.pi * m / nz
    s = math.sin(theta / 2)
    k = np.arange(nz + 1)
    kc = np.arange(nz) + 0.5
    a, b, c = 1e-11, 1e-4, 0.0
    v, sig, chi = _state(nx, ny, nz)
    comp_v, comp_s, M = (0, 4, MU) if mode == "shear" else (2, 2, LAM + 2 * MU)
    v[comp_v] = a * np.sin(theta * k)[:, None, None]
    sig[comp_s] = b * np.cos(theta * kc)[:, None, None]
    p, bc = _stz(), _bc()
    t = 1.0
    for _ in range(5):
        O.explicit_step(v, sig, chi, h, dt, RHO, LAM, MU, kappa, p, bc, t)
        t += dt
        a, b, c = (a - 2 * dt / (RHO * h) * s * b - 4 * kappa * dt / (h * h) * s * s * a,
                   b + 2 * M * dt / h * s * a,
                   c + 2 * LAM * dt / h * s * a)
        want_v = a * np.sin(theta * k)[:, None, None] * np.ones((1, ny, nx))
        want_s = b * np.cos(theta * kc)[:, None, None] * np.ones((1, ny, nx))
        assert np.allclose(v[comp_v], want_v, rtol=0, atol=1e-12 * abs(a))
        assert np.allclose(sig[comp_s], want_s, rtol=0, atol=1e-12 * abs(b))
        if mode == "longitudinal":
            want_c = c * np.cos(theta * kc)[:, None, None] * np.ones((1, ny, nx))
            for q in (0, 1):
                assert np.allclose(sig[q], want_c, rtol=0, atol=1e-12 * abs(c))
    assert np.all(chi == 600.0)


# ---------------------------------------------------------------- advection

@pytest.mark.parametrize("U", [1.3, -0.7])
def test_advection_of_stress_along_x_and_z(U):
    """Uniform velocity (L = 0): sigma' = sigma - dt (u.grad) sigma.  A stress
    quadratic in x is advected exactly at cells two or more away from the
    periodic wrap; one linear in z exactly in every layer, the wall layers
    included (linear ghost extrapolation)."""
    nx, ny, nz = 16, 4, 8
    h, dt = 1e-3, 1e-5
    p, bc = _stz(), _bc()
    # x
    v, sig, chi = _state(nx, ny, nz)
    v[0] = U
    xc = (np.arange(nx) + 0.5) * h
    qa, qb, qc = 3e6, -2e3, 50.0
    sig[0] = (qa * xc * xc + qb * xc + qc)[None, None, :]
    O.explicit_step(v, sig, chi, h, dt, RHO, LAM, MU, 0.0, p, bc, 0.0)
    want = qa * xc * xc + qb * xc + qc - dt * U * (2 * qa * xc + qb)
    assert np.allclose(sig[0][:, :, 2:nx - 2], want[None, None, 2:nx - 2], rtol=1e-13)
    # z
    v, sig, chi = _state(nx, ny, nz)
    v[2] = U
    zc = (np.arange(nz) + 0.5) * h
    sig[3] = (4e5 * zc + 7.0)[:, None, None]
    O.explicit_step(v, sig, chi, h, dt, RHO, LAM, MU, 0.0, p, bc, 0.0)
    want = 4e5 * zc + 7.0 - dt * U * 4e5
    assert np.allclose(sig[3], want[:, None, None] * np.ones((1, ny, nx)), rtol=1e-13)


@pytest.mark.parametrize("U", [0.9, -1.1])
def test_advection_and_damping_of_velocity(U):
    """v_x = U, v_y = g(x) quadratic, no stress: at corners away from the wrap
    v_y' = g - dt U g' + dt kappa g'' exactly; v_x = U, v_z = 0 stay.  A
    shear profile v_x linear in z advected by a uniform v_z: exact up to the
    walls (the reflected ghosts continue linear profiles)."""
    nx, ny, nz = 16, 4, 8
    h, dt, kappa = 1e-3, 1e-5, 2e-3
    p, bc = _stz(), _bc()
    v, sig, chi = _state(nx, ny, nz)
    x = np.arange(nx) * h
    ga, gb = 5e3, -3.0
    v[0] = U
    v[1] = (ga * x * x + gb * x)[None, None, :]
    O.explicit_step(v, sig, chi, h, dt, RHO, LAM, MU, kappa, p, bc, 0.0)
    want = ga * x * x + gb * x - dt * U * (2 * ga * x + gb) + dt * kappa * 2 * ga
    assert np.allclose(v[1][1:nz, :, 2:nx - 2], want[None, None, 2:nx - 2], rtol=1e-12)
    assert np.allclose(v[0][1:nz], U, rtol=1e-15) and np.all(v[2][1:nz] == 0.0)
    # z
    v, sig, chi = _state(nx, ny, nz)
    z = np.arange(nz + 1) * h
    v[0] = (2e2 * z - 0.3)[:, None, None]
    v[2] = U
    O.explicit_step(v, sig, chi, h, dt, RHO, LAM, MU, kappa, p, bc, 0.0)
    want = 2e2 * z - 0.3 - dt * U * 2e2
    assert np.allclose(v[0][1:nz], want[1:nz, None, None] * np.ones((1, ny, nx)), rtol=1e-12)


# ---------------------------------------------------- uniform simple shear

def _zero_d(sig6, chi, gdot, dt, steps, p):
    """0-D forward Euler of Eqs. 25-26 for a uniform state under L_xz = gdot."""
    L = np.zeros((3, 3))
    L[0, 2] = gdot
    Dm = 0.5 * (L + L.T)
    idx = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
    s = np.zeros((3, 3))
    for q, (i, j) in enumerate(idx):
        s[i, j] = s[j, i] = sig6[q]
    for _ in range(steps):
        s0 = s - np.trace(s) / 3 * np.eye(3)
        sb = math.sqrt(0.5 * np.sum(s0 * s0))
        D = O.dpl(p, sb, chi)
        rate = L @ s + s @ L.T - np.trace(L) * s + LAM * np.trace(Dm) * np.eye(3) + 2 * MU * Dm
        if D > 0:
            rate -= 2 * MU * D * s0 / sb
        chi = chi + dt / p.c0 * (2 * D * sb / p.sY * (p.chi_inf - chi))
        s = s + dt * rate
    return np.array([s[i, j] for i, j in idx]), chi


def test_uniform_simple_shear_reduces_to_zero_d():
    nx, ny, nz = 4, 4, 8
    h = 1e-3
    H = nz * h
    U = 2.0
    gdot = 2 * U / H
    dt = 2e-7
    p = _stz(h)
    bc = _bc(U_B=U, t_ramp=1e-9)
    v, sig, chi = _state(nx, ny, nz)
    z = (np.arange(nz + 1) - nz / 2) * h
    v[0] = (gdot * z)[:, None, None]
    sig[4] = 1.5e9
    sig[0] = 2e8
    chi[:] = 620.0
    t = 1e-6
    steps = 6
    for _ in range(steps):
        O.explicit_step(v, sig, chi, h, dt, RHO, LAM, MU, 0.1, p, bc, t)
        t += dt
    s_want, chi_want = _zero_d([2e8, 0, 0, 0, 1.5e9, 0], 620.0, gdot, dt, steps, p)
    assert chi_want > 620.0 + 1e-9  # the STZ rate is active
    assert np.allclose(v[0], (gdot * z)[:, None, None], rtol=1e-13, atol=1e-13 * U)
    assert np.all(v[1] == 0.0) and np.all(v[2] == 0.0)
    for q in range(6):
        assert np.allclose(sig[q], s_want[q], rtol=1e-12, atol=1e-6), q
    assert np.allclose(chi, chi_want, rtol=1e-13)


def test_constant_velocity_gradient_and_uniform_stress():
    """v = L x with a general constant L (no wall of its own: the walls carry
    the same field) and a uniform stress below yield: the advection of the
    uniform stress vanishes, and in every cell whose corners do not wrap
    sigma' = sigma + dt (L sigma + sigma L^T - tr(L) sigma + C:D); a wrong
    sign of the tr(L) term or of C:D fails this."""
    nx, ny, nz = 8, 8, 6
    h, dt = 1e-3, 1e-6
    rng = np.random.default_rng(2)
    L = rng.normal(size=(3, 3)) * 10.0
    v, sig, chi = _state(nx, ny, nz)
    kk, jj, ii = np.meshgrid(np.arange(nz + 1), np.arange(ny), np.arange(nx), indexing="ij")
    X = np.stack([ii * h, jj * h, kk * h])
    for a in range(3):
        v[a] = sum(L[a, b] * X[b] for b in range(3))
    s = rng.normal(size=(3, 3)) * 1e7
    s = 0.5 * (s + s.T)
    idx = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
    for q, (i, j) in enumerate(idx):
        sig[q] = s[i, j]
    O.explicit_step(v, sig, chi, h, dt, RHO, LAM, MU, 0.0, _stz(), _bc(), 0.0)
    Dm = 0.5 * (L + L.T)
    want = s + dt * (L @ s + s @ L.T - np.trace(L) * s + LAM * np.trace(Dm) * np.eye(3) + 2 * MU * Dm)
    for q, (i, j) in enumerate(idx):
        assert np.allclose(sig[q][:, :ny - 1, :nx - 1], want[i, j], rtol=1e-12, atol=1e-12 * abs(want).max())


@pytest.mark.parametrize("W", [0.8, -0.8])
def test_wall_ghost_of_the_velocity(W):
    """The ghost corners beyond a wall reflect v through the wall value,
    v(-m) = 2 v(0) - v(m), so the curvature at the wall vanishes; for a
    profile v_x = q(z) quadratic advected towards the interior by v_z = W the
    ENO derivative at the corner next to the wall takes the one-sided
    upwind stencil through the ghost, which reduces to (q(h) - q(0)) / h
    (bottom, W > 0) or (q(H) - q(H - h)) / h (top, W < 0); elsewhere the
    centred difference, exact on the quadratic."""
    nx, ny, nz = 4, 4, 8
    h, dt, kappa = 1e-3, 1e-5, 0.0
    v, sig, chi = _state(nx, ny, nz)
    z = np.arange(nz + 1) * h
    qa, qb = 4e4, 3.0
    q = qa * z * z + qb * z
    v[0] = q[:, None, None]
    v[2] = W
    O.explicit_step(v, sig, chi, h, dt, RHO, LAM, MU, kappa, _stz(), _bc(), 0.0)
    d = 2 * qa * z + qb
    if W > 0:
        d[1] = (q[1] - q[0]) / h
    else:
        d[nz - 1] = (q[nz] - q[nz - 1]) / h
    want = q - dt * W * d
    assert np.allclose(v[0][1:nz], want[1:nz, None, None] * np.ones((1, ny, nx)), rtol=1e-13)
